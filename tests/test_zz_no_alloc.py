"""The allocation-free statistics entry point against the library's ordinary path.

dpmm_suffstats_noalloc serves callers that cannot allocate device memory where they
need sufficient statistics: an application that reserves the GPU's memory up front in
its own pool and forbids later cudaMalloc, or latency-critical code that must not take
the device-wide synchronisation an allocation can cause.  It must give the same
counts, sums and sums of outer products as the ordinary path (dpmm_set_state +
dpmm_get_stats on the same points and labels), within the FP32 tolerance the other
FP32 statistics tests use, and agree with an FP64 recount in numpy.  Each case makes
two calls in a row, the second with other labels, so stale scratch from the first
call would show; labels outside [0, K) x {0, 1} must be ignored.  The sizes cover
d = 1, the largest d and K it takes (32, 16: the fixed scratch is exactly full) and a
middle case.  This file is collected last so that a failure here leaves every other
test already run."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ordinary_path(P, X, K, z, zb):
    g = P.DPMM(P.PRIOR_NIW, X.shape[1], 16, 1.0, prec=P.PREC_FP32, psi0=np.eye(X.shape[1]))
    g.set_data(X)
    g.set_state(K, z, zb)
    n, sx, sxx = g.stats()
    g.close()
    sub = np.array([3 * k + 1 + h for k in range(K) for h in range(2)])
    return n[sub], sx[sub], sxx[sub]


def _recount(X, K, z, zb):
    d = X.shape[1]
    X64 = X.astype(np.float64)
    n = np.zeros(2 * K)
    sx = np.zeros((2 * K, d))
    sxx = np.zeros((2 * K, d, d))
    for k in range(K):
        for h in range(2):
            sel = (z == k) & (zb == h)
            n[2 * k + h] = sel.sum()
            sx[2 * k + h] = X64[sel].sum(0)
            sxx[2 * k + h] = X64[sel].T @ X64[sel]
    return n, sx, sxx


def _close(a, b, n):
    for s in range(len(n)):
        tol = max(1.0, n[s]) ** 0.5
        assert np.allclose(a[0][s], b[0][s], rtol=1e-5, atol=1e-2 * tol), s
        assert np.allclose(a[1][s], b[1][s], rtol=1e-5, atol=1e-1 * tol), s


@pytest.mark.parametrize("d,K", [(8, 5), (1, 1), (32, 16)])
def test_noalloc_statistics_match_ordinary_path(d, K):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2204_08988_gb300 as P
    import synth

    N = 100_003
    X, y = synth.gaussian_mixture(N, d, K, 4.0, seed=71 + d)
    rng = np.random.default_rng(3 + d)
    z2 = rng.integers(0, K, N).astype(np.int32)
    zb2 = rng.integers(0, 2, N).astype(np.uint8)
    # labels the entry point must ignore: a cluster id of K and a sub-label of 2
    bad = rng.choice(N, size=257, replace=False)
    z2[bad[:128]] = K
    zb2[bad[128:]] = 2
    cases = [(y.astype(np.int32) % K, rng.integers(0, 2, N).astype(np.uint8)), (z2, zb2)]
    Xd = torch.from_numpy(X).cuda()
    for z, zb in cases:
        zd = torch.from_numpy(z).cuda()
        zbd = torch.from_numpy(zb).cuda()
        n_out = torch.full((2 * K,), -1.0, dtype=torch.float64, device="cuda")
        sx_out = torch.full((2 * K, d), -1.0, dtype=torch.float64, device="cuda")
        sxx_out = torch.full((2 * K, d, d), -1.0, dtype=torch.float64, device="cuda")
        P.dpmm_suffstats_noalloc(Xd, zd, zbd, K, n_out, sx_out, sxx_out)
        torch.cuda.synchronize()
        n, sx, sxx = n_out.cpu().numpy(), sx_out.cpu().numpy(), sxx_out.cpu().numpy()
        ok = (z < K) & (zb <= 1)
        n_ref, sx_ref, sxx_ref = _ordinary_path(P, X[ok], K, z[ok], zb[ok])
        assert np.array_equal(n, n_ref)
        _close((sx, sxx), (sx_ref, sxx_ref), n)
        n_rc, sx_rc, sxx_rc = _recount(X, K, z, zb)
        assert np.array_equal(n, n_rc)
        _close((sx, sxx), (sx_rc, sxx_rc), n)


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2204_08988_gb300 as P

    X = torch.zeros((10, 33), dtype=torch.float32, device="cuda")
    z = torch.zeros(10, dtype=torch.int32, device="cuda")
    zb = torch.zeros(10, dtype=torch.uint8, device="cuda")
    out = torch.zeros(2 * 33 * 33 * 20, dtype=torch.float64, device="cuda")
    with pytest.raises(P.DPMMError) as e:
        P.dpmm_suffstats_noalloc(X, z, zb, 2, out, out, out)
    assert e.value.status == P.DPMM_EINVAL
    X = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(P.DPMMError) as e:
        P.dpmm_suffstats_noalloc(X, z, zb, 17, out, out, out)
    assert e.value.status == P.DPMM_EINVAL
    # the binding refuses a wrong dtype before the call
    with pytest.raises(ValueError):
        P.dpmm_suffstats_noalloc(X.double(), z, zb, 2, out, out, out)
