"""The allocation-free statistics entry point against the library's ordinary path.

dpmm_suffstats_noalloc exists for callers that cannot allocate device memory where
they need sufficient statistics (inside a stream capture, or under an allocator that
forbids later allocation).  It must give the same counts, sums and sums of outer
products as dpmm_set_state + dpmm_get_stats, within the FP32 tolerance used by the
other FP32 statistics tests, on two calls in a row (the second with other labels,
so stale scratch from the first call would show)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _reference(P, X, K, z, zb):
    g = P.DPMM(P.PRIOR_NIW, X.shape[1], 16, 1.0, prec=P.PREC_FP32, psi0=np.eye(X.shape[1]))
    g.set_data(X)
    g.set_state(K, z, zb)
    n, sx, sxx = g.stats()
    g.close()
    sub = np.array([3 * k + 1 + h for k in range(K) for h in range(2)])
    return n[sub], sx[sub], sxx[sub]


def test_noalloc_statistics_match_ordinary_path():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2204_08988_gb300 as P
    import synth

    N, d = 100_003, 8
    X, y = synth.gaussian_mixture(N, d, 5, 4.0, seed=71)
    rng = np.random.default_rng(3)
    cases = [(5, y.astype(np.int32), rng.integers(0, 2, N).astype(np.uint8)),
             (3, rng.integers(0, 3, N).astype(np.int32), rng.integers(0, 2, N).astype(np.uint8))]
    Xd = torch.from_numpy(X).cuda()
    for K, z, zb in cases:
        zd = torch.from_numpy(z).cuda()
        zbd = torch.from_numpy(zb).cuda()
        n_out = torch.full((2 * K,), -1.0, dtype=torch.float64, device="cuda")
        sx_out = torch.full((2 * K, d), -1.0, dtype=torch.float64, device="cuda")
        sxx_out = torch.full((2 * K, d, d), -1.0, dtype=torch.float64, device="cuda")
        P.dpmm_suffstats_noalloc(Xd, zd, zbd, K, n_out, sx_out, sxx_out)
        torch.cuda.synchronize()
        n_ref, sx_ref, sxx_ref = _reference(P, X, K, z, zb)
        n, sx, sxx = n_out.cpu().numpy(), sx_out.cpu().numpy(), sxx_out.cpu().numpy()
        assert np.array_equal(n, n_ref)
        for s in range(2 * K):
            tol = max(1.0, n[s]) ** 0.5
            assert np.allclose(sx[s], sx_ref[s], rtol=1e-5, atol=1e-2 * tol)
            assert np.allclose(sxx[s], sxx_ref[s], rtol=1e-5, atol=1e-1 * tol)


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
