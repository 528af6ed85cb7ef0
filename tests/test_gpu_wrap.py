"""Parity at sizes where every persistent tensor-core kernel cycles its pipelines.

The label kernels run one CTA per SM (152 on GB300) over 128-point tiles (TF32,
multinomial) or 256-point passes (split BF16), with a ring of X stages and
double-buffered TMEM accumulators whose mbarrier phases flip every time a stage or
buffer is reused.  At the small sizes of the other parity tests no CTA gets past its
first one or two tiles, so the phase logic of the later passes is never exercised.
Here N = 160,001 points:
  - TF32 (d = 32, 3 X stages, 2 TMEM buffers): 1,251 tiles, 8 or 9 tiles per CTA, the
    stage ring wraps 2-3 times and each TMEM buffer is reused about 4 times per chunk;
  - split BF16 (d = 128, K = 64): 626 passes of two tiles, 4 or 5 passes per CTA;
  - multinomial BF16 (d = 200, K = 50, four 128-byte atoms per row, 8-slot atom ring):
    8 or 9 tiles per CTA, 33-36 atom loads, the ring wraps 4 times;
with the last tile ragged (160,001 = 1,250 x 128 + 1).  Labels and sub-labels are
compared with the FP64 oracle on the same parameters and Philox keys, within the
budgets of the smaller tests (labels 1e-3, sub-labels 1e-2).  The statistics are
compared with an FP64 recount of the GPU's own labels at the benchmark's size
(TF32, d = 32, N = 1e6: about 6,600 points per range) and at N = 2e6 for split BF16
at d = 128, so every FP32 range sum is as long as at full size."""
import numpy as np
import pytest
from scipy import stats

import oracle as O

pytestmark = pytest.mark.gpu
P = None
N_WRAP = 160_001


@pytest.fixture(scope="module", autouse=True)
def gpu():
    global P
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2204_08988_gb300 as mod

    P = mod


def _prior(d):
    return dict(kappa0=1.0, m0=np.zeros(d), nu0=float(d + 3), psi0=np.eye(d))


def _gauss_pair(N, d, K, seed, prec, K_max=64, mean_scale=5.0):
    import synth

    X, y = synth.gaussian_mixture(N, d, K, mean_scale, seed=seed)
    o = O.Oracle(O.NIW, d, K_max, 3.0, **_prior(d))
    o.set_data(X.astype(np.float64))
    zb = (np.arange(N) % 2).astype(np.uint8)
    o.set_state(K, y, zb)
    o.draw_params(seed)
    p = o.params()
    g = P.DPMM(0, d, K_max, 3.0, prec=prec, **_prior(d))
    g.set_data(X)
    g.set_state(K, y, zb)
    g.set_params(K, p)
    return X, o, g, p


def _compare_sampled(o, g, seed, n_sample, rng_seed):
    """One label step on the GPU (all points) against the oracle's step at the same
    sweep index on a random sample of the points (the oracle's streams are keyed by
    the global point index, so a sample sees the same random numbers)."""
    K, it = g.info()
    g.set_mask(2)
    g.sweep(1, seed)
    assert g.K == K  # no cluster emptied (ids would be compacted and no longer comparable)
    zg, zbg = g.labels()
    idx = np.sort(np.random.default_rng(rng_seed).choice(len(zg), size=min(n_sample, len(zg)), replace=False))
    idx = np.union1d(idx, [0, len(zg) - 1])  # the first point and the ragged last tile
    zo, zbo = o.label_probe_points(seed, it, idx)
    dz = (zo != zg[idx]).mean()
    same = zo == zg[idx]
    dzb = (zbo[same] != zbg[idx][same]).mean()
    return dz, dzb, len(idx)


@pytest.mark.parametrize("K", [20, 26, 27])
def test_tc_labels_wrap(K):
    """TF32 at d = 32: K = 20 (the benchmark's cluster count), K = 26, the most clusters
    whose factors fit the kernel's shared memory at K_max = 64, and K = 27 (two groups)."""
    X, o, g, p = _gauss_pair(N_WRAP, 32, K, seed=400 + K, prec=P.PREC_TF32)
    dz, dzb, n = _compare_sampled(o, g, 77, 40_000, K)
    assert dz < 1e-3, dz
    assert dzb < 1e-2, dzb
    g.close()


def test_tc_scores_wrap():
    """Every score of every point at N = 160,001 (K = 26, one full group of factors)
    against FP64: the budgets of the small-size test, and empty-cluster scores (-inf)
    exactly where FP64 has them."""
    K = 26
    X, o, g, p = _gauss_pair(N_WRAP, 32, K, seed=427, prec=P.PREC_TF32)
    s_tc = g.label_scores()
    s_64 = np.empty_like(s_tc)
    for k in range(K):
        W = p["W"][3 * k]
        s_64[:, k] = p["logw"][3 * k] + stats.multivariate_normal(p["mu"][3 * k], np.linalg.inv(W @ W.T)).logpdf(
            X.astype(np.float64))
    assert np.array_equal(np.isneginf(s_tc), np.isneginf(s_64))
    fin = np.isfinite(s_64)
    err = np.where(fin, np.abs(s_tc - np.where(fin, s_64, 0.0)), 0.0)
    cont = fin & (s_64 >= s_64.max(1, keepdims=True) - 20.0)
    assert err[cont].mean() < 0.02, err[cont].mean()
    assert np.quantile(err[cont], 0.99) < 0.1
    assert err[cont].max() < 0.5, err[cont].max()
    assert (err[fin] / np.maximum(1.0, np.abs(s_64[fin]))).max() < 0.01
    g.close()


def test_x3_labels_wrap():
    """Split BF16 at d = 128 with K = 64 clusters streamed through the factor stages:
    4 or 5 passes of 256 points per CTA."""
    X, o, g, p = _gauss_pair(N_WRAP, 128, 64, seed=464, prec=P.PREC_BF16X3, K_max=128, mean_scale=4.0)
    dz, dzb, n = _compare_sampled(o, g, 91, 4_000, 5)
    assert dz < 1e-3 + 3.0 / n, dz
    assert dzb < 1e-2 + 3.0 / n, dzb
    g.close()


def test_mult_labels_wrap():
    """Multinomial BF16 at d = 200, K = 50 (the benchmark's shape): the 8-slot atom ring
    wraps about four times per CTA."""
    import synth

    N, d, K = N_WRAP, 200, 50
    X, y = synth.multinomial_mixture(N, d, K, 100, seed=450)
    o = O.Oracle(O.DIRICHLET, d, 64, 3.0, beta=np.ones(d))
    o.set_data(X.astype(np.float64))
    zb = (np.arange(N) % 2).astype(np.uint8)
    o.set_state(K, y, zb)
    o.draw_params(450)
    g = P.DPMM(1, d, 64, 3.0, prec=P.PREC_BF16, beta=np.ones(d))
    g.set_data(X)
    g.set_state(K, y, zb)
    g.set_params(K, o.params())
    dz, dzb, n = _compare_sampled(o, g, 55, 40_000, 9)
    assert dz < 1e-3, dz
    assert dzb < 1e-2, dzb
    g.close()


def _round_tf32(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    fin = (u & 0x7F800000) != 0x7F800000
    return np.where(fin, (u + np.uint32(0x1000)) & np.uint32(0xFFFFE000), u).view(np.float32)


def _recount_check(X64, z, zb, n, sx, sxx, K, atol1, atol2):
    """Counts exact; sums and sums of outer products against an FP64 recount of the
    given labels (points grouped by slot once, then one product per slot)."""
    assert n[0::3].sum() == len(z) and np.array_equal(n[0::3], n[1::3] + n[2::3])
    key = 2 * z.astype(np.int64) + zb
    order = np.argsort(key, kind="stable")
    bounds = np.searchsorted(key[order], np.arange(2 * K + 1))
    for k in range(K):
        for h in range(2):
            a, b = bounds[2 * k + h], bounds[2 * k + h + 1]
            Xs = X64[order[a:b]]
            s = 3 * k + 1 + h
            assert n[s] == b - a, (k, h)
            c = max(1, b - a)
            assert np.allclose(sx[s], Xs.sum(0), rtol=1e-5, atol=atol1 * c ** 0.5), (k, h)
            assert np.allclose(sxx[s], Xs.T @ Xs, rtol=1e-5, atol=atol2 * c ** 0.5), (k, h)


def test_tc_statistics_full_size():
    """TF32 statistics at the benchmark's workload (d = 32, N = 1e6, from the
    generating labels, two full sweeps) against an FP64 recount of the GPU's labels."""
    import synth

    X, y, prior, opt = synth.workload("gauss_d32", seed=1002)
    N, d = X.shape
    kw = {k: v for k, v in prior.items() if k != "kind"}
    g = P.DPMM(0, d, 64, opt["alpha"], prec=P.PREC_TF32, burn_out=15, **kw)
    g.set_data(X)
    g.set_state(int(y.max()) + 1, y, (np.arange(N) % 2).astype(np.uint8))
    g.sweep(2, 0)
    K = g.K
    z, zb = g.labels()
    n, sx, sxx = g.stats()
    c = X.astype(np.float64).mean(0)
    X64 = _round_tf32((X.astype(np.float64) - c).astype(np.float32)).astype(np.float64) + c
    _recount_check(X64, z, zb, n, sx, sxx, K, 1e-3, 1e-2)
    g.close()


def test_x3_statistics_two_million_points():
    """Split BF16 path at d = 128 (FP32 sub-label and statistics kernel) on 2e6 points
    of the d = 128 workload's generator (64 clusters), two full sweeps from the
    generating labels, against an FP64 recount."""
    import synth

    N, d, K0 = 2_000_000, 128, 64
    X, y = synth.gaussian_mixture(N, d, K0, 4.0, seed=1004)
    g = P.DPMM(0, d, 128, 100.0, prec=P.PREC_BF16X3, burn_out=15, **_prior(d))
    g.set_data(X)
    g.set_state(K0, y, (np.arange(N) % 2).astype(np.uint8))
    g.sweep(2, 0)
    K = g.K
    z, zb = g.labels()
    n, sx, sxx = g.stats()
    _recount_check(X.astype(np.float64), z, zb, n, sx, sxx, K, 1e-2, 1e-1)
    g.close()
