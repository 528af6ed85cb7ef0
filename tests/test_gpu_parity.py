"""CUDA path against the FP64 oracle, through the C ABI, on the same seeded inputs
and Philox keys.

FP64-plain: labels and counts bit-exact (a mismatch is allowed only where the
oracle's top two perturbed scores are within 1e-9 relative: a near tie, counted);
statistics and parameters to 1e-10 relative.  FP32: agreement with FP64 labels
measured against a stated budget.  Sizes span several 256-point tiles with ragged
tails, plus the degenerate cases (N=1, d=1, K=1, K at K_max)."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

P = None


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
    return mod


def _niw_prior(d, nu0=None):
    return dict(kappa0=1.0, m0=np.zeros(d), nu0=float(d + 3) if nu0 is None else nu0, psi0=np.eye(d))


def _pair(kind, d, K_max, alpha, X, prec=0, init_K=1, burn_out=2, **prior):
    okind = O.NIW if kind == 0 else O.DIRICHLET
    o = O.Oracle(okind, d, K_max, alpha, init_K=init_K, burn_out=burn_out, **prior)
    g = P.DPMM(kind, d, K_max, alpha, prec=prec, init_K=init_K, burn_out=burn_out, **prior)
    o.set_data(X.astype(np.float64))
    g.set_data(X)
    return o, g


def _perturbed_gap(o, X, seed, it, i, p):
    """Relative gap between the top two perturbed cluster scores of point i (numpy)."""
    from scipy import stats

    K = len(p["logw"]) // 3
    v = []
    for k in range(K):
        w = O.philox4x32_10([i, it, (5 << 24) | (k // 2), 0], [seed & 0xFFFFFFFF, seed >> 32])
        u = O.u01(w[0], w[1]) if k % 2 == 0 else O.u01(w[2], w[3])
        if "W" in p:
            S = np.linalg.inv(p["W"][3 * k] @ p["W"][3 * k].T)
            ll = stats.multivariate_normal(p["mu"][3 * k], S).logpdf(X[i])
        else:
            ll = X[i] @ p["logtheta"][3 * k]
        v.append(p["logw"][3 * k] + ll - np.log(-np.log(u)))
    v = np.sort(v)[::-1]
    return (v[0] - v[1]) / max(1.0, abs(v[0]))


def _check_stats(o, g, rtol=1e-10):
    no, sxo, sxxo = o.stats()
    ng, sxg, sxxg = g.stats()
    assert np.array_equal(no, ng)
    scale = np.abs(sxo).max() + 1.0
    assert np.abs(sxg - sxo).max() <= rtol * scale * max(1.0, no.max())
    if sxxo is not None:
        scale2 = np.abs(sxxo).max() + 1.0
        assert np.abs(sxxg - sxxo).max() <= rtol * scale2


@pytest.mark.parametrize("N,d,K", [(1000, 2, 3), (2049, 5, 4), (777, 1, 2)])
def test_label_step_fp64_matches_oracle(N, d, K):
    """Steps (e), (f) with the oracle's parameters injected: labels bit-exact."""
    import synth

    X, y = synth.gaussian_mixture(N, d, K, 4.0, seed=100 + N, dtype=np.float64)
    prior = _niw_prior(d)
    o, g = _pair(0, d, 16, 3.0, X, **prior)
    zb0 = (np.arange(N) % 2).astype(np.uint8)
    o.set_state(K, y, zb0)
    g.set_state(K, y, zb0)
    _check_stats(o, g)
    seed, it = 0x1234_5678_9ABC, 7
    o.iter = it
    o.draw_params(seed)
    p = o.params()
    g.set_params(K, p)
    g.set_iter(it)
    g.set_mask(2)
    o.sweep(1, seed, mask=O.MASK_LABELS)
    g.sweep(1, seed)
    zo, zbo = o.labels()
    zg, zbg = g.labels()
    assert o.K == g.K
    bad = np.nonzero((zo != zg) | (zbo != zbg))[0]
    for i in bad:  # only near ties may differ
        assert _perturbed_gap(o, X, seed, it, i, p) < 1e-9, i
    assert len(bad) <= 2
    if len(bad) == 0:
        _check_stats(o, g)


def test_param_draws_fp64_match_oracle():
    """Steps (a)-(d): weights, sub-weights, NIW draws from identical statistics."""
    import synth

    N, d, K = 3000, 4, 3
    X, y = synth.gaussian_mixture(N, d, K, 5.0, seed=5, dtype=np.float64)
    prior = _niw_prior(d)
    o, g = _pair(0, d, 16, 2.0, X, **prior)
    zb0 = (np.arange(N) % 3 == 0).astype(np.uint8)
    o.set_state(K, y, zb0)
    g.set_state(K, y, zb0)
    o.iter = 3
    g.set_iter(3)
    o.draw_params(99)
    g.set_mask(1)
    g.sweep(1, 99)
    po, pg = o.params(), g.params()
    for key in ("logw", "mu", "W", "logdetW"):
        a, b = po[key], pg[key]
        assert np.allclose(a, b, rtol=1e-10, atol=1e-10), (key, np.abs(a - b).max())


@pytest.mark.parametrize("prec,d", [("fp32", 8), ("tf32", 32)])
def test_param_draws_reduced_precision(prec, d):
    """Steps (c), (d) on the reduced-precision paths: the NIW factorisation and solves
    run in FP32, and a slot whose pivots lose more than 10 of their 24 bits to
    cancellation is redone in FP64.  Every slot is checked against the oracle's draw
    from the GPU's own statistics and the same Philox stream: the well-conditioned
    clusters to FP32 accuracy, the ill-conditioned one (two coordinates equal up to
    1e-3 noise) to FP64 accuracy, which only the FP64 retry reaches."""
    import synth

    N, K, it, seed = 4000, 4, 3, 99
    X, y = synth.gaussian_mixture(N, d, K, 5.0, seed=21)
    X = X.astype(np.float32)
    sel = y == 0
    rng = np.random.default_rng(3)
    X[sel, 0] *= 10.0  # pivot 1 of Psi_n ~ 2 against a diagonal ~ 1e4
    X[sel, 1] = X[sel, 0] + (1e-3 * rng.standard_normal(sel.sum())).astype(np.float32)
    prior = _niw_prior(d)
    pr = P.PREC_FP32 if prec == "fp32" else P.PREC_TF32
    g = P.DPMM(0, d, 16, 2.0, prec=pr, **prior)
    g.set_data(X)
    zb0 = (np.arange(N) % 3 == 0).astype(np.uint8)
    g.set_state(K, y, zb0)
    g.set_iter(it)
    g.set_mask(1)
    g.sweep(1, seed)
    n, sx, sxx = g.stats()
    pg = g.params()
    g.close()
    o = O.Oracle(O.NIW, d, 16, 2.0, **prior)
    for s in range(3 * K):
        kn, mn, nun, psin = o.niw_posterior(n[s], sx[s], sxx[s])
        W, mu, ld = o.niw_draw(seed, it, s, kn, mn, nun, psin)
        ew = np.abs(pg["W"][s] - W).max() / np.abs(W).max()
        em = np.abs(pg["mu"][s] - mu).max() / (1.0 + np.abs(mu).max())
        el = abs(pg["logdetW"][s] - ld)
        tol = 1e-8 if s < 3 else 1e-4  # cluster 0 (slots 0-2) is the ill-conditioned one
        assert ew < tol and em < tol and el < 100 * tol, (s, ew, em, el)


@pytest.mark.parametrize("kind", [0, 1])
def test_full_sweeps_fp64_match_oracle(kind):
    """Whole sweeps (params, labels, statistics, splits, merges) from K=1."""
    import synth

    if kind == 0:
        d = 3
        X, _ = synth.gaussian_mixture(4001, d, 4, 6.0, seed=21, dtype=np.float64)
        prior = _niw_prior(d)
    else:
        d = 12
        X, _ = synth.multinomial_mixture(3001, d, 4, 40, seed=22)
        prior = dict(beta=np.ones(d))
    o, g = _pair(kind, d, 12, 5.0, X, burn_out=2, **prior)
    splits = 0
    for t in range(25):
        o.sweep(1, 31)
        g.sweep(1, 31)
        assert o.K == g.K, t
        zo, zbo = o.labels()
        zg, zbg = g.labels()
        assert np.array_equal(zo, zg) and np.array_equal(zbo, zbg), t
        _check_stats(o, g)
        co, cg = o.counters(), g.counters()
        assert co == cg, (t, co, cg)
        splits += co["splits"]
    assert splits >= 2 and g.K >= 3


def test_many_clusters_split_merge_fp64_match_oracle():
    """Whole FP64 sweeps from 40 random clusters (K_max = 64): the split and merge
    bookkeeping runs over two chunks of 32 clusters (prefix counts carried from one chunk
    to the next), and the merge walk over the bit masks of 40 clusters; K, labels,
    statistics and counters must match the oracle at every sweep."""
    import synth

    d = 2
    X, _ = synth.gaussian_mixture(6000, d, 5, 6.0, seed=71, dtype=np.float64)
    o, g = _pair(0, d, 64, 5.0, X, init_K=40, burn_out=0, **_niw_prior(d))
    merges = 0
    for t in range(6):
        o.sweep(1, 57)
        g.sweep(1, 57)
        assert o.K == g.K, t
        zo, zbo = o.labels()
        zg, zbg = g.labels()
        assert np.array_equal(zo, zg) and np.array_equal(zbo, zbg), t
        _check_stats(o, g)
        co, cg = o.counters(), g.counters()
        assert co == cg, (t, co, cg)
        merges += co["merges"]
    assert merges >= 1


def test_k_max_saturation_counts_rejections():
    import synth

    d = 2
    X, _ = synth.gaussian_mixture(3000, d, 6, 10.0, seed=3, dtype=np.float64)
    o, g = _pair(0, d, 2, 5.0, X, burn_out=0, **_niw_prior(d))
    rej = 0
    for t in range(20):
        o.sweep(1, 8)
        g.sweep(1, 8)
        assert o.K == g.K <= 2
        assert o.counters() == g.counters()
        rej += g.counters()["split_rejected_kmax"]
    assert rej > 0


@pytest.mark.parametrize("N", [1, 2, 255, 256, 257])
def test_tiny_and_ragged_sizes(N):
    import synth

    d = 2
    X, _ = synth.gaussian_mixture(N, d, 2, 3.0, seed=N, dtype=np.float64)
    o, g = _pair(0, d, 8, 1.0, X, burn_out=0, **_niw_prior(d))
    for t in range(6):
        o.sweep(1, 4)
        g.sweep(1, 4)
        assert o.K == g.K
        assert all(np.array_equal(a, b) for a, b in zip(o.labels(), g.labels()))
        _check_stats(o, g)


@pytest.mark.parametrize("init_K", [1, 5])
def test_invariants_large_fp32(init_K):
    """FP32 path at 200k points: invariants and statistics against a numpy recount
    of the GPU's own labels."""
    import synth

    N, d = 200_003, 8
    X, _ = synth.gaussian_mixture(N, d, 6, 6.0, seed=9)
    g = P.DPMM(0, d, 32, 10.0, prec=P.PREC_FP32, init_K=init_K, burn_out=3, **_niw_prior(d))
    g.set_data(X)
    X64 = X.astype(np.float64)
    for t in range(12):
        g.sweep(1, 17)
    K = g.K
    z, zb = g.labels()
    n, sx, sxx = g.stats()
    assert z.min() >= 0 and z.max() < K and zb.max() <= 1
    assert n[0::3].sum() == N and np.all(n[0::3] > 0)
    assert np.array_equal(n[0::3], n[1::3] + n[2::3])
    for k in range(K):
        for h in range(2):
            sel = (z == k) & (zb == h)
            assert n[3 * k + 1 + h] == sel.sum()
            ref1 = X64[sel].sum(0)
            ref2 = X64[sel].T @ X64[sel]
            assert np.allclose(sx[3 * k + 1 + h], ref1, rtol=1e-5, atol=1e-2 * max(1, sel.sum()) ** 0.5)
            assert np.allclose(sxx[3 * k + 1 + h], ref2, rtol=1e-5, atol=1e-1 * max(1, sel.sum()) ** 0.5)
    g.close()


def test_fp32_labels_agree_with_fp64():
    """Reduced precision (FP32 CUDA cores) against the FP64 path on the same state,
    parameters and keys: label disagreement within budget."""
    import synth

    N, d, K = 50_000, 8, 5
    X, y = synth.gaussian_mixture(N, d, K, 5.0, seed=44)
    prior = _niw_prior(d)
    o = O.Oracle(O.NIW, d, 16, 3.0, **prior)
    o.set_data(X.astype(np.float64))
    zb0 = (np.arange(N) % 2).astype(np.uint8)
    o.set_state(K, y, zb0)
    o.draw_params(5)
    p = o.params()
    g = P.DPMM(0, d, 16, 3.0, prec=P.PREC_FP32, **prior)
    g.set_data(X)
    g.set_state(K, y, zb0)
    g.set_params(K, p)
    g.set_mask(2)
    g.sweep(1, 5)
    o.sweep(1, 5, mask=O.MASK_LABELS)
    zo, zbo = o.labels()
    zg, zbg = g.labels()
    assert (zo != zg).mean() < 1e-3
    assert (zbo != zbg).mean() < 1e-2


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_graph_replay_matches_eager(prec):
    """Sweeps on an explicit stream are replayed from a captured CUDA graph; the chain
    must be identical to the eager one (legacy default stream)."""
    import torch
    import synth

    d = 8 if prec == "fp64" else 32
    X, _ = synth.gaussian_mixture(20_001, d, 5, 6.0, seed=12)
    pr = P.PREC_FP64_PLAIN if prec == "fp64" else P.PREC_TF32
    s = torch.cuda.Stream()
    ge = P.DPMM(0, d, 16, 5.0, prec=pr, burn_out=2, **_niw_prior(d))
    gg = P.DPMM(0, d, 16, 5.0, prec=pr, burn_out=2, stream=s.cuda_stream, **_niw_prior(d))
    ge.set_data(X)
    gg.set_data(X)
    for t in range(4):
        ge.sweep(5, 77)
        gg.sweep(5, 77)
        assert ge.K == gg.K
        assert all(np.array_equal(a, b) for a, b in zip(ge.labels(), gg.labels()))
    ne, sxe, _ = ge.stats()
    ng, sxg, _ = gg.stats()
    assert np.array_equal(ne, ng) and np.array_equal(sxe, sxg)


def test_high_dimension_d128():
    """The d = 128 configuration (CUDA-core kernels: one cluster's factor per shared-memory
    pass, statistics blocks beyond the staged layouts): FP64 sweeps bit-exact against the
    oracle; the FP32 path (the TF32 setting is refused above d = 32) keeps the statistics
    consistent with its labels."""
    import synth

    d = 128
    X, _ = synth.gaussian_mixture(1501, d, 3, 4.0, seed=128, dtype=np.float64)
    prior = _niw_prior(d)
    o, g = _pair(0, d, 8, 3.0, X, burn_out=1, **prior)
    for t in range(4):
        o.sweep(1, 5)
        g.sweep(1, 5)
        assert o.K == g.K, t
        zo, zbo = o.labels()
        zg, zbg = g.labels()
        assert np.array_equal(zo, zg) and np.array_equal(zbo, zbg), t
        _check_stats(o, g, rtol=1e-9)
    g.close()
    X32 = X.astype(np.float32)
    g = P.DPMM(0, d, 8, 3.0, prec=P.PREC_FP32, burn_out=1, **prior)
    g.set_data(X32)
    X64 = X32.astype(np.float64)
    for t in range(4):
        g.sweep(1, 9)
        z, zb = g.labels()
        n, sx, sxx = g.stats()
        assert n[0::3].sum() == len(X) and np.array_equal(n[0::3], n[1::3] + n[2::3])
        for k in range(g.K):
            for h in range(2):
                sel = (z == k) & (zb == h)
                assert n[3 * k + 1 + h] == sel.sum()
                c = max(1, sel.sum())
                assert np.allclose(sx[3 * k + 1 + h], X64[sel].sum(0), rtol=1e-5, atol=1e-3 * c ** 0.5)
                assert np.allclose(sxx[3 * k + 1 + h], X64[sel].T @ X64[sel], rtol=1e-5, atol=1e-2 * c ** 0.5)
    g.close()
