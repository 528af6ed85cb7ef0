"""Split-BF16 tensor-core label step (precision BF16X3: Gaussian, d <= 128) against
FP64 on the same parameters and keys, through the C ABI.

Each operand keeps about 16 significant bits (x = x_h + x_l, W = W_h + W_l, both BF16;
the dropped x_l W_l term is 2^-18 relative) and the accumulation is FP32, so the
score error grows with the cancellation between x W and b.  A CPU emulation of this
arithmetic on the d = 128 workload (64 clusters, covariances ~ Wishart(I, d + 2))
gave 0.0013 nat mean, 0.014 at the 99th percentile and 0.11 at worst on the clusters
that can win a draw; a single TF32 product gave 0.085 / 0.97 / 4.1.  Budgets: on the
clusters within 20 nats of a point's best score, mean error <= 0.01 nat, 99th
percentile <= 0.05, worst <= 0.5; labels disagree with the FP64 path on fewer than
1e-3 of the points."""
import numpy as np
import pytest
from scipy import stats

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


def _prior(d):
    return dict(kappa0=1.0, m0=np.zeros(d), nu0=float(d + 3), psi0=np.eye(d))


def _setup(N, d, K, seed, K_max=64):
    import synth

    X, y = synth.gaussian_mixture(N, d, K, 5.0, seed=seed)
    o = O.Oracle(O.NIW, d, K_max, 3.0, **_prior(d))
    o.set_data(X.astype(np.float64))
    zb = (np.arange(N) % 2).astype(np.uint8)
    o.set_state(K, y, zb)
    o.draw_params(seed)
    p = o.params()
    g = P.DPMM(0, d, K_max, 3.0, prec=P.PREC_BF16X3, **_prior(d))
    g.set_data(X)
    g.set_state(K, y, zb)
    g.set_params(K, p)
    return X, y, zb, o, g, p


def _fp64_scores(X, p, K):
    out = np.empty((X.shape[0], K))
    for k in range(K):
        W = p["W"][3 * k]
        S = np.linalg.inv(W @ W.T)
        out[:, k] = p["logw"][3 * k] + stats.multivariate_normal(p["mu"][3 * k], S, allow_singular=True).logpdf(
            X.astype(np.float64))
    return out


@pytest.mark.parametrize("N,d,K", [(3001, 128, 7), (1000, 64, 5), (2049, 100, 9), (777, 20, 3), (1, 128, 1),
                                   (4001, 128, 40)])
def test_x3_scores_within_budget(N, d, K):
    """Every cluster score of every point (including the padded rows of the last tile
    pair, the padded features d < 64 or 128, K = 1 and N = 1, and K = 40 clusters
    streamed through the factor stages and TMEM buffers many times) against FP64."""
    if N < K:
        pytest.skip("needs a point per cluster")
    X, y, zb, o, g, p = _setup(max(N, 1), d, K, seed=N + d) if N > 1 else _setup_single(d)
    s_x3 = g.label_scores()
    s_64 = _fp64_scores(X, p, g.K)
    err = np.abs(s_x3 - s_64)
    cont = s_64 >= s_64.max(1, keepdims=True) - 20.0
    assert err[cont].mean() < 0.01, err[cont].mean()
    assert np.quantile(err[cont], 0.99) < 0.05, np.quantile(err[cont], 0.99)
    assert err[cont].max() < 0.5, err[cont].max()
    g.close()


def _setup_single(d):
    """One point, one cluster whose parameters come from the points of a larger draw."""
    import synth

    X, _ = synth.gaussian_mixture(4 * d, d, 1, 5.0, seed=d)
    o = O.Oracle(O.NIW, d, 4, 3.0, **_prior(d))
    o.set_data(X.astype(np.float64))
    o.set_state(1, np.zeros(len(X), np.int32), (np.arange(len(X)) % 2).astype(np.uint8))
    o.draw_params(3)
    p = o.params()
    x1 = X[:1]
    g = P.DPMM(0, d, 4, 3.0, prec=P.PREC_BF16X3, **_prior(d))
    g.set_data(x1)
    g.set_state(1, np.zeros(1, np.int32), np.zeros(1, np.uint8))
    g.set_params(1, p)
    return x1, None, None, o, g, p


@pytest.mark.parametrize("d", [64, 99, 128])
def test_x3_labels_agree_with_fp64(d):
    """One label and sub-label step from the same parameters and Philox keys as the
    FP64 oracle: labels within the disagreement budget (d = 99 pads the features of
    both the tensor-core kernel and the FP32 sub-label kernel)."""
    N, K = 20_000, 12
    X, y, zb, o, g, p = _setup(N, d, K, seed=5 + d)
    g.set_mask(2)
    g.sweep(1, 321)
    o.sweep(1, 321, mask=O.MASK_LABELS)
    zo, zbo = o.labels()
    zg, zbg = g.labels()
    assert o.K == g.K
    assert (zo != zg).mean() < 1e-3, (zo != zg).mean()
    assert (zbo != zbg).mean() < 1e-2, (zbo != zbg).mean()
    g.close()


@pytest.mark.parametrize("d,N,K", [(64, 40_001, 6), (128, 30_001, 4)])
def test_x3_chain_finds_clusters_and_keeps_statistics(d, N, K):
    """Full sweeps from K = 1: the chain recovers the mixture, and after every sweep
    the statistics agree with an FP64 recount of the GPU's own labels (FP32 path)."""
    from collections import Counter

    import synth

    X, y = synth.gaussian_mixture(N, d, K, 8.0, seed=d + N)
    g = P.DPMM(0, d, 32, 10.0, prec=P.PREC_BF16X3, burn_out=3, **_prior(d))
    g.set_data(X)
    X64 = X.astype(np.float64)
    for t in range(40):
        g.sweep(1, 17)
        if t % 10 == 9:
            z, zb = g.labels()
            n, sx, sxx = g.stats()
            assert n[0::3].sum() == N and np.array_equal(n[0::3], n[1::3] + n[2::3])
            for k in range(g.K):
                for h in range(2):
                    sel = (z == k) & (zb == h)
                    s = 3 * k + 1 + h
                    assert n[s] == sel.sum()
                    c = max(1, sel.sum())
                    assert np.allclose(sx[s], X64[sel].sum(0), rtol=1e-5, atol=1e-2 * c ** 0.5)
                    assert np.allclose(sxx[s], X64[sel].T @ X64[sel], rtol=1e-5, atol=1e-1 * c ** 0.5)
    z, _ = g.labels()
    purity = sum(Counter(z[y == k]).most_common(1)[0][1] for k in range(K) if (y == k).any()) / N
    assert purity > 0.95, (purity, g.K)
    g.close()


def test_x3_refuses_unsupported():
    """BF16X3 is the Gaussian path up to d = 128."""
    with pytest.raises(Exception):
        P.DPMM(0, 129, 8, 1.0, prec=P.PREC_BF16X3, **_prior(129))
    with pytest.raises(Exception):
        P.DPMM(1, 16, 8, 1.0, prec=P.PREC_BF16X3, beta=np.ones(16))
