"""Multinomial data of many categories (Sec. 5.3's document-word shapes) held as
compressed rows, through the C ABI, against the FP64 oracle.

Above 256 categories the library keeps each point's nonzero categories and counts only.
The multinomial score sums count x log theta over them, which equals the oracle's sum
over all d categories (zero terms change no sum); the FP64 path adds in increasing
category order without fused multiply-adds, as the oracle's loop does, so its labels,
counts and split/merge decisions match the oracle's exactly.  The FP32 path's labels
agree with FP64 within the budgets of the other FP32 paths (labels 1e-3, sub-labels
1e-2).  Statistics are integer counts, added atomically (exact in any order)."""
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


def _data(N, d, K, seed, lo=20, hi=200):
    import synth

    ip, ix, ct, y = synth.newsgroups_like(N=N, d=d, K=K, seed=seed, len_lo=lo, len_hi=hi)
    return ip, ix, ct, y, synth.csr_to_dense(ip, ix, ct, d)


def _check_counts(o, g):
    no, sxo, _ = o.stats()
    ng, sxg, _ = g.stats()
    assert np.array_equal(no, ng)
    assert np.array_equal(sxo, sxg)  # integer counts: exact


def test_full_sweeps_fp64_match_oracle():
    """Whole sweeps from K = 1 at d = 1,500 (compressed rows): labels, sub-labels, K,
    counts and split/merge counters identical to the oracle's after every sweep."""
    N, d = 2_001, 1_500
    ip, ix, ct, y, X = _data(N, d, 5, seed=31)
    beta = np.ones(d)
    o = O.Oracle(O.DIRICHLET, d, 12, 5.0, burn_out=2, beta=beta)
    g = P.DPMM(1, d, 12, 5.0, prec=P.PREC_FP64_PLAIN, burn_out=2, beta=beta)
    o.set_data(X.astype(np.float64))
    g.set_data(X)
    splits = 0
    for t in range(20):
        o.sweep(1, 41)
        g.sweep(1, 41)
        assert o.K == g.K, t
        zo, zbo = o.labels()
        zg, zbg = g.labels()
        assert np.array_equal(zo, zg) and np.array_equal(zbo, zbg), t
        _check_counts(o, g)
        co, cg = o.counters(), g.counters()
        assert co == cg, (t, co, cg)
        splits += co["splits"]
    assert splits >= 2 and g.K >= 3
    g.close()


def _with_oracle_params(N, d, K, seed, prec):
    ip, ix, ct, y, X = _data(N, d, K, seed=seed)
    # consecutive ids over the topics that have documents (an empty cluster would be
    # removed by the label step and the ids after it renumbered)
    y = np.unique(y, return_inverse=True)[1].astype(np.int32)
    assert y.max() + 1 == K, "every topic needs documents at this size"
    beta = np.ones(d)
    zb = (np.arange(N) % 2).astype(np.uint8)
    o = O.Oracle(O.DIRICHLET, d, 64, 3.0, beta=beta)
    o.set_data(X.astype(np.float64))
    o.set_state(K, y, zb)
    o.draw_params(seed)
    g = P.DPMM(1, d, 64, 3.0, prec=prec, beta=beta)
    g.set_data_csr(ip, ix, ct)
    g.set_state(K, y, zb)
    g.set_params(K, o.params())
    return X, o, g


def test_label_step_fp64_newsgroups_dimension():
    """One label step at the 20newsgroups dimension (d = 20,000, K = 20) with the
    oracle's parameters: the labels of a sample of 1,500 points bit-exact (the oracle's
    random streams are keyed by the point, so a sample sees the whole step's draws)."""
    N, d, K = 3_000, 20_000, 20
    X, o, g = _with_oracle_params(N, d, K, 7, P.PREC_FP64_PLAIN)
    it = g.info()[1]
    g.set_mask(2)
    g.sweep(1, 13)
    assert g.K == K
    zg, zbg = g.labels()
    idx = np.sort(np.random.default_rng(1).choice(N, 1_500, replace=False))
    zo, zbo = o.label_probe_points(13, it, idx)
    assert np.array_equal(zo, zg[idx])
    assert np.array_equal(zbo, zbg[idx])
    g.close()


def test_fp32_labels_and_scores_within_budget():
    """FP32 path at d = 20,000: every cluster score against FP64 (sparse dot products in
    numpy), and one label step against the oracle's on a sample."""
    N, d, K = 3_000, 20_000, 20
    X, o, g = _with_oracle_params(N, d, K, 12, P.PREC_FP32)
    p = o.params()
    s32 = g.label_scores()
    X64 = X.astype(np.float64)
    s64 = np.stack([p["logw"][3 * k] + X64 @ p["logtheta"][3 * k] for k in range(K)], 1)
    cont = s64 >= s64.max(1, keepdims=True) - 20.0
    err = np.abs(s32 - s64)
    assert err[cont].mean() < 0.02, err[cont].mean()
    assert err[cont].max() < 0.2, err[cont].max()
    it = g.info()[1]
    g.set_mask(2)
    g.sweep(1, 17)
    assert g.K == K
    zg, zbg = g.labels()
    idx = np.sort(np.random.default_rng(2).choice(N, 2_000, replace=False))
    zo, zbo = o.label_probe_points(17, it, idx)
    assert (zo != zg[idx]).mean() < 1e-3
    same = zo == zg[idx]
    assert (zbo[same] != zbg[idx][same]).mean() < 1e-2
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_csr_input_equals_dense_input(prec):
    """dpmm_set_data (dense counts, compressed on the device) and dpmm_set_data_csr give
    the same chain."""
    N, d = 1_500, 700
    ip, ix, ct, y, X = _data(N, d, 4, seed=9)
    pr = P.PREC_FP64_PLAIN if prec == "fp64" else P.PREC_FP32
    a = P.DPMM(1, d, 16, 5.0, prec=pr, burn_out=2, beta=np.ones(d))
    b = P.DPMM(1, d, 16, 5.0, prec=pr, burn_out=2, beta=np.ones(d))
    a.set_data(X)
    b.set_data_csr(ip, ix, ct)
    a.sweep(12, 3)
    b.sweep(12, 3)
    za, zba = a.labels()
    zb, zbb = b.labels()
    assert np.array_equal(za, zb) and np.array_equal(zba, zbb)
    assert np.array_equal(a.stats()[1], b.stats()[1])
    a.close()
    b.close()


def test_statistics_and_checkpoint():
    """FP32 chain on a 20newsgroups-shaped data set: the count table matches a recount
    of the labels after every sweep, the chain finds the topics, and a checkpoint taken
    mid-chain continues exactly (the compact counts are rebuilt from the labels)."""
    import synth

    N, d, K = 11_314, 20_000, 20
    ip, ix, ct, y = synth.newsgroups_like(N=N, d=d, K=K, seed=1006)
    g = P.DPMM(1, d, 64, 10.0, prec=P.PREC_FP32, burn_out=5, beta=np.ones(d))
    g.set_data_csr(ip, ix, ct)
    rows = np.repeat(np.arange(N), np.diff(ip))
    ck = None
    for t in range(60):
        g.sweep(1, 5)
        if t == 39:
            ck = g.checkpoint()
        if t % 10 == 9:
            z, zb = g.labels()
            n, sx, _ = g.stats()
            Kn = g.K
            slot = 2 * z[rows] + zb[rows]
            ref = np.zeros((2 * Kn, d))
            np.add.at(ref, (slot, ix), ct)
            for k in range(Kn):
                for h in range(2):
                    assert n[3 * k + 1 + h] == ((z == k) & (zb == h)).sum()
                    assert np.array_equal(sx[3 * k + 1 + h], ref[2 * k + h])
    from collections import Counter

    z, _ = g.labels()
    purity = sum(Counter(z[y == k]).most_common(1)[0][1] for k in range(K) if (y == k).any()) / N
    assert purity > 0.9, (purity, g.K)
    z60, zb60 = g.labels()
    g2 = P.DPMM(1, d, 64, 10.0, prec=P.PREC_FP32, burn_out=5, beta=np.ones(d))
    g2.set_data_csr(ip, ix, ct)
    g2.restore(ck)
    g2.sweep(20, 5)
    z2, zb2 = g2.labels()
    assert np.array_equal(z2, z60) and np.array_equal(zb2, zb60)
    g.close()
    g2.close()


def test_rejects_malformed_rows():
    d = 300
    g = P.DPMM(1, d, 8, 1.0, prec=P.PREC_FP32, beta=np.ones(d))
    bad = [
        (np.array([0, 2]), np.array([5, 5]), np.array([1, 1])),    # repeated category
        (np.array([0, 2]), np.array([7, 3]), np.array([1, 1])),    # not increasing
        (np.array([0, 1]), np.array([d]), np.array([1])),          # out of range
        (np.array([0, 1]), np.array([3]), np.array([-1])),         # negative count
    ]
    for ip, ix, ct in bad:
        with pytest.raises(P.DPMMError) as e:
            g.set_data_csr(ip, ix, ct)
        assert e.value.status == P.DPMM_EINVAL
    g.close()
    # compressed rows are for multinomial data of more than 256 categories only
    h = P.DPMM(1, 200, 8, 1.0, prec=P.PREC_FP32, beta=np.ones(200))
    with pytest.raises(P.DPMMError):
        h.set_data_csr(np.array([0, 1]), np.array([3]), np.array([1]))
    h.close()
