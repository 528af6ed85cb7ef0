"""Point-sharded chains (the data of one chain split over several contexts, as over the
GPUs of a multi-GPU run) on one GPU, against the FP64 oracle on the whole data set.

Each shard labels its own points with the random streams of their index in the whole set;
the shards' statistics are summed in shard order after the label step and after any
relabelling, so every shard draws the same parameters and takes the same split/merge
decisions.  The concatenated labels of the shards must equal the oracle's exactly, the
counts exactly and the FP64 sums to 1e-10 relative (the sums of a sharded chain differ
from an unsharded one's by rounding only), sweep after sweep from K = 1."""
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


def _shards(kind, d, K_max, alpha, parts, prec, **prior):
    gs, off = [], 0
    for Xs in parts:
        g = P.DPMM(kind, d, K_max, alpha, prec=prec, burn_out=2, **prior)
        if isinstance(Xs, tuple):
            g.set_data_csr(*Xs)
            n = len(Xs[0]) - 1
        else:
            g.set_data(Xs)
            n = Xs.shape[0]
        g.set_shard(off)
        off += n
        gs.append(g)
    return gs


def _close(o, g):
    no, sxo, sxxo = o.stats()
    ng, sxg, sxxg = g.stats()
    assert np.array_equal(no, ng)
    scale = np.abs(sxo).max() + 1.0
    assert np.abs(sxg - sxo).max() <= 1e-10 * scale * max(1.0, no.max())
    if sxxo is not None:
        assert np.abs(sxxg - sxxo).max() <= 1e-10 * (np.abs(sxxo).max() + 1.0)


def test_gaussian_fp64_three_shards_match_oracle():
    import synth

    d = 3
    X, _ = synth.gaussian_mixture(5003, d, 4, 6.0, seed=61, dtype=np.float64)
    prior = dict(kappa0=1.0, m0=np.zeros(d), nu0=float(d + 3), psi0=np.eye(d))
    cuts = [0, 1200, 3307, 5003]  # uneven shards
    gs = _shards(0, d, 12, 5.0, [X[a:b] for a, b in zip(cuts, cuts[1:])], P.PREC_FP64_PLAIN, **prior)
    o = O.Oracle(O.NIW, d, 12, 5.0, burn_out=2, **prior)
    o.set_data(X)
    splits = 0
    for t in range(20):
        o.sweep(1, 71)
        P.dpmm_sweep_sharded([g.h for g in gs], 1, 71)
        assert all(g.K == o.K for g in gs), t
        zo, zbo = o.labels()
        zg = np.concatenate([g.labels()[0] for g in gs])
        zbg = np.concatenate([g.labels()[1] for g in gs])
        assert np.array_equal(zo, zg) and np.array_equal(zbo, zbg), t
        for g in gs:  # every shard holds the whole chain's statistics
            _close(o, g)
        assert all(g.counters() == o.counters() for g in gs), t
        splits += o.counters()["splits"]
    assert splits >= 2 and o.K >= 3
    for g in gs:
        g.close()


def test_multinomial_compressed_rows_two_shards_match_oracle():
    import synth

    N, d = 2_400, 900
    ip, ix, ct, y = synth.newsgroups_like(N=N, d=d, K=4, seed=62, len_lo=20, len_hi=120)
    X = synth.csr_to_dense(ip, ix, ct, d)
    cut = 1_000
    parts = [(ip[: cut + 1], ix[: ip[cut]], ct[: ip[cut]]),
             (ip[cut:] - ip[cut], ix[ip[cut]:], ct[ip[cut]:])]
    beta = np.ones(d)
    gs = _shards(1, d, 12, 5.0, parts, P.PREC_FP64_PLAIN, beta=beta)
    o = O.Oracle(O.DIRICHLET, d, 12, 5.0, burn_out=2, beta=beta)
    o.set_data(X.astype(np.float64))
    for t in range(15):
        o.sweep(1, 73)
        P.dpmm_sweep_sharded([g.h for g in gs], 1, 73)
        assert all(g.K == o.K for g in gs), t
        zg = np.concatenate([g.labels()[0] for g in gs])
        zbg = np.concatenate([g.labels()[1] for g in gs])
        zo, zbo = o.labels()
        assert np.array_equal(zo, zg) and np.array_equal(zbo, zbg), t
        no, sxo, _ = o.stats()
        for g in gs:
            ng, sxg, _ = g.stats()
            assert np.array_equal(no, ng) and np.array_equal(sxo, sxg)
    assert o.K >= 3
    for g in gs:
        g.close()


def test_sharded_chain_refuses_mismatched_shards():
    import synth

    d = 3
    X, _ = synth.gaussian_mixture(600, d, 2, 6.0, seed=63, dtype=np.float64)
    prior = dict(kappa0=1.0, m0=np.zeros(d), nu0=float(d + 3), psi0=np.eye(d))
    a, b = _shards(0, d, 8, 5.0, [X[:300], X[300:]], P.PREC_FP64_PLAIN, **prior)
    b.set_shard(301)  # a gap between the shards
    with pytest.raises(P.DPMMError) as e:
        P.dpmm_sweep_sharded([a.h, b.h], 1, 1)
    assert e.value.status == P.DPMM_EINVAL
    # reduced-precision Gaussian shards centre their data separately: refused
    c, f = _shards(0, d, 8, 5.0, [X[:300].astype(np.float32), X[300:].astype(np.float32)], P.PREC_FP32, **prior)
    with pytest.raises(P.DPMMError) as e:
        P.dpmm_sweep_sharded([c.h, f.h], 1, 1)
    assert e.value.status == P.DPMM_EINVAL
    for g in (a, b, c, f):
        g.close()


def test_compressed_rows_fp32_three_shards_equal_unsharded_chain():
    """The FP32 compressed-row path (20newsgroups shape, smaller N): statistics are integer
    counts, which add exactly in any order, so three shards give the very chain of one
    context: labels, sub-labels, K and counts identical sweep after sweep."""
    import synth

    N, d = 3_001, 2_000
    ip, ix, ct, y = synth.newsgroups_like(N=N, d=d, K=6, seed=64, len_lo=20, len_hi=150)
    cuts = [0, 700, 1_901, N]
    parts = [(ip[a: b + 1] - ip[a], ix[ip[a]: ip[b]], ct[ip[a]: ip[b]]) for a, b in zip(cuts, cuts[1:])]
    beta = np.ones(d)
    gs = _shards(1, d, 16, 5.0, parts, P.PREC_FP32, beta=beta)
    one = P.DPMM(1, d, 16, 5.0, prec=P.PREC_FP32, burn_out=2, beta=beta)
    one.set_data_csr(ip, ix, ct)
    for t in range(15):
        one.sweep(1, 75)
        P.dpmm_sweep_sharded([g.h for g in gs], 1, 75)
        assert all(g.K == one.K for g in gs), t
        z1, zb1 = one.labels()
        assert np.array_equal(z1, np.concatenate([g.labels()[0] for g in gs])), t
        assert np.array_equal(zb1, np.concatenate([g.labels()[1] for g in gs])), t
        n1, sx1, _ = one.stats()
        for g in gs:
            ng, sxg, _ = g.stats()
            assert np.array_equal(n1, ng) and np.array_equal(sx1, sxg), t
    assert one.K >= 3
    for g in gs + [one]:
        g.close()


def test_dense_multinomial_bf16_two_shards_equal_unsharded_chain():
    """Dense multinomial counts on the BF16 tensor-core path: the statistics are integer
    counts (exact in any order) and every later step reads the exchanged statistics table,
    so two shards give the very chain of one context."""
    import synth

    N, d = 30_001, 120
    X, y = synth.multinomial_mixture(N, d, 6, 60, seed=66)
    cut = 12_345
    beta = np.ones(d)
    gs = _shards(1, d, 16, 5.0, [X[:cut], X[cut:]], P.PREC_BF16, beta=beta)
    one = P.DPMM(1, d, 16, 5.0, prec=P.PREC_BF16, burn_out=2, beta=beta)
    one.set_data(X)
    for t in range(12):
        one.sweep(1, 77)
        P.dpmm_sweep_sharded([g.h for g in gs], 1, 77)
        assert all(g.K == one.K for g in gs), t
        z1, zb1 = one.labels()
        assert np.array_equal(z1, np.concatenate([g.labels()[0] for g in gs])), t
        assert np.array_equal(zb1, np.concatenate([g.labels()[1] for g in gs])), t
        n1, sx1, _ = one.stats()
        for g in gs:
            ng, sxg, _ = g.stats()
            assert np.array_equal(n1, ng) and np.array_equal(sx1, sxg), t
    assert one.K >= 3
    for g in gs + [one]:
        g.close()
