"""Batched independent problems through the C ABI: the problem id (fourth Philox
counter word) and dpmm_sweep_batch, which queues the sweeps of many chains on their
own streams so that they run concurrently.

FP64: every problem of a batch follows the oracle chain with the same problem id
bit-exactly (labels, counts, statistics to 1e-10, split/merge counters).  Reduced
precision: a batch gives the same chains as running each problem alone."""
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


def _prior(d):
    return dict(kappa0=1.0, m0=np.zeros(d), nu0=float(d + 3), psi0=np.eye(d))


def _problems():
    import synth

    out = []
    for j, (N, d, K) in enumerate([(1500, 2, 4), (2049, 5, 3), (777, 3, 5), (3001, 4, 4)]):
        X, _ = synth.gaussian_mixture(N, d, K, 7.0, seed=300 + j, dtype=np.float64)
        out.append((X, d))
    return out


def test_batch_fp64_problems_match_oracle():
    import torch

    seed, probs = 57, _problems()
    streams = [torch.cuda.Stream() for _ in probs]
    gs, os_ = [], []
    for j, ((X, d), s) in enumerate(zip(probs, streams)):
        g = P.DPMM(0, d, 12, 5.0, burn_out=2, stream=s.cuda_stream, **_prior(d))
        g.set_data(X)
        g.set_problem(j + 1)
        o = O.Oracle(O.NIW, d, 12, 5.0, burn_out=2, **_prior(d))
        o.set_data(X)
        gs.append(g)
        os_.append(o)
    total_splits = 0
    for t in range(12):
        P.dpmm_sweep_batch([g.h for g in gs], 1, seed)
        for j, (g, o) in enumerate(zip(gs, os_)):
            o.sweep(1, seed, problem=j + 1)
            assert o.K == g.K, (t, j)
            zo, zbo = o.labels()
            zg, zbg = g.labels()
            assert np.array_equal(zo, zg) and np.array_equal(zbo, zbg), (t, j)
            no, sxo, sxxo = o.stats()
            ng, sxg, sxxg = g.stats()
            assert np.array_equal(no, ng)
            assert np.abs(sxg - sxo).max() <= 1e-10 * (np.abs(sxo).max() + 1.0) * max(1.0, no.max())
            assert np.abs(sxxg - sxxo).max() <= 1e-10 * (np.abs(sxxo).max() + 1.0)
            co, cg = o.counters(), g.counters()
            assert co == cg, (t, j, co, cg)
            total_splits += co["splits"]
    assert total_splits >= 4
    for g in gs:
        g.close()


def test_problem_id_separates_streams():
    """Problem 0 in a batch is the chain of dpmm_sweep alone; problem 1 on the same
    data draws other labels."""
    import torch

    X, d = _problems()[0]
    s0, s1, s2 = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    a = P.DPMM(0, d, 12, 5.0, burn_out=2, stream=s0.cuda_stream, **_prior(d))
    b = P.DPMM(0, d, 12, 5.0, burn_out=2, stream=s1.cuda_stream, **_prior(d))
    c = P.DPMM(0, d, 12, 5.0, burn_out=2, stream=s2.cuda_stream, **_prior(d))
    for g in (a, b, c):
        g.set_data(X)
    b.set_problem(1)
    P.dpmm_sweep_batch([a.h, b.h], 3, 11)
    c.sweep(3, 11)
    za, zba = a.labels()
    zb, zbb = b.labels()
    zc, zbc = c.labels()
    assert np.array_equal(za, zc) and np.array_equal(zba, zbc)
    assert not np.array_equal(zba, zbb)
    for g in (a, b, c):
        g.close()


@pytest.mark.parametrize("prec,d", [("tf32", 32), ("bf16x3", 64), ("fp32", 8)])
def test_batch_equals_alone_reduced_precision(prec, d):
    """Concurrent chains on the tensor-core and CUDA-core reduced-precision paths give
    the same chains as running each alone (the kernels are deterministic and share no
    state across contexts)."""
    import torch

    import synth

    pr = {"tf32": P.PREC_TF32, "bf16x3": P.PREC_BF16X3, "fp32": P.PREC_FP32}[prec]
    data = [synth.gaussian_mixture(N, d, 4, 6.0, seed=N)[0] for N in (20_001, 9_000, 33_333)]
    streams = [torch.cuda.Stream() for _ in data]
    batch = []
    for j, (X, s) in enumerate(zip(data, streams)):
        g = P.DPMM(0, d, 16, 5.0, prec=pr, burn_out=2, stream=s.cuda_stream, **_prior(d))
        g.set_data(X)
        g.set_problem(j)
        batch.append(g)
    P.dpmm_sweep_batch([g.h for g in batch], 8, 5)
    for j, X in enumerate(data):
        alone = P.DPMM(0, d, 16, 5.0, prec=pr, burn_out=2, stream=torch.cuda.Stream().cuda_stream, **_prior(d))
        alone.set_data(X)
        alone.set_problem(j)
        alone.sweep(8, 5)
        assert alone.K == batch[j].K
        for u, v in zip(alone.labels(), batch[j].labels()):
            assert np.array_equal(u, v), j
        na, sxa, _ = alone.stats()
        nb, sxb, _ = batch[j].stats()
        assert np.array_equal(na, nb) and np.array_equal(sxa, sxb)
        alone.close()
    for g in batch:
        g.close()


def test_batch_rejects_bad_arguments():
    X, d = _problems()[0]
    g = P.DPMM(0, d, 8, 1.0, **_prior(d))
    g.set_data(X)
    with pytest.raises(Exception):
        P.dpmm_sweep_batch([g.h, None], 1, 0)
    g.close()
