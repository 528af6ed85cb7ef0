"""Checkpoint and resume through the C ABI: a chain stopped at a sweep boundary and
restored into a fresh context (same prior, data and options) continues bit for bit as
the uninterrupted chain, in FP64, TF32, BF16X3 (d = 96) and BF16 (multinomial); bad
checkpoints are refused."""
import numpy as np
import pytest

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


def _case(name):
    import synth

    if name == "fp64":
        X, _ = synth.gaussian_mixture(4001, 3, 4, 6.0, seed=21, dtype=np.float64)
        return X, 0, P.PREC_FP64_PLAIN, dict(kappa0=1.0, m0=np.zeros(3), nu0=6.0, psi0=np.eye(3))
    if name == "tf32":
        X, _ = synth.gaussian_mixture(20_001, 32, 5, 6.0, seed=22)
        return X, 0, P.PREC_TF32, dict(kappa0=1.0, m0=np.zeros(32), nu0=35.0, psi0=np.eye(32))
    if name == "bf16x3":
        X, _ = synth.gaussian_mixture(20_001, 96, 4, 6.0, seed=24)
        return X, 0, P.PREC_BF16X3, dict(kappa0=1.0, m0=np.zeros(96), nu0=99.0, psi0=np.eye(96))
    X, _ = synth.multinomial_mixture(20_001, 64, 5, 60, seed=23)
    return X, 1, P.PREC_BF16, dict(beta=np.ones(64))


def _snap(g):
    z, zb = g.labels()
    n, sx, sxx = g.stats()
    return g.K, z, zb, n, sx, sxx, g.counters()


def _same(a, b):
    assert a[0] == b[0]
    for u, v in zip(a[1:6], b[1:6]):
        if u is None:
            assert v is None
        else:
            assert np.array_equal(u, v)
    assert a[6] == b[6]


@pytest.mark.parametrize("name", ["fp64", "tf32", "bf16x3", "bf16"])
def test_resume_continues_the_chain_exactly(name):
    X, kind, pr, prior = _case(name)
    seed = 77
    a = P.DPMM(kind, X.shape[1], 24, 5.0, prec=pr, burn_out=2, **prior)
    a.set_data(X)
    a.sweep(6, seed)
    ck = a.checkpoint()
    a.sweep(6, seed)
    ref = _snap(a)
    b = P.DPMM(kind, X.shape[1], 24, 5.0, prec=pr, burn_out=2, **prior)
    b.set_data(X)
    b.restore(ck)
    b.sweep(6, seed)
    _same(ref, _snap(b))
    # rewinding the first chain to the checkpoint replays the same sweeps
    a.restore(ck)
    a.sweep(6, seed)
    _same(ref, _snap(a))
    a.close()
    b.close()


def test_bad_checkpoints_refused():
    X, kind, pr, prior = _case("fp64")
    a = P.DPMM(kind, 3, 24, 5.0, prec=pr, **prior)
    a.set_data(X)
    a.sweep(2, 1)
    ck = a.checkpoint()
    b = P.DPMM(kind, 3, 24, 5.0, prec=pr, **prior)
    b.set_data(X[:-1])  # another N
    with pytest.raises(P.DPMMError) as e:
        b.restore(ck)
    assert e.value.status == P.DPMM_EINVAL
    bad = bytearray(ck)
    bad[0] ^= 0xFF  # magic
    with pytest.raises(P.DPMMError):
        a.restore(bytes(bad))
    with pytest.raises(P.DPMMError):
        a.restore(ck[: len(ck) // 2])  # truncated
    a.restore(ck)  # a good one still loads
    a.close()
    b.close()
