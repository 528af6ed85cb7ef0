"""dpmm_update_data through the C ABI from the three kinds of source memory: device
memory, page-locked host memory (read in place by the conversion kernels) and pageable
host memory (staged).  The stored data, and so the statistics recounted from a fixed
state, are the same bit for bit whichever the source; they match a fresh chain on the
new data to rounding (the centre stays the one of the first data)."""
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


def _prior(d):
    return dict(kappa0=1.0, m0=np.zeros(d), nu0=float(d + 3), psi0=np.eye(d))


@pytest.mark.parametrize("prec,d", [("fp32", 8), ("tf32", 32), ("fp64", 5)])
def test_update_data_sources_agree(prec, d):
    import torch

    import synth

    pr = {"fp32": P.PREC_FP32, "tf32": P.PREC_TF32, "fp64": P.PREC_FP64_PLAIN}[prec]
    dt = np.float64 if prec == "fp64" else np.float32
    N, K = 30_001, 4
    X1, y = synth.gaussian_mixture(N, d, K, 6.0, seed=1, dtype=dt)
    X2, _ = synth.gaussian_mixture(N, d, K, 6.0, seed=2, dtype=dt)
    zb = (np.arange(N) % 2).astype(np.uint8)
    srcs = {"pageable": X2, "pinned": torch.from_numpy(X2).pin_memory(), "device": torch.from_numpy(X2).cuda()}
    out = {}
    for name, src in srcs.items():
        g = P.DPMM(0, d, 8, 3.0, prec=pr, **_prior(d))
        g.set_data(X1)
        g.set_state(K, y, zb)
        g.update_data(src)
        g.set_state(K, y, zb)  # statistics recounted from the new data
        out[name] = g.stats()
        g.close()
    for name in ("pinned", "device"):
        for a, b in zip(out["pageable"], out[name]):
            assert np.array_equal(a, b), name
    fresh = P.DPMM(0, d, 8, 3.0, prec=pr, **_prior(d))
    fresh.set_data(X2)
    fresh.set_state(K, y, zb)
    n, sx, sxx = fresh.stats()
    fresh.close()
    n0, sx0, sxx0 = out["pageable"]
    assert np.array_equal(n, n0)
    # the stored values are x - centre rounded to the working precision, and the two chains
    # centre differently: FP64 exact to rounding, FP32 to 2^-24, TF32 to 2^-11 of |x - centre|
    rtol = {"fp64": 1e-10, "fp32": 1e-5, "tf32": 2e-3}[prec]
    scale1 = np.abs(sx).max() + 1.0
    scale2 = np.abs(sxx).max() + 1.0
    assert np.abs(sx0 - sx).max() <= rtol * scale1
    assert np.abs(sxx0 - sxx).max() <= rtol * scale2


@pytest.mark.parametrize("prec,d", [("tf32", 32), ("fp64", 5), ("bf16x3", 64)])
def test_staged_data_give_the_chain_of_updated_data(prec, d):
    """dpmm_stage_data (the copy overlaps the sweep in flight; the next sweep takes the
    values) gives, sweep for sweep, the chain of dpmm_update_data called right before that
    sweep: same labels, sub-labels, K and statistics, from page-locked and pageable
    sources, with a second staging call replacing the first."""
    import torch

    import synth

    pr = {"tf32": P.PREC_TF32, "fp64": P.PREC_FP64_PLAIN, "bf16x3": P.PREC_BF16X3}[prec]
    dt = np.float64 if prec == "fp64" else np.float32
    N, K = 40_001, 4
    Xs = [synth.gaussian_mixture(N, d, K, 6.0, seed=10 + t, dtype=dt)[0] for t in range(4)]
    y = synth.gaussian_mixture(N, d, K, 6.0, seed=10, dtype=dt)[1]
    zb = (np.arange(N) % 2).astype(np.uint8)
    pinned = [torch.from_numpy(x).pin_memory() for x in Xs]

    def chain(staged):
        g = P.DPMM(0, d, 16, 3.0, prec=pr, burn_out=2, **_prior(d))
        g.set_data(Xs[0])
        g.set_state(K, y, zb)
        g.sweep(2, 9)
        out = []
        for t in (1, 2, 3):
            src = pinned[t] if t != 2 else Xs[t]  # page-locked and pageable sources
            if staged:
                if t == 3:
                    g.stage_data(pinned[1])  # replaced by the next call
                g.stage_data(src)
            else:
                g.update_data(src)
            g.sweep(2, 9)
            out.append((g.K, *g.labels(), *[s.copy() for s in g.stats()[:2]]))
        g.close()
        return out

    for a, b in zip(chain(False), chain(True)):
        assert a[0] == b[0]
        for u, v in zip(a[1:], b[1:]):
            assert np.array_equal(u, v)
