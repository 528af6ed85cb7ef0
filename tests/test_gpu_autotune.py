"""Run-time choice of the label-step kernel (Sec. 4.2, "Two kernels for optimization": the
paper picks between a hand-written kernel and a library product at run time, from d, N
and the GPU), through the C ABI.

With DPMM_KERNEL_AUTO the next eager sweep times the tensor-core and the CUDA-core label
kernels on the context's data and keeps the faster; the choice is cached for contexts of
the same shape.  The label step is a deterministic function of the parameters and the
sweep counter, so an automatic chain must equal, bit for bit, a chain pinned to the kernel
it chose.  A context pinned to the CUDA cores draws its labels in FP32 and must agree with
the FP64 label step within the budget of the reduced-precision paths."""
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


def _gauss(N, d, K, seed, prec, choice=None):
    import synth

    X, y = synth.gaussian_mixture(N, d, K, 5.0, seed=seed)
    g = P.DPMM(0, d, 32, 10.0, prec=prec, burn_out=3, **_prior(d))
    if choice is not None:
        g.set_kernel(choice)
    g.set_data(X)
    g.set_state(K, y.astype(np.int32), (np.arange(N) % 2).astype(np.uint8))
    return X, y, g


def test_auto_chain_equals_the_chain_of_the_chosen_kernel():
    N, d, K = 150_001, 32, 6
    _, _, a = _gauss(N, d, K, 11, P.PREC_TF32, P.KERNEL_AUTO)
    a.sweep(4, 5)
    use, mt, mc = a.kernel()
    assert mt > 0 and mc > 0
    assert use == (P.KERNEL_CUDA_CORE if mc < mt else P.KERNEL_TENSOR)
    _, _, b = _gauss(N, d, K, 11, P.PREC_TF32, use)
    b.sweep(4, 5)
    assert b.kernel()[0] == use and b.kernel()[1] == -1.0  # pinned: never timed
    za, zba = a.labels()
    zb, zbb = b.labels()
    assert a.K == b.K
    assert np.array_equal(za, zb) and np.array_equal(zba, zbb)
    assert np.array_equal(a.stats()[1], b.stats()[1])
    # a third context of the same shape takes the cached choice and figures
    _, _, c = _gauss(N, d, K, 12, P.PREC_TF32, P.KERNEL_AUTO)
    c.sweep(1, 5)
    assert c.kernel() == (use, mt, mc)
    for g in (a, b, c):
        g.close()


def test_cuda_core_labels_on_a_tf32_context_agree_with_fp64():
    """Pinned to the CUDA cores, a TF32 context's label step runs the FP32 kernel on the
    same parameters: labels within 1e-3 and sub-labels within 1e-2 of the FP64 step."""
    import synth

    N, d, K = 20_000, 32, 8
    X, y = synth.gaussian_mixture(N, d, K, 5.0, seed=21)
    zb = (np.arange(N) % 2).astype(np.uint8)
    o = O.Oracle(O.NIW, d, 64, 10.0, **_prior(d))
    o.set_data(X.astype(np.float64))
    o.set_state(K, y.astype(np.int32), zb)
    o.draw_params(21)
    g = P.DPMM(0, d, 64, 10.0, prec=P.PREC_TF32, **_prior(d))
    g.set_kernel(P.KERNEL_CUDA_CORE)
    g.set_data(X)
    g.set_state(K, y.astype(np.int32), zb)
    g.set_params(K, o.params())  # the label step alone (mask 2) on the oracle's parameters
    g.set_mask(2)
    g.sweep(1, 123)
    o.sweep(1, 123, mask=O.MASK_LABELS)
    assert g.kernel()[0] == P.KERNEL_CUDA_CORE
    zo, zbo = o.labels()
    zg, zbg = g.labels()
    assert o.K == g.K
    assert (zo != zg).mean() < 1e-3
    assert (zbo != zbg).mean() < 1e-2
    g.close()


@pytest.mark.parametrize("case", ["multinomial_bf16", "gauss_bf16x3"])
def test_auto_on_the_other_tensor_core_precisions(case):
    import synth

    if case == "multinomial_bf16":
        N, d, K = 40_000, 100, 5
        X, y = synth.multinomial_mixture(N, d, K, 60, seed=31)
        g = P.DPMM(1, d, 32, 10.0, prec=P.PREC_BF16, burn_out=3, beta=np.ones(d))
    else:
        N, d, K = 40_000, 64, 5
        X, y = synth.gaussian_mixture(N, d, K, 5.0, seed=32)
        g = P.DPMM(0, d, 32, 10.0, prec=P.PREC_BF16X3, burn_out=3, **_prior(d))
    g.set_kernel(P.KERNEL_AUTO)
    g.set_data(X)
    g.set_state(K, y.astype(np.int32), (np.arange(N) % 2).astype(np.uint8))
    g.sweep(3, 7)
    use, mt, mc = g.kernel()
    assert mt > 0 and mc > 0 and use in (P.KERNEL_TENSOR, P.KERNEL_CUDA_CORE)
    n = g.stats()[0]
    assert n[0::3].sum() == N and g.K >= 2
    g.close()


def test_fp64_plain_and_bad_choices():
    _, _, g = _gauss(5_000, 4, 3, 41, P.PREC_FP64_PLAIN, P.KERNEL_AUTO)
    g.sweep(1, 1)
    assert g.kernel() == (P.KERNEL_CUDA_CORE, -1.0, -1.0)  # one kernel: nothing to time
    with pytest.raises(P.DPMMError) as e:
        g.set_kernel(7)
    assert e.value.status == P.DPMM_EINVAL
    g.close()
