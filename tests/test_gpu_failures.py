"""Failure detection through the C ABI, without any GPU fault: a device wait that runs
out ends with DPMM_ETIMEOUT in bounded time and leaves the context usable; NaN data
surface as DPMM_ENUMERIC at the next synchronising call (the factorisation meets a
non-positive pivot) and the error word clears; an allocation that cannot succeed
returns DPMM_ENOMEM."""
import time

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


def _data(d, N=5000, seed=3):
    import synth

    return synth.gaussian_mixture(N, d, 3, 6.0, seed=seed)[0]


def test_device_wait_times_out_and_context_survives():
    d = 32
    g = P.DPMM(0, d, 8, 2.0, prec=P.PREC_TF32, **_prior(d))
    g.set_data(_data(d))
    g.sweep(2, 1)
    t0 = time.time()
    st = P.dpmm_check_wait_timeout(g.h)
    el = time.time() - t0
    assert st == P.DPMM_ETIMEOUT
    assert el < 30.0, el
    # the error word is clear again and the tensor-core sweeps still run
    g.sweep(2, 1)
    z, zb = g.labels()
    assert z.min() >= 0 and z.max() < g.K
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nan_data_reported_as_numeric_error(prec):
    d = 4
    pr = P.PREC_FP64_PLAIN if prec == "fp64" else P.PREC_FP32
    X = _data(d).astype(np.float64 if prec == "fp64" else np.float32)
    X[17, 2] = np.nan
    g = P.DPMM(0, d, 8, 2.0, prec=pr, **_prior(d))
    g.set_data(X)
    g.sweep(1, 5)
    with pytest.raises(P.DPMMError) as e:
        g.labels()
    assert e.value.status == P.DPMM_ENUMERIC
    # clean data again: the context recovers
    g.set_data(_data(d).astype(X.dtype))
    g.sweep(2, 5)
    z, _ = g.labels()
    assert z.min() >= 0
    g.close()


def test_impossible_allocation_is_enomem():
    # N = 2^31 - 1 points of dimension 32 in FP64 need 550 GB of device memory: the
    # allocation fails before the input is read (the host buffer passed is one row)
    import ctypes as C

    d = 32
    g = P.DPMM(0, d, 4, 1.0, prec=P.PREC_FP64_PLAIN, **_prior(d))
    row = np.zeros(d)
    st = P.load().dpmm_set_data(g.h, C.c_void_p(row.ctypes.data), (1 << 31) - 1, P.F64, 0)
    assert st == P.DPMM_ENOMEM, (st, P.dpmm_last_error(g.h))
    # the context is still usable
    X = np.random.default_rng(0).standard_normal((500, d))
    g.set_data(X)
    g.sweep(1, 1)
    assert g.labels()[0].shape == (500,)
    g.close()
