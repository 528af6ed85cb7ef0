"""The C-ABI library loads, exports every symbol include/dpmm.h declares, and
rejects bad arguments before touching a device (no GPU needed)."""
import os
import re

import numpy as np
import pytest

import paper_2204_08988_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_08988_gb300 import _build

    _build.build()
    return P.load()


def test_header_and_exports_agree(lib):
    hdr = open(os.path.join(ROOT, "include", "dpmm.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = set(re.findall(r"\b(dpmm_[a-z_]+)\s*\(", hdr))
    assert declared == set(P.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def _create(**kw):
    d = kw.pop("d", 2)
    args = dict(kind=P.PRIOR_NIW, d=d, K_max=8, alpha=1.0)
    args.update(kw)
    return P.dpmm_create(**args)


@pytest.mark.parametrize("bad", [
    dict(alpha=0.0), dict(alpha=-1.0), dict(d=0), dict(K_max=0), dict(K_max=1001), dict(kappa0=0.0), dict(nu0=1.0),
    dict(d=161, nu0=170.0),
    dict(psi0=np.array([[1.0, 2.0], [2.0, 1.0]])), dict(psi0=np.array([[1.0, 0.5], [0.4, 1.0]])),
])
def test_invalid_niw_hyperparameters_rejected(lib, bad):
    with pytest.raises(P.DPMMError) as e:
        _create(**bad)
    assert e.value.status == P.DPMM_EINVAL


def test_invalid_dirichlet_rejected(lib):
    with pytest.raises(P.DPMMError) as e:
        P.dpmm_create(P.PRIOR_DIRICHLET, 3, 4, 1.0, beta=np.array([1.0, 0.0, 1.0]))
    assert e.value.status == P.DPMM_EINVAL


def test_no_device_means_no_fallback(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.DPMMError) as e:
        _create()
    assert e.value.status == P.DPMM_ECUDA
