"""FP64 CPU oracle of the sub-cluster split/merge DPMM sampler (arXiv 2204.08988,
Sec. 2.3 and Sec. 4.1).  TEST INFRASTRUCTURE ONLY: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it.

The arithmetic lives in ``dpmm_oracle.c`` (plain C, double precision, straight
loops).  This module only compiles it with gcc and marshals arguments through
ctypes.  It shares nothing with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpmm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libdpmm_oracle.so")
_lock = threading.Lock()
_lib = None

NIW = 0
DIRICHLET = 1

MASK_PARAMS = 1
MASK_LABELS = 2
MASK_SPLITMERGE = 4
MASK_ALL = 7


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only: it runs on x86 and Arm)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.POINTER
            d, i32, u32, u64, i64, vp = C.c_double, C.c_int, C.c_uint32, C.c_uint64, C.c_int64, C.c_void_p
            L.orc_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
            L.orc_u01.argtypes = [u32, u32]
            L.orc_u01.restype = d
            L.orc_u01_f32.argtypes = [u32]
            L.orc_u01_f32.restype = C.c_float
            L.orc_log_gamma_variate.argtypes = [u64, u32, u32, u32, u32, u32, d]
            L.orc_log_gamma_variate.restype = d
            L.orc_normal_variate.argtypes = [u64, u32, u32, u32, u32, u32, u32]
            L.orc_normal_variate.restype = d
            L.orc_create.argtypes = [i32, i32, i32, d, d, vp, d, vp, vp, i32, i32]
            L.orc_create.restype = vp
            L.orc_destroy.argtypes = [vp]
            L.orc_set_data.argtypes = [vp, vp, i64]
            L.orc_set_state.argtypes = [vp, i32, vp, vp]
            L.orc_sweep.argtypes = [vp, i32, u64, u32, C.c_uint]
            L.orc_draw_params_only.argtypes = [vp, u64, u32]
            L.orc_get_K.argtypes = [vp]
            L.orc_get_iter.argtypes = [vp]
            L.orc_get_iter.restype = u32
            L.orc_set_iter.argtypes = [vp, u32]
            L.orc_get_labels.argtypes = [vp, vp, vp]
            L.orc_get_stats.argtypes = [vp, vp, vp, vp]
            L.orc_get_params.argtypes = [vp, vp, vp, vp, vp, vp]
            L.orc_get_counters.argtypes = [vp, vp]
            L.orc_get_ages.argtypes = [vp, vp]
            L.orc_niw_posterior.argtypes = [vp, d, vp, vp, vp, vp, vp, vp]
            L.orc_niw_log_marginal.argtypes = [vp, d, vp, vp]
            L.orc_niw_log_marginal.restype = d
            L.orc_dirmult_log_marginal.argtypes = [vp, vp]
            L.orc_dirmult_log_marginal.restype = d
            L.orc_niw_draw.argtypes = [vp, u64, u32, u32, u32, d, vp, d, vp, vp, vp, vp]
            L.orc_dirichlet_draw.argtypes = [vp, u64, u32, u32, u32, vp, vp]
            L.orc_label_probe.argtypes = [vp, u64, u32, u32, vp, vp]
            L.orc_label_probe_points.argtypes = [vp, u64, u32, u32, vp, i64, vp, vp]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def u01(a, b):
    return lib().orc_u01(a & 0xFFFFFFFF, b & 0xFFFFFFFF)


def u01_f32(a):
    return lib().orc_u01_f32(a & 0xFFFFFFFF)


def log_gamma_variate(seed, it, problem, c0, tag, base, a):
    return lib().orc_log_gamma_variate(seed, it, problem, c0, tag, base, float(a))


def normal_variate(seed, it, problem, c0, tag, base, q):
    return lib().orc_normal_variate(seed, it, problem, c0, tag, base, q)


class Oracle:
    """One DPMM chain in the oracle.  Gaussian/NIW (kind=NIW) or multinomial/Dirichlet."""

    def __init__(self, kind, d, K_max, alpha, kappa0=1.0, m0=None, nu0=None, psi0=None,
                 beta=None, init_K=1, burn_out=15):
        self.kind, self.d, self.K_max = kind, d, K_max
        m0 = np.zeros(d) if m0 is None else np.ascontiguousarray(m0, dtype=np.float64)
        psi0 = np.eye(d) if psi0 is None else np.ascontiguousarray(psi0, dtype=np.float64)
        beta = np.ones(d) if beta is None else np.ascontiguousarray(beta, dtype=np.float64)
        nu0 = float(d + 3) if nu0 is None else float(nu0)
        self._keep = (m0, psi0, beta)
        self.h = lib().orc_create(kind, d, K_max, float(alpha), float(kappa0), _p(m0), nu0, _p(psi0),
                                  _p(beta), init_K, burn_out)
        if not self.h:
            raise ValueError("oracle: invalid hyper-parameters")
        self.N = 0

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def set_data(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64)
        assert X.ndim == 2 and X.shape[1] == self.d
        self.N = X.shape[0]
        if lib().orc_set_data(self.h, _p(X), self.N) != 0:
            raise ValueError("oracle: bad data")

    def set_state(self, K, z, zbar):
        z = np.ascontiguousarray(z, dtype=np.int32)
        zb = np.ascontiguousarray(zbar, dtype=np.uint8)
        if lib().orc_set_state(self.h, K, _p(z), _p(zb)) != 0:
            raise ValueError("oracle: bad state")

    def sweep(self, iters, seed, mask=MASK_ALL, problem=0):
        r = lib().orc_sweep(self.h, iters, seed, problem, mask)
        if r != 0:
            raise RuntimeError("oracle: sweep failed (%d)" % r)

    def draw_params(self, seed, problem=0):
        lib().orc_draw_params_only(self.h, seed, problem)

    @property
    def K(self):
        return lib().orc_get_K(self.h)

    @property
    def iter(self):
        return lib().orc_get_iter(self.h)

    @iter.setter
    def iter(self, t):
        lib().orc_set_iter(self.h, t)

    def labels(self):
        z = np.empty(self.N, np.int32)
        zb = np.empty(self.N, np.uint8)
        lib().orc_get_labels(self.h, _p(z), _p(zb))
        return z, zb

    def stats(self):
        S, d = 3 * self.K, self.d
        n = np.empty(S)
        sx = np.empty((S, d))
        sxx = np.empty((S, d, d)) if self.kind == NIW else None
        lib().orc_get_stats(self.h, _p(n), _p(sx), _p(sxx) if sxx is not None else None)
        return n, sx, sxx

    def params(self):
        S, d = 3 * self.K, self.d
        logw = np.empty(S)
        if self.kind == NIW:
            mu, W, ld = np.empty((S, d)), np.empty((S, d, d)), np.empty(S)
            lib().orc_get_params(self.h, _p(logw), _p(mu), _p(W), _p(ld), None)
            return dict(logw=logw, mu=mu, W=W, logdetW=ld)
        lt = np.empty((S, d))
        lib().orc_get_params(self.h, _p(logw), None, None, None, _p(lt))
        return dict(logw=logw, logtheta=lt)

    def label_probe(self, seed, it, problem=0):
        """Labels the current parameters give at sweep index `it` (state untouched)."""
        z = np.empty(self.N, np.int32)
        zb = np.empty(self.N, np.uint8)
        lib().orc_label_probe(self.h, seed, it, problem, _p(z), _p(zb))
        return z, zb

    def label_probe_points(self, seed, it, idx, problem=0):
        """label_probe for the points idx only (global indices; same random streams)."""
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        assert idx.size == 0 or (idx.min() >= 0 and idx.max() < self.N)
        z = np.empty(idx.size, np.int32)
        zb = np.empty(idx.size, np.uint8)
        lib().orc_label_probe_points(self.h, seed, it, problem, _p(idx), idx.size, _p(z), _p(zb))
        return z, zb

    def counters(self):
        c = np.zeros(4, np.int32)
        lib().orc_get_counters(self.h, _p(c))
        return dict(splits=int(c[0]), merges=int(c[1]), split_rejected_kmax=int(c[2]), removed=int(c[3]))

    def ages(self):
        a = np.zeros(self.K, np.int32)
        lib().orc_get_ages(self.h, _p(a))
        return a

    # --- closed forms, exposed for the pins ---------------------------------
    def niw_posterior(self, n, sx, sxx):
        d = self.d
        sx = np.ascontiguousarray(sx, dtype=np.float64)
        sxx = np.ascontiguousarray(sxx, dtype=np.float64)
        kn, nun = C.c_double(), C.c_double()
        mn, psin = np.empty(d), np.empty((d, d))
        lib().orc_niw_posterior(self.h, float(n), _p(sx), _p(sxx), C.byref(kn), _p(mn), C.byref(nun), _p(psin))
        return kn.value, mn, nun.value, psin

    def niw_log_marginal(self, n, sx, sxx):
        sx = np.ascontiguousarray(sx, dtype=np.float64)
        sxx = np.ascontiguousarray(sxx, dtype=np.float64)
        return lib().orc_niw_log_marginal(self.h, float(n), _p(sx), _p(sxx))

    def log_marginal_points(self, X):
        """f_x(C; lambda) of a set of points (rows of X)."""
        X = np.asarray(X, dtype=np.float64).reshape(-1, self.d)
        if self.kind == NIW:
            return self.niw_log_marginal(X.shape[0], X.sum(0), X.T @ X)
        return self.dirmult_log_marginal(X.sum(0))

    def dirmult_log_marginal(self, counts):
        c = np.ascontiguousarray(counts, dtype=np.float64)
        return lib().orc_dirmult_log_marginal(self.h, _p(c))

    def niw_draw(self, seed, it, slot, kn, mn, nun, psin, problem=0):
        d = self.d
        mn = np.ascontiguousarray(mn, dtype=np.float64)
        psin = np.ascontiguousarray(psin, dtype=np.float64)
        W, mu, ld = np.empty((d, d)), np.empty(d), C.c_double()
        lib().orc_niw_draw(self.h, seed, it, problem, slot, float(kn), _p(mn), float(nun), _p(psin),
                           _p(W), _p(mu), C.byref(ld))
        return W, mu, ld.value

    def dirichlet_draw(self, seed, it, slot, counts, problem=0):
        c = np.ascontiguousarray(counts, dtype=np.float64)
        lt = np.empty(self.d)
        lib().orc_dirichlet_draw(self.h, seed, it, problem, slot, _p(c), _p(lt))
        return lt
