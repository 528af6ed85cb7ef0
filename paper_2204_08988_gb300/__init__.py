"""GB300-native data-parallel hot path of the sub-cluster split/merge DPMM sampler
(arXiv 2204.08988, Sec. 4.1).

The compute path is the CUDA library ``libdpmm.so`` (C ABI in ``include/dpmm.h``);
this module only loads it with ctypes and marshals arguments.  Functions keep the
C names (``dpmm_create``, ``dpmm_sweep``, ...).  ``DPMM`` is a small convenience
wrapper over them.  There is no CPU fallback: without the library or a GPU every
call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libdpmm.so")
_lock = threading.Lock()
_lib = None

DPMM_OK, DPMM_EINVAL, DPMM_ENOMEM, DPMM_ECUDA, DPMM_ESTATE, DPMM_ENUMERIC, DPMM_ETIMEOUT = range(7)
PRIOR_NIW, PRIOR_DIRICHLET = 0, 1
F64, F32, BF16, I32 = 0, 1, 2, 3
PREC_FP64_PLAIN, PREC_TF32, PREC_BF16, PREC_FP32, PREC_BF16X3 = 0, 1, 2, 3, 4
KERNEL_TENSOR, KERNEL_CUDA_CORE, KERNEL_AUTO = 0, 1, 2
_STATUS = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ESTATE", 5: "ENUMERIC", 6: "ETIMEOUT"}

# every symbol include/dpmm.h declares
EXPORTS = [
    "dpmm_create", "dpmm_set_options", "dpmm_set_data", "dpmm_update_data", "dpmm_sweep", "dpmm_get_labels",
    "dpmm_get_stats", "dpmm_get_info", "dpmm_get_counters", "dpmm_last_error", "dpmm_destroy",
    "dpmm_set_state", "dpmm_set_step_mask", "dpmm_set_params", "dpmm_get_params", "dpmm_set_iter",
    "dpmm_profile", "dpmm_get_profile", "dpmm_suffstats_noalloc", "dpmm_label_scores", "dpmm_set_problem",
    "dpmm_sweep_batch", "dpmm_check_wait_timeout", "dpmm_checkpoint_size", "dpmm_save_checkpoint",
    "dpmm_load_checkpoint", "dpmm_set_data_csr", "dpmm_set_shard", "dpmm_sweep_sharded", "dpmm_set_kernel",
    "dpmm_get_kernel", "dpmm_stage_data",
]


class DPMMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class _Prior(C.Structure):
    _fields_ = [("kind", C.c_int), ("kappa0", C.c_double), ("m0", C.c_void_p), ("nu0", C.c_double),
                ("psi0", C.c_void_p), ("beta", C.c_void_p)]


def lib_path():
    return _LIB_PATH


def load():
    """Load libdpmm.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libdpmm.so is not built: run __graft_entry__.build() (no CPU fallback exists)")
        L = C.CDLL(_LIB_PATH)
        vp, i32, u32, u64, i64, d = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_int64, C.c_double
        sig = {
            "dpmm_create": ([C.POINTER(_Prior), d, i32, i32, C.POINTER(vp)], i32),
            "dpmm_set_options": ([vp, i32, i32, i32, vp], i32),
            "dpmm_set_data": ([vp, vp, i64, i32, i32], i32),
            "dpmm_update_data": ([vp, vp, i32, i32], i32),
            "dpmm_sweep": ([vp, i32, u64], i32),
            "dpmm_get_labels": ([vp, vp, vp], i32),
            "dpmm_get_stats": ([vp, C.POINTER(i32), vp, vp, vp, vp], i32),
            "dpmm_get_info": ([vp, C.POINTER(i32), C.POINTER(u32)], i32),
            "dpmm_get_counters": ([vp, vp], i32),
            "dpmm_last_error": ([vp], C.c_char_p),
            "dpmm_destroy": ([vp], None),
            "dpmm_set_state": ([vp, i32, vp, vp], i32),
            "dpmm_set_step_mask": ([vp, C.c_uint], i32),
            "dpmm_set_params": ([vp, i32, vp, vp, vp, vp, vp], i32),
            "dpmm_get_params": ([vp, vp, vp, vp, vp, vp], i32),
            "dpmm_set_iter": ([vp, u32], i32),
            "dpmm_profile": ([vp, i32], i32),
            "dpmm_get_profile": ([vp, i32, vp, vp, vp, C.POINTER(i32)], i32),
            "dpmm_suffstats_noalloc": ([vp, i64, i32, vp, vp, i32, vp, vp, vp, vp], i32),
            "dpmm_label_scores": ([vp, vp], i32),
            "dpmm_set_problem": ([vp, u32], i32),
            "dpmm_sweep_batch": ([vp, i32, i32, u64], i32),
            "dpmm_check_wait_timeout": ([vp], i32),
            "dpmm_checkpoint_size": ([vp, C.POINTER(C.c_size_t)], i32),
            "dpmm_save_checkpoint": ([vp, vp, C.c_size_t], i32),
            "dpmm_load_checkpoint": ([vp, vp, C.c_size_t], i32),
            "dpmm_set_data_csr": ([vp, vp, vp, vp, i64], i32),
            "dpmm_set_shard": ([vp, i64], i32),
            "dpmm_sweep_sharded": ([vp, i32, i32, u64], i32),
            "dpmm_set_kernel": ([vp, i32], i32),
            "dpmm_stage_data": ([vp, vp, i32], i32),
            "dpmm_get_kernel": ([vp, C.POINTER(i32), C.POINTER(C.c_float), C.POINTER(C.c_float)], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def _p(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _check(h, st):
    if st != DPMM_OK:
        msg = load().dpmm_last_error(h) if h else b""
        raise DPMMError(st, (msg or b"").decode())


# ------------------------------------------------------------- C-named wrappers
def dpmm_create(kind, d, K_max, alpha, kappa0=1.0, m0=None, nu0=None, psi0=None, beta=None):
    L = load()
    niw = kind == PRIOR_NIW  # the prior's unused fields get a one-element placeholder
    m0 = np.ascontiguousarray((np.zeros(d) if niw else np.zeros(1)) if m0 is None else m0, dtype=np.float64)
    psi0 = np.ascontiguousarray((np.eye(d) if niw else np.ones(1)) if psi0 is None else psi0, dtype=np.float64)
    beta = np.ascontiguousarray((np.ones(d) if not niw else np.ones(1)) if beta is None else beta, dtype=np.float64)
    pr = _Prior(kind, float(kappa0), m0.ctypes.data, float(d + 3 if nu0 is None else nu0), psi0.ctypes.data,
                beta.ctypes.data)
    h = C.c_void_p()
    _check(None, L.dpmm_create(C.byref(pr), float(alpha), int(d), int(K_max), C.byref(h)))
    return h


def dpmm_set_options(h, prec, init_K=1, burn_out=15, stream=None):
    _check(h, load().dpmm_set_options(h, prec, init_K, burn_out, stream))


def _array_arg(X):
    """(pointer, dtype code, on_device) for a numpy array or a CUDA torch tensor."""
    if hasattr(X, "data_ptr"):  # torch tensor
        import torch

        code = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16, torch.int32: I32}[X.dtype]
        assert X.is_contiguous()
        return C.c_void_p(X.data_ptr()), code, 1 if X.is_cuda else 0
    X = np.ascontiguousarray(X)
    code = {np.dtype(np.float64): F64, np.dtype(np.float32): F32, np.dtype(np.int32): I32}[X.dtype]
    return C.c_void_p(X.ctypes.data), code, 0


def dpmm_set_data(h, X):
    ptr, code, dev = _array_arg(X)
    _check(h, load().dpmm_set_data(h, ptr, int(X.shape[0]), code, dev))


def dpmm_set_data_csr(h, indptr, indices, counts):
    """Compressed rows (host arrays): indptr int64[N + 1], indices int32[nnz], counts int32[nnz]."""
    ip = np.ascontiguousarray(indptr, dtype=np.int64)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    ct = np.ascontiguousarray(counts, dtype=np.int32)
    _check(h, load().dpmm_set_data_csr(h, _p(ip), _p(ix), _p(ct), int(ip.size - 1)))


def dpmm_update_data(h, X):
    ptr, code, dev = _array_arg(X)
    _check(h, load().dpmm_update_data(h, ptr, code, dev))


def dpmm_stage_data(h, X):
    """Stage host values for the next sweep (copied while the current sweep runs)."""
    ptr, code, dev = _array_arg(X)
    if dev:
        raise ValueError("dpmm_stage_data takes host memory")
    _check(h, load().dpmm_stage_data(h, ptr, code))


def dpmm_sweep(h, iters, seed):
    _check(h, load().dpmm_sweep(h, int(iters), int(seed)))


def dpmm_get_labels(h, N, z=None, zbar=None):
    z = np.empty(N, np.int32) if z is None else z
    zb = np.empty(N, np.uint8) if zbar is None else zbar
    _check(h, load().dpmm_get_labels(h, _p(z) if isinstance(z, np.ndarray) else C.c_void_p(z.data_ptr()),
                                     _p(zb) if isinstance(zb, np.ndarray) else C.c_void_p(zb.data_ptr())))
    return z, zb


def dpmm_get_info(h):
    K, it = C.c_int(), C.c_uint32()
    _check(h, load().dpmm_get_info(h, C.byref(K), C.byref(it)))
    return K.value, it.value


def dpmm_get_stats(h, d, K_max, gaussian=True):
    K = C.c_int()
    n = np.zeros(3 * K_max, np.int64)
    sx = np.zeros((3 * K_max, d))
    sxx = np.zeros((3 * K_max, d, d)) if gaussian else None
    w = np.zeros(K_max)
    _check(h, load().dpmm_get_stats(h, C.byref(K), _p(n), _p(sx), _p(sxx), _p(w)))
    k = K.value
    return k, n[: 3 * k], sx[: 3 * k], (sxx[: 3 * k] if gaussian else None), w[:k]


def dpmm_get_counters(h):
    out = np.zeros(4, np.int32)
    _check(h, load().dpmm_get_counters(h, _p(out)))
    return dict(splits=int(out[0]), merges=int(out[1]), split_rejected_kmax=int(out[2]), removed=int(out[3]))


def dpmm_set_state(h, K, z, zbar):
    z = np.ascontiguousarray(z, dtype=np.int32)
    zb = np.ascontiguousarray(zbar, dtype=np.uint8)
    _check(h, load().dpmm_set_state(h, int(K), _p(z), _p(zb)))


def dpmm_set_step_mask(h, mask):
    _check(h, load().dpmm_set_step_mask(h, int(mask)))


def dpmm_set_kernel(h, choice):
    _check(h, load().dpmm_set_kernel(h, int(choice)))


def dpmm_get_kernel(h):
    """(kernel in use, timed ms on the tensor cores, timed ms on the CUDA cores); -1: not timed."""
    use, mt, mc = C.c_int32(), C.c_float(), C.c_float()
    _check(h, load().dpmm_get_kernel(h, C.byref(use), C.byref(mt), C.byref(mc)))
    return use.value, mt.value, mc.value


def dpmm_set_iter(h, it):
    _check(h, load().dpmm_set_iter(h, int(it)))


def dpmm_set_problem(h, problem):
    _check(h, load().dpmm_set_problem(h, int(problem)))


def dpmm_save_checkpoint(h):
    """The chain's checkpoint as bytes."""
    n = C.c_size_t()
    _check(h, load().dpmm_checkpoint_size(h, C.byref(n)))
    buf = np.empty(n.value, dtype=np.uint8)
    _check(h, load().dpmm_save_checkpoint(h, _p(buf), n.value))
    return buf.tobytes()


def dpmm_load_checkpoint(h, data):
    buf = np.frombuffer(data, dtype=np.uint8).copy()
    _check(h, load().dpmm_load_checkpoint(h, _p(buf), buf.size))


def dpmm_check_wait_timeout(h):
    """Status of the bounded-wait check (DPMM_ETIMEOUT when device waits end as designed)."""
    return int(load().dpmm_check_wait_timeout(h))


def dpmm_sweep_batch(handles, iters, seed):
    """Sweeps of several chains (their handles), interleaved; asynchronous."""
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    st = load().dpmm_sweep_batch(arr, len(handles), int(iters), int(seed))
    if st != DPMM_OK:
        raise DPMMError(st, "dpmm_sweep_batch failed (see the failing chain's dpmm_last_error)")


def dpmm_set_shard(h, point_offset):
    _check(h, load().dpmm_set_shard(h, int(point_offset)))


def dpmm_sweep_sharded(handles, iters, seed):
    """Sweeps of one chain whose points are split over the given contexts (in order)."""
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    st = load().dpmm_sweep_sharded(arr, len(handles), int(iters), int(seed))
    if st != DPMM_OK:
        msgs = [dpmm_last_error(h) for h in handles]
        raise DPMMError(st, "; ".join(m for m in msgs if m) or "dpmm_sweep_sharded failed")


def shard_allreduce(table, group=None):
    """The sum of a statistics table over the ranks of a torch.distributed process group,
    added in rank order (rank 0 + rank 1 + ...), the same bits on every rank: the exchange
    of a point-sharded chain across processes (one GPU each).  `table` is a numpy array;
    every rank passes the same shape."""
    import torch
    import torch.distributed as dist

    t = torch.from_numpy(np.ascontiguousarray(table))
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t, group=group)
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out.numpy()


def dpmm_set_params(h, K, logw, mu=None, W=None, logdetW=None, logtheta=None):
    a = [None if v is None else np.ascontiguousarray(v, dtype=np.float64) for v in (logw, mu, W, logdetW, logtheta)]
    _check(h, load().dpmm_set_params(h, int(K), *[_p(v) for v in a]))


def dpmm_get_params(h, d, gaussian=True):
    K, _ = dpmm_get_info(h)
    S = 3 * K
    logw = np.empty(S)
    if gaussian:
        mu, W, ld = np.empty((S, d)), np.empty((S, d, d)), np.empty(S)
        _check(h, load().dpmm_get_params(h, _p(logw), _p(mu), _p(W), _p(ld), None))
        return dict(logw=logw, mu=mu, W=W, logdetW=ld)
    lt = np.empty((S, d))
    _check(h, load().dpmm_get_params(h, _p(logw), None, None, None, _p(lt)))
    return dict(logw=logw, logtheta=lt)


def dpmm_label_scores(h, N, K):
    out = np.empty((N, K))
    _check(h, load().dpmm_label_scores(h, _p(out)))
    return out


def dpmm_profile(h, enable):
    _check(h, load().dpmm_profile(h, int(enable)))


def dpmm_get_profile(h):
    cap = 64
    names = (C.c_char_p * cap)()
    launches = np.zeros(cap, np.int32)
    ms = np.zeros(cap)
    cnt = C.c_int()
    _check(h, load().dpmm_get_profile(h, cap, C.cast(names, C.c_void_p), _p(launches), _p(ms), C.byref(cnt)))
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(min(cnt.value, cap))}


def dpmm_suffstats_noalloc(X, z, zbar, K, n_out, sx_out, sxx_out, stream=None):
    """Statistics of given labels with no allocation (CUDA tensors in and out).

    X is N x d float32, z int32[N], zbar uint8[N]; the outputs are float64 with at
    least 2K, 2K*d and 2K*d*d elements.  All must be contiguous and on the current
    device.  The call is ordered on `stream` (a cudaStream_t handle), by default on
    torch's current stream."""
    import torch

    if X.dim() != 2:
        raise ValueError("X must be N x d")
    N, d = X.shape
    dev = torch.cuda.current_device()
    want = [(X, torch.float32, "X", None), (z, torch.int32, "z", N), (zbar, torch.uint8, "zbar", N),
            (n_out, torch.float64, "n_out", 2 * K), (sx_out, torch.float64, "sx_out", 2 * K * d),
            (sxx_out, torch.float64, "sxx_out", 2 * K * d * d)]
    for t, dt, name, numel in want:
        if not t.is_cuda or t.device.index != dev:
            raise ValueError("%s must be a CUDA tensor on the current device" % name)
        if t.dtype != dt:
            raise ValueError("%s must be %s, not %s" % (name, dt, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        if numel is not None and t.numel() < numel:
            raise ValueError("%s needs at least %d elements" % (name, numel))
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    st = load().dpmm_suffstats_noalloc(C.c_void_p(X.data_ptr()), int(N), int(d), C.c_void_p(z.data_ptr()),
                                       C.c_void_p(zbar.data_ptr()), int(K), C.c_void_p(n_out.data_ptr()),
                                       C.c_void_p(sx_out.data_ptr()), C.c_void_p(sxx_out.data_ptr()),
                                       C.c_void_p(stream))
    _check(None, st)


def dpmm_last_error(h):
    return (load().dpmm_last_error(h) or b"").decode()


def dpmm_destroy(h):
    if h:
        load().dpmm_destroy(h)


class DPMM:
    """One chain on the GPU: a thin object over the C-named functions."""

    def __init__(self, kind, d, K_max, alpha, prec=PREC_FP64_PLAIN, init_K=1, burn_out=15, stream=None, **prior):
        self.kind, self.d, self.K_max = kind, d, K_max
        self.h = dpmm_create(kind, d, K_max, alpha, **prior)
        dpmm_set_options(self.h, prec, init_K, burn_out, stream)
        self.N = 0

    def close(self):
        if getattr(self, "h", None):
            dpmm_destroy(self.h)
            self.h = None

    __del__ = close

    def set_data(self, X):
        dpmm_set_data(self.h, X)
        self.N = int(X.shape[0])

    def update_data(self, X):
        dpmm_update_data(self.h, X)

    def stage_data(self, X):
        dpmm_stage_data(self.h, X)

    def set_data_csr(self, indptr, indices, counts):
        dpmm_set_data_csr(self.h, indptr, indices, counts)
        self.N = int(len(indptr) - 1)

    def sweep(self, iters, seed):
        dpmm_sweep(self.h, iters, seed)

    def labels(self):
        return dpmm_get_labels(self.h, self.N)

    def info(self):
        return dpmm_get_info(self.h)

    @property
    def K(self):
        return self.info()[0]

    def stats(self):
        K, n, sx, sxx, w = dpmm_get_stats(self.h, self.d, self.K_max, self.kind == PRIOR_NIW)
        return n.astype(np.float64), sx, sxx

    def weights(self):
        return dpmm_get_stats(self.h, self.d, self.K_max, self.kind == PRIOR_NIW)[4]

    def counters(self):
        return dpmm_get_counters(self.h)

    def set_state(self, K, z, zbar):
        dpmm_set_state(self.h, K, z, zbar)

    def set_mask(self, mask):
        dpmm_set_step_mask(self.h, mask)

    def set_kernel(self, choice):
        dpmm_set_kernel(self.h, choice)

    def kernel(self):
        return dpmm_get_kernel(self.h)

    def set_iter(self, it):
        dpmm_set_iter(self.h, it)

    def set_problem(self, problem):
        dpmm_set_problem(self.h, problem)

    def set_shard(self, point_offset):
        dpmm_set_shard(self.h, point_offset)

    def checkpoint(self):
        return dpmm_save_checkpoint(self.h)

    def restore(self, data):
        dpmm_load_checkpoint(self.h, data)

    def set_params(self, K, p):
        if self.kind == PRIOR_NIW:
            dpmm_set_params(self.h, K, p["logw"], p["mu"], p["W"], p["logdetW"], None)
        else:
            dpmm_set_params(self.h, K, p["logw"], None, None, None, p["logtheta"])

    def params(self):
        return dpmm_get_params(self.h, self.d, self.kind == PRIOR_NIW)

    def label_scores(self):
        return dpmm_label_scores(self.h, self.N, self.K)
