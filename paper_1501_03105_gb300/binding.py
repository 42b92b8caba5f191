"""Thin ctypes binding of libpirmcut (the C ABI declared in include/pirmcut.h).

Argument marshalling only: every step of the IRLS path runs in the library's
CUDA kernels.  The functions carry the names of the C entry points.  Arrays
are numpy arrays (host memory) or torch tensors (host or CUDA memory); the
memory kind passed to the library follows the array.  Importing this module
does not load the library; the first call does, and it raises
``RuntimeError`` when ``libpirmcut.so`` has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpirmcut.so")

MEM_HOST, MEM_DEVICE = 0, 1
REWEIGHT_WEIGHTED_L1, REWEIGHT_PAPER = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
FORMAT_AUTO, FORMAT_DIA, FORMAT_CSR = 0, 1, 2
MLP_PREDICT, MLP_TRAIN = 1, 2
MLP_FEATURES, MLP_PARAMS = 6, 4673

STATUS = {0: "OK", 1: "EINVAL", 2: "EDISCONNECTED", 3: "ENOMEM", 4: "ECUDA",
          5: "ENOCONV", 6: "ETIMEOUT", 7: "ENUMERIC"}
OK, EINVAL, EDISCONNECTED, ENOMEM, ECUDA, ENOCONV, ETIMEOUT, ENUMERIC = range(8)


class Options(ctypes.Structure):
    _fields_ = [("reweight_form", ctypes.c_int), ("precision", ctypes.c_int),
                ("pcg_tol", ctypes.c_double), ("pcg_max_iter", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("format", ctypes.c_int),
                ("track_cut", ctypes.c_int), ("graph_launch", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("time_spmv", ctypes.c_int),
                ("reduce_on_host", ctypes.c_int), ("batch_threads_per_row", ctypes.c_int),
                ("batch_tile_rows", ctypes.c_int), ("batch_medium_deg", ctypes.c_int),
                ("step_stats", ctypes.c_int), ("capacity_fp32", ctypes.c_int),
                ("fuse_reweight", ctypes.c_int)]


class StepInfo(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int), ("pcg_iters", ctypes.c_int), ("eps", ctypes.c_double),
                ("rel_residual", ctypes.c_double), ("x_min", ctypes.c_double),
                ("x_max", ctypes.c_double), ("cut_value", ctypes.c_double),
                ("ms", ctypes.c_double), ("status", ctypes.c_int), ("refinements", ctypes.c_int),
                ("objective", ctypes.c_double), ("flow_value", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class MlpInfo(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("used", ctypes.c_int), ("train_steps", ctypes.c_int),
                ("loss", ctypes.c_float), ("alpha", ctypes.c_double),
                ("energy_change", ctypes.c_double), ("res_plain", ctypes.c_double),
                ("mean_alpha", ctypes.c_double), ("tensor_timeouts", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PirmcutError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


_LIB = None
_P = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Load libpirmcut.so (once)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_1501_03105_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.pirmcut_default_options.argtypes = [ctypes.POINTER(Options)]
    L.pirmcut_default_options.restype = None
    L.pirmcut_create.argtypes = [i64, _P, _P, _P, i32, i32, ctypes.POINTER(Options), ctypes.c_int,
                                 _P, ctypes.POINTER(_P)]
    L.pirmcut_create.restype = ctypes.c_int
    L.pirmcut_initial.argtypes = [_P, ctypes.POINTER(StepInfo)]
    L.pirmcut_initial.restype = ctypes.c_int
    L.pirmcut_irls_step.argtypes = [_P, dbl, ctypes.POINTER(StepInfo)]
    L.pirmcut_irls_step.restype = ctypes.c_int
    L.pirmcut_solve.argtypes = [_P, ctypes.c_int, _P, _P]
    L.pirmcut_solve.restype = ctypes.c_int
    L.pirmcut_cut.argtypes = [_P, _P, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.c_int]
    L.pirmcut_cut.restype = ctypes.c_int
    L.pirmcut_get_x.argtypes = [_P, _P, ctypes.c_int]
    L.pirmcut_get_x.restype = ctypes.c_int
    L.pirmcut_set_x.argtypes = [_P, _P, ctypes.c_int]
    L.pirmcut_set_x.restype = ctypes.c_int
    L.pirmcut_update_weights.argtypes = [_P, _P, ctypes.c_int]
    L.pirmcut_update_weights.restype = ctypes.c_int
    L.pirmcut_problem_size.argtypes = [_P, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                       ctypes.POINTER(ctypes.c_int)]
    L.pirmcut_problem_size.restype = ctypes.c_int
    L.pirmcut_time_spmv.argtypes = [_P, ctypes.c_int, ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                    ctypes.POINTER(dbl)]
    L.pirmcut_time_spmv.restype = ctypes.c_int
    L.pirmcut_sweep_cut_static.argtypes = [i64, _P, _P, _P, i32, i32, _P, _P, _P, _P]
    L.pirmcut_sweep_cut_static.restype = ctypes.c_int
    L.pirmcut_cut_two_level.argtypes = [_P, _P, ctypes.POINTER(dbl), _P, ctypes.POINTER(i64), ctypes.c_int]
    L.pirmcut_cut_two_level.restype = ctypes.c_int
    PP = ctypes.POINTER(ctypes.c_void_p)
    L.pirmcut_batch_create.argtypes = [ctypes.c_int, _P, PP, PP, PP, _P, _P, ctypes.POINTER(Options),
                                       _P, ctypes.POINTER(_P)]
    L.pirmcut_batch_create.restype = ctypes.c_int
    L.pirmcut_batch_solve.argtypes = [_P, ctypes.c_int, _P, _P]
    L.pirmcut_batch_solve.restype = ctypes.c_int
    L.pirmcut_batch_cut.argtypes = [_P, ctypes.c_int, _P, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    L.pirmcut_batch_cut.restype = ctypes.c_int
    L.pirmcut_batch_get_x.argtypes = [_P, ctypes.c_int, _P]
    L.pirmcut_batch_get_x.restype = ctypes.c_int
    L.pirmcut_batch_info.argtypes = [_P, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(i64)]
    L.pirmcut_batch_info.restype = ctypes.c_int
    L.pirmcut_batch_kernel_launches.argtypes = [_P]
    L.pirmcut_batch_kernel_launches.restype = i64
    L.pirmcut_batch_destroy.argtypes = [_P]
    L.pirmcut_batch_destroy.restype = None
    L.pirmcut_mlp_enable.argtypes = [_P, ctypes.c_int, ctypes.c_uint64]
    L.pirmcut_mlp_enable.restype = ctypes.c_int
    L.pirmcut_mlp_configure.argtypes = [_P, ctypes.c_int, ctypes.c_float]
    L.pirmcut_mlp_configure.restype = ctypes.c_int
    L.pirmcut_mlp_predict.argtypes = [_P, _P, i64, _P, ctypes.c_int]
    L.pirmcut_mlp_predict.restype = ctypes.c_int
    L.pirmcut_mlp_weights.argtypes = [_P, _P, ctypes.c_int]
    L.pirmcut_mlp_weights.restype = ctypes.c_int
    L.pirmcut_mlp_stats.argtypes = [_P, ctypes.POINTER(MlpInfo)]
    L.pirmcut_mlp_stats.restype = ctypes.c_int
    L.pirmcut_mlp_time_predict.argtypes = [_P, _P, ctypes.c_int64, _P, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_double)]
    L.pirmcut_mlp_time_predict.restype = ctypes.c_int
    L.pirmcut_mlp_features.argtypes = [_P, _P]
    L.pirmcut_mlp_features.restype = ctypes.c_int
    L.pirmcut_spmv_timing.argtypes = [_P, ctypes.POINTER(dbl), ctypes.POINTER(i64), ctypes.c_int]
    L.pirmcut_spmv_timing.restype = ctypes.c_int
    L.pirmcut_kernel_launches.argtypes = [_P]
    L.pirmcut_kernel_launches.restype = i64
    L.pirmcut_last_error.argtypes = [_P]
    L.pirmcut_last_error.restype = ctypes.c_char_p
    L.pirmcut_destroy.argtypes = [_P]
    L.pirmcut_destroy.restype = None
    _LIB = L
    return L


def _ptr(a, dtype):
    """(pointer, mem_kind, keepalive) of a numpy array or torch tensor of ``dtype``."""
    if a is None:
        return None, MEM_HOST, None
    if isinstance(a, np.ndarray):
        arr = np.ascontiguousarray(a, dtype=dtype)
        return arr.ctypes.data, MEM_HOST, arr
    import torch  # only for tensors
    if not isinstance(a, torch.Tensor):
        arr = np.ascontiguousarray(np.asarray(a), dtype=dtype)
        return arr.ctypes.data, MEM_HOST, arr
    tdt = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32,
           np.uint8: torch.uint8, np.float32: torch.float32}[np.dtype(dtype).type]
    if a.dtype != tdt or not a.is_contiguous():
        raise TypeError(f"tensor must be contiguous {tdt}")
    return a.data_ptr(), (MEM_DEVICE if a.is_cuda else MEM_HOST), a


def _check(h, status: int, soft=(OK,)):
    if status in soft:
        return status
    msg = lib().pirmcut_last_error(h)
    raise PirmcutError(status, msg.decode() if msg else "")


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def pirmcut_default_options(**kw) -> Options:
    o = Options()
    lib().pirmcut_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def pirmcut_create(n, row_ptr, col, c, s, t, opt: Options | None = None, stream=None):
    """Create a context; returns the opaque handle (int).  Raises PirmcutError.
    c is float64, or float32 when opt.capacity_fp32 is set."""
    prp, k1, a1 = _ptr(row_ptr, np.int64)
    pcl, k2, a2 = _ptr(col, np.int32)
    fp32 = opt is not None and opt.capacity_fp32
    pc, k3, a3 = _ptr(c, np.float32 if fp32 else np.float64)
    if len({k1, k2, k3}) != 1:
        raise ValueError("row_ptr, col and c must live in the same memory")
    h = _P()
    st = lib().pirmcut_create(int(n), prp, pcl, pc, int(s), int(t),
                              ctypes.byref(opt) if opt is not None else None, k1,
                              _stream_ptr(stream), ctypes.byref(h))
    _check(None, st)
    del a1, a2, a3
    return h.value


def pirmcut_initial(h) -> StepInfo:
    info = StepInfo()
    _check(h, lib().pirmcut_initial(h, ctypes.byref(info)), soft=(OK, ENOCONV))
    return info


def pirmcut_irls_step(h, eps: float) -> StepInfo:
    info = StepInfo()
    _check(h, lib().pirmcut_irls_step(h, float(eps), ctypes.byref(info)), soft=(OK, ENOCONV))
    return info


def pirmcut_solve(h, T: int, eps) -> list:
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    if eps.shape != (T,):
        raise ValueError("need one eps per step")
    infos = (StepInfo * (T + 1))()
    _check(h, lib().pirmcut_solve(h, int(T), eps.ctypes.data, ctypes.addressof(infos)),
           soft=(OK, ENOCONV))
    return list(infos)


def pirmcut_cut(h, side=None, n=None):
    """Sweep cut.  ``side``: a uint8 output array/tensor of length n, or None
    (a numpy array of length ``n`` is allocated when n is given).
    Returns (side, value, tau)."""
    if side is None and n is not None:
        side = np.zeros(int(n), dtype=np.uint8)
    ps, kind, keep = _ptr(side, np.uint8)
    if isinstance(side, np.ndarray) and keep is not side:
        raise TypeError("side must be a contiguous uint8 array")
    val = ctypes.c_double()
    tau = ctypes.c_double()
    _check(h, lib().pirmcut_cut(h, ps, ctypes.byref(val), ctypes.byref(tau), kind))
    return side, val.value, tau.value


def pirmcut_cut_two_level(h, side=None, n=None):
    """Two-level rounding.  Returns (side, value, (gamma0, gamma1), coarse_vertices)."""
    if side is None and n is not None:
        side = np.zeros(int(n), dtype=np.uint8)
    ps, kind, keep = _ptr(side, np.uint8)
    val = ctypes.c_double()
    gam = np.zeros(2, dtype=np.float64)
    nc = ctypes.c_int64()
    _check(h, lib().pirmcut_cut_two_level(h, ps, ctypes.byref(val), gam.ctypes.data, ctypes.byref(nc), kind))
    return side, val.value, (float(gam[0]), float(gam[1])), nc.value


def pirmcut_get_x(h, out):
    p, kind, keep = _ptr(out, np.float64)
    if isinstance(out, np.ndarray) and keep is not out:
        raise TypeError("out must be a contiguous float64 array")
    _check(h, lib().pirmcut_get_x(h, p, kind))
    return out


def pirmcut_set_x(h, x):
    p, kind, keep = _ptr(x, np.float64)
    _check(h, lib().pirmcut_set_x(h, p, kind))


def pirmcut_update_weights(h, c, fp32=False):
    """New capacities (float32 when the context was created with
    capacity_fp32, else float64) on the same structure."""
    p, kind, keep = _ptr(c, np.float32 if fp32 else np.float64)
    _check(h, lib().pirmcut_update_weights(h, p, kind))


def pirmcut_problem_size(h):
    a, b, f = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    _check(h, lib().pirmcut_problem_size(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(f)))
    return a.value, b.value, f.value


def pirmcut_time_spmv(h, reps: int = 20):
    """(mean ms per SpMV launch, algorithmic bytes, flops) on the current state."""
    ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(h, lib().pirmcut_time_spmv(h, int(reps), ctypes.byref(ms), ctypes.byref(by), ctypes.byref(fl)))
    return ms.value, by.value, fl.value


STATIC_MAX_NONTERMINALS = 65536


def pirmcut_sweep_cut_static(n, row_ptr, col, c, s, t, x, side, result, stream=None):
    """Allocation-free sweep cut on device-resident arrays (torch CUDA tensors):
    queues one kernel on ``stream``; ``side`` (uint8[n]) and ``result``
    (float64[4]: value, tau, k, bad-column flag) are filled on the device."""
    ptrs = []
    for a, dt in ((row_ptr, np.int64), (col, np.int32), (c, np.float64), (x, np.float64),
                  (side, np.uint8), (result, np.float64)):
        p, kind, _ = _ptr(a, dt)
        if kind != MEM_DEVICE:
            raise TypeError("every array must be in device memory")
        ptrs.append(p)
    st = lib().pirmcut_sweep_cut_static(int(n), ptrs[0], ptrs[1], ptrs[2], int(s), int(t),
                                        ptrs[3], ptrs[4], ptrs[5], _stream_ptr(stream))
    _check(None, st)


def pirmcut_mlp_enable(h, mode: int, seed: int = 1):
    _check(h, lib().pirmcut_mlp_enable(h, int(mode), int(seed) & (2**64 - 1)))


def pirmcut_mlp_configure(h, iters_per_step: int = 8, learning_rate: float = 1e-3):
    _check(h, lib().pirmcut_mlp_configure(h, int(iters_per_step), float(learning_rate)))


def pirmcut_mlp_predict(h, features, delta=None):
    """Raw model output for feature rows (numpy float32 [count, 6], or CUDA tensors)."""
    if isinstance(features, np.ndarray):
        f = np.ascontiguousarray(features, dtype=np.float32).reshape(-1, MLP_FEATURES)
        if delta is None:
            delta = np.empty(f.shape[0], dtype=np.float32)
        pf, kind, keep = _ptr(f, np.float32)
    else:
        pf, kind, keep = _ptr(features, np.float32)
        f = features
    pd, kind2, keep2 = _ptr(delta, np.float32)
    if kind != kind2:
        raise TypeError("features and delta must be in the same kind of memory")
    _check(h, lib().pirmcut_mlp_predict(h, pf, int(f.shape[0]), pd, kind))
    return delta


def pirmcut_mlp_time_predict(h, features, delta, reps=20):
    """Mean device time (ms) of one launch of the inference kernel on the
    device feature rows (reps back-to-back launches between CUDA events)."""
    pf, kf, a1 = _ptr(features, np.float32)
    pd, kd, a2 = _ptr(delta, np.float32)
    if kf != MEM_DEVICE or kd != MEM_DEVICE:
        raise ValueError("features and delta must be device tensors")
    ms = ctypes.c_double()
    _check(h, lib().pirmcut_mlp_time_predict(h, pf, int(features.shape[0]), pd, int(reps),
                                             ctypes.byref(ms)))
    return ms.value


def pirmcut_mlp_weights(h, w=None):
    """With ``w`` None: return the FP32 master weights (numpy float32[4673]).
    Otherwise load ``w`` into the model (optimizer state reset)."""
    if w is None:
        out = np.empty(MLP_PARAMS, dtype=np.float32)
        _check(h, lib().pirmcut_mlp_weights(h, out.ctypes.data, 0))
        return out
    a = np.ascontiguousarray(w, dtype=np.float32)
    if a.size != MLP_PARAMS:
        raise ValueError(f"expected {MLP_PARAMS} weights, got {a.size}")
    _check(h, lib().pirmcut_mlp_weights(h, a.ctypes.data, 1))
    return None


def pirmcut_mlp_stats(h) -> MlpInfo:
    info = MlpInfo()
    _check(h, lib().pirmcut_mlp_stats(h, ctypes.byref(info)))
    return info


def pirmcut_mlp_features(h, nt: int):
    out = np.empty((int(nt), MLP_FEATURES), dtype=np.float32)
    _check(h, lib().pirmcut_mlp_features(h, out.ctypes.data))
    return out


def pirmcut_spmv_timing(h, reset: bool = True):
    """(total ms, launches) of the SpMV launches timed live (time_spmv=1,
    graph_launch=0) since creation or the last reset."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    _check(h, lib().pirmcut_spmv_timing(h, ctypes.byref(ms), ctypes.byref(n), int(bool(reset))))
    return ms.value, n.value


def pirmcut_kernel_launches(h) -> int:
    return int(lib().pirmcut_kernel_launches(h))


def pirmcut_last_error(h=None) -> str:
    m = lib().pirmcut_last_error(h)
    return m.decode() if m else ""


def pirmcut_destroy(h):
    lib().pirmcut_destroy(h)


def pirmcut_batch_create(graphs, opt: Options | None = None, stream=None):
    """Create a batch from a list of graphs (host numpy arrays)."""
    k = len(graphs)
    keep = []
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    ss = np.array([g.s for g in graphs], dtype=np.int32)
    ts = np.array([g.t for g in graphs], dtype=np.int32)
    arrs = []
    for dt, attr in ((np.int64, "row_ptr"), (np.int32, "col"), (np.float64, "c")):
        ptrs = (ctypes.c_void_p * k)()
        for i, g in enumerate(graphs):
            a = np.ascontiguousarray(getattr(g, attr), dtype=dt)
            keep.append(a)
            ptrs[i] = a.ctypes.data
        arrs.append(ptrs)
    h = _P()
    st = lib().pirmcut_batch_create(k, ns.ctypes.data, arrs[0], arrs[1], arrs[2], ss.ctypes.data,
                                    ts.ctypes.data, ctypes.byref(opt) if opt is not None else None,
                                    _stream_ptr(stream), ctypes.byref(h))
    _check(None, st)
    return h.value


def pirmcut_batch_solve(h, count: int, T: int, eps):
    """Returns infos as a list (per instance) of lists of T+1 StepInfo."""
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    infos = (StepInfo * (count * (T + 1)))()
    st = lib().pirmcut_batch_solve(h, int(T), eps.ctypes.data, ctypes.addressof(infos))
    if st not in (OK, ENOCONV):
        msg = lib().pirmcut_last_error(None)
        raise PirmcutError(st, msg.decode() if msg else "")
    return [list(infos[i * (T + 1):(i + 1) * (T + 1)]) for i in range(count)]


def pirmcut_batch_cut(h, index: int, n: int):
    side = np.zeros(int(n), dtype=np.uint8)
    val, tau = ctypes.c_double(), ctypes.c_double()
    st = lib().pirmcut_batch_cut(h, int(index), side.ctypes.data, ctypes.byref(val), ctypes.byref(tau))
    if st != OK:
        msg = lib().pirmcut_last_error(None)
        raise PirmcutError(st, msg.decode() if msg else "")
    return side, val.value, tau.value


def pirmcut_batch_get_x(h, index: int, n: int):
    x = np.empty(int(n), dtype=np.float64)
    st = lib().pirmcut_batch_get_x(h, int(index), x.ctypes.data)
    if st != OK:
        msg = lib().pirmcut_last_error(None)
        raise PirmcutError(st, msg.decode() if msg else "")
    return x


def pirmcut_batch_info(h):
    a, b, m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    g, t, nt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    lib().pirmcut_batch_info(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(g), ctypes.byref(t),
                             ctypes.byref(nt), ctypes.byref(m))
    return dict(rows=a.value, nnz=b.value, threads_per_row=g.value, tile_rows=t.value, tiles=nt.value,
                medium_deg=m.value)


def pirmcut_batch_kernel_launches(h) -> int:
    return int(lib().pirmcut_batch_kernel_launches(h))


def pirmcut_batch_destroy(h):
    lib().pirmcut_batch_destroy(h)


class Batch:
    """Owner of one batch context."""

    def __init__(self, graphs, opt: Options | None = None, stream=None, **kw):
        if opt is None:
            opt = pirmcut_default_options(**kw)
        self.ns = [int(g.n) for g in graphs]
        self.h = pirmcut_batch_create(graphs, opt, stream)

    def solve(self, T, eps):
        return pirmcut_batch_solve(self.h, len(self.ns), T, eps)

    def cut(self, i):
        return pirmcut_batch_cut(self.h, i, self.ns[i])

    def get_x(self, i):
        return pirmcut_batch_get_x(self.h, i, self.ns[i])

    def info(self):
        return pirmcut_batch_info(self.h)

    def kernel_launches(self):
        return pirmcut_batch_kernel_launches(self.h)

    def close(self):
        if self.h:
            pirmcut_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Convenience owner of one context (same calls, object style)."""

    def __init__(self, graph, opt: Options | None = None, stream=None, **kw):
        if opt is None:
            opt = pirmcut_default_options(**kw)
        self.n = int(graph.n)
        self.fp32 = bool(opt.capacity_fp32)
        c = graph.c.astype(np.float32) if self.fp32 and isinstance(graph.c, np.ndarray) else graph.c
        self.h = pirmcut_create(graph.n, graph.row_ptr, graph.col, c, graph.s, graph.t,
                                opt, stream)

    def initial(self):
        return pirmcut_initial(self.h)

    def irls_step(self, eps):
        return pirmcut_irls_step(self.h, eps)

    def solve(self, T, eps):
        return pirmcut_solve(self.h, T, eps)

    def cut(self, side=None):
        return pirmcut_cut(self.h, side, n=self.n if side is None else None)

    def get_x(self, out=None):
        if out is None:
            out = np.empty(self.n, dtype=np.float64)
        return pirmcut_get_x(self.h, out)

    def cut_two_level(self, side=None):
        return pirmcut_cut_two_level(self.h, side, n=self.n if side is None else None)

    def set_x(self, x):
        pirmcut_set_x(self.h, x)

    def update_weights(self, c):
        if self.fp32 and isinstance(c, np.ndarray):
            c = c.astype(np.float32)
        pirmcut_update_weights(self.h, c, self.fp32)

    def problem_size(self):
        return pirmcut_problem_size(self.h)

    def time_spmv(self, reps=20):
        return pirmcut_time_spmv(self.h, reps)

    def spmv_timing(self, reset=True):
        return pirmcut_spmv_timing(self.h, reset)

    def kernel_launches(self):
        return pirmcut_kernel_launches(self.h)

    def mlp_enable(self, mode, seed=1):
        pirmcut_mlp_enable(self.h, mode, seed)

    def mlp_configure(self, iters_per_step=8, learning_rate=1e-3):
        pirmcut_mlp_configure(self.h, iters_per_step, learning_rate)

    def mlp_predict(self, features, delta=None):
        return pirmcut_mlp_predict(self.h, features, delta)

    def mlp_time_predict(self, features, delta, reps=20):
        return pirmcut_mlp_time_predict(self.h, features, delta, reps)

    def mlp_weights(self, w=None):
        return pirmcut_mlp_weights(self.h, w)

    def mlp_stats(self):
        return pirmcut_mlp_stats(self.h)

    def mlp_features(self):
        return pirmcut_mlp_features(self.h, self.n - 2)

    def close(self):
        if self.h:
            pirmcut_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
