"""ctypes binding of ``liblp.so`` (declared in ``include/lp.h``).

Argument marshalling only: every step of label propagation and modularity
runs in the library's CUDA kernels.  Arrays may be numpy arrays (host) or
torch tensors (host or CUDA); CUDA tensors are passed as device pointers
together with the current torch stream.  There is no fallback: if the library
is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblp.so")

LP_OK, LP_EINVAL, LP_ENOMEM, LP_ECUDA, LP_ETIMEOUT, LP_ENOTREADY = range(6)
LP_SYNC, LP_ASYNC = 0, 1
LP_FLAG_DEVICE_PTRS, LP_FLAG_CHECK_SYMMETRIC, LP_FLAG_BORROW = 1, 2, 4

_STATUS = {LP_EINVAL: "LP_EINVAL", LP_ENOMEM: "LP_ENOMEM", LP_ECUDA: "LP_ECUDA",
           LP_ETIMEOUT: "LP_ETIMEOUT", LP_ENOTREADY: "LP_ENOTREADY"}


class LPError(RuntimeError):
    """A library call returned a status other than LP_OK."""

    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class lp_rak_params(ctypes.Structure):
    _fields_ = [("tolerance", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("strict", ctypes.c_int32),
                ("iter_offset", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("init_labels", ctypes.c_void_p), ("init_labels_on_device", ctypes.c_int32),
                ("waves", ctypes.c_int32)]


class lp_rak_result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("last_changed", ctypes.c_int64), ("gpu_ms", ctypes.c_float)]

    def as_dict(self):
        return {"iterations": self.iterations, "converged": bool(self.converged),
                "last_changed": self.last_changed, "gpu_ms": self.gpu_ms}


class lp_graph_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int64), ("offsets", ctypes.c_void_p),
                ("indices", ctypes.c_void_p), ("weights", ctypes.c_void_p)]


class lp_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_int64), ("max_active", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("max_cohort", ctypes.c_int32),
                ("admitters", ctypes.c_int32), ("cohort_max_entries", ctypes.c_int64)]


class lp_serve_result(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_int64), ("status", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("modularity", ctypes.c_double),
                ("queued_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class lp_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("vertices", ctypes.c_double),
                ("entries", ctypes.c_double), ("bytes", ctypes.c_double)]


class lp_tune_result(ctypes.Structure):
    _fields_ = [("small_max", ctypes.c_int32), ("warp_max", ctypes.c_int32),
                ("cta_max", ctypes.c_int32), ("cta2_max", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("default_ms", ctypes.c_float),
                ("best_ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class lp_copra_params(ctypes.Structure):
    _fields_ = [("max_labels", ctypes.c_int32), ("tolerance", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("mode", ctypes.c_int32), ("waves", ctypes.c_int32),
                ("strict", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class lp_slpa_params(ctypes.Structure):
    _fields_ = [("memory_size", ctypes.c_int32), ("tolerance", ctypes.c_double),
                ("strict", ctypes.c_int32), ("seed", ctypes.c_uint64)]


_lib = None

# Every symbol include/lp.h declares, with its ctypes signature.
_P = ctypes.c_void_p
SIGNATURES = {
    "lp_rak_params_default": (ctypes.c_int, [ctypes.POINTER(lp_rak_params)]),
    "lp_graph_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _P, _P, _P,
                                       ctypes.c_uint32, _P, ctypes.POINTER(_P)]),
    "lp_graph_destroy": (ctypes.c_int, [_P]),
    "lp_graph_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int64)]),
    "lp_rak_run": (ctypes.c_int, [_P, ctypes.POINTER(lp_rak_params),
                                  ctypes.POINTER(lp_rak_result)]),
    "lp_rak_history": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int32)]),
    "lp_labels_get": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "lp_modularity": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "lp_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(lp_graph_desc),
                                       ctypes.c_uint32, _P, ctypes.POINTER(_P)]),
    "lp_batch_destroy": (ctypes.c_int, [_P]),
    "lp_batch_run": (ctypes.c_int, [_P, ctypes.POINTER(lp_rak_params),
                                    ctypes.POINTER(lp_rak_result)]),
    "lp_batch_autotune": (ctypes.c_int, [_P, ctypes.POINTER(lp_rak_params), ctypes.c_int32,
                                         ctypes.POINTER(lp_tune_result)]),
    "lp_graph_autotune": (ctypes.c_int, [_P, ctypes.POINTER(lp_rak_params), ctypes.c_int32,
                                         ctypes.POINTER(lp_tune_result)]),
    "lp_graph_set_buckets": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "lp_batch_set_buckets": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "lp_batch_labels_get": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    "lp_batch_modularity": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "lp_server_config_default": (ctypes.c_int, [ctypes.POINTER(lp_server_config)]),
    "lp_server_create": (ctypes.c_int, [ctypes.POINTER(lp_server_config),
                                        ctypes.POINTER(lp_rak_params), ctypes.POINTER(_P)]),
    "lp_server_submit": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64,
                                        _P, _P, _P, _P]),
    "lp_server_poll": (ctypes.c_int, [_P, ctypes.POINTER(lp_serve_result), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
    "lp_server_drain": (ctypes.c_int, [_P]),
    "lp_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64)]),
    "lp_server_destroy": (ctypes.c_int, [_P]),
    "lp_profile_enable": (ctypes.c_int, [ctypes.c_int32]),
    "lp_profile_reset": (ctypes.c_int, []),
    "lp_profile_read": (ctypes.c_int, [ctypes.POINTER(lp_kernel_stat), ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32)]),
    "lp_rak_sweep_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _P, _P, _P, _P, _P,
                                            ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_int64), _P]),
    "lp_copra_params_default": (ctypes.c_int, [ctypes.POINTER(lp_copra_params)]),
    "lp_copra_run": (ctypes.c_int, [_P, ctypes.POINTER(lp_copra_params),
                                    ctypes.POINTER(lp_rak_result)]),
    "lp_copra_sets_get": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32]),
    "lp_slpa_params_default": (ctypes.c_int, [ctypes.POINTER(lp_slpa_params)]),
    "lp_slpa_run": (ctypes.c_int, [_P, ctypes.POINTER(lp_slpa_params),
                                   ctypes.POINTER(lp_rak_result)]),
    "lp_slpa_memory_get": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32]),
    "lp_probe_gather": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _P, _P, _P,
                                       ctypes.c_int32, ctypes.c_int32, _P,
                                       ctypes.POINTER(ctypes.c_float), _P]),
    "lp_split_communities": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "lp_selftest_barrier_timeout": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32)]),
    "lp_last_error": (ctypes.c_char_p, []),
    "lp_launch_count": (ctypes.c_int64, []),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load ``liblp.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(
                f"{path} is missing: build it with paper_2301_09125_gb300.build.build() "
                "(nvcc, sm_103a); there is no CPU fallback")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int):
    if status != LP_OK:
        raise LPError(status, load().lp_last_error().decode(errors="replace"))


# ---------------------------------------------------------------- marshalling
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _int32_buffer(x, name):
    """(pointer, on_device, keepalive) of an int32 array-like."""
    if x is None:
        return None, False, None
    if _is_torch(x):
        import torch
        if x.dtype != torch.int32:
            raise TypeError(f"{name} must be int32")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return x.data_ptr(), bool(x.is_cuda), x
    a = np.ascontiguousarray(x, dtype=np.int32)
    return a.ctypes.data, False, a


def _stream_of(*tensors):
    for t in tensors:
        if t is not None and _is_torch(t) and t.is_cuda:
            import torch
            return torch.cuda.current_stream(t.device).cuda_stream
    return None


def lp_rak_params_default() -> lp_rak_params:
    p = lp_rak_params()
    _check(load().lp_rak_params_default(ctypes.byref(p)))
    return p


def make_params(tolerance=0.05, max_iter=20, mode="sync", strict=True, seed=0, iter_offset=0,
                init_labels=None, waves=None) -> tuple:
    """(lp_rak_params, keepalive) from Python values."""
    p = lp_rak_params_default()
    p.tolerance = float(tolerance)
    p.max_iter = int(max_iter)
    p.mode = {"sync": LP_SYNC, "async": LP_ASYNC}[mode] if isinstance(mode, str) else int(mode)
    p.strict = 1 if strict else 0
    p.seed = int(seed) & (2**64 - 1)
    p.iter_offset = int(iter_offset)
    if waves is not None:
        p.waves = int(waves)
    ptr, on_dev, keep = _int32_buffer(init_labels, "init_labels")
    p.init_labels = ptr
    p.init_labels_on_device = 1 if on_dev else 0
    return p, keep


# ---------------------------------------------------------------- graphs
def lp_graph_create(offsets, indices, weights=None, check_symmetric=False, borrow=False,
                    stream=None) -> int:
    """Create a graph from a CSR; returns the opaque handle.

    All three arrays must live on the same side (host numpy/torch-CPU, or CUDA
    tensors).  ``borrow=True`` (CUDA tensors only) keeps references to the
    caller's memory instead of copying; the caller must keep the tensors alive
    and unchanged until ``lp_graph_destroy``.
    """
    po, do, ko = _int32_buffer(offsets, "offsets")
    pi, di, ki = _int32_buffer(indices, "indices")
    pw, dw, kw = _int32_buffer(weights, "weights")
    sides = {do, di} | ({dw} if weights is not None else set())
    if len(sides) != 1:
        raise ValueError("offsets, indices and weights must all be host or all be device arrays")
    on_dev = do
    n = (ko.shape[0] if hasattr(ko, "shape") else len(ko)) - 1
    m = ki.shape[0] if hasattr(ki, "shape") else len(ki)
    flags = (LP_FLAG_DEVICE_PTRS if on_dev else 0) | (LP_FLAG_CHECK_SYMMETRIC if check_symmetric else 0)
    if borrow:
        if not on_dev:
            raise ValueError("borrow needs CUDA tensors")
        flags |= LP_FLAG_BORROW
    if stream is None:
        stream = _stream_of(offsets, indices, weights)
    h = ctypes.c_void_p()
    _check(load().lp_graph_create(int(n), int(m), po, pi, pw, flags, stream, ctypes.byref(h)))
    return h.value


def lp_graph_destroy(handle: Optional[int]) -> None:
    if handle:
        _check(load().lp_graph_destroy(handle))


def lp_graph_info(handle: int):
    n = ctypes.c_int32()
    m = ctypes.c_int64()
    _check(load().lp_graph_info(handle, ctypes.byref(n), ctypes.byref(m)))
    return n.value, m.value


def lp_rak_run(handle: int, params: Optional[lp_rak_params] = None, **kw) -> lp_rak_result:
    """Run RAK on a graph.  Pass an ``lp_rak_params`` or keyword arguments of
    ``make_params``."""
    keep = None
    if params is None:
        params, keep = make_params(**kw)
    r = lp_rak_result()
    _check(load().lp_rak_run(handle, ctypes.byref(params), ctypes.byref(r)))
    del keep
    return r


def lp_rak_history(handle: int) -> np.ndarray:
    cnt = ctypes.c_int32()
    _check(load().lp_rak_history(handle, None, 0, ctypes.byref(cnt)))
    out = np.zeros(cnt.value, dtype=np.int64)
    _check(load().lp_rak_history(handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 cnt.value, ctypes.byref(cnt)))
    return out


def lp_labels_get(handle: int, out=None):
    """Current labels: into ``out`` (numpy or torch, host or CUDA) or a new
    numpy array."""
    n, _ = lp_graph_info(handle)
    if out is None:
        out = np.empty(n, dtype=np.int32)
    ptr, on_dev, keep = _int32_buffer(out, "out")
    if keep is not out:
        raise ValueError("out must be a contiguous int32 array")
    _check(load().lp_labels_get(handle, ptr, 1 if on_dev else 0))
    return out


def lp_modularity(handle: int, labels=None) -> float:
    """Modularity of ``labels`` (or of the graph's current labels)."""
    ptr, on_dev, keep = _int32_buffer(labels, "labels")
    q = ctypes.c_double()
    _check(load().lp_modularity(handle, ptr, 1 if on_dev else 0, ctypes.byref(q)))
    del keep
    return q.value


# ---------------------------------------------------------------- batches
def lp_batch_create(graphs: Sequence, check_symmetric=False, stream=None) -> int:
    """Create a batch from host CSR triples ``(offsets, indices, weights|None)``."""
    descs = (lp_graph_desc * len(graphs))()
    keep = []
    for i, g in enumerate(graphs):
        off, idx, w = g[0], g[1], (g[2] if len(g) > 2 else None)
        off = np.ascontiguousarray(off, dtype=np.int32)
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        w = None if w is None else np.ascontiguousarray(w, dtype=np.int32)
        keep += [off, idx, w]
        descs[i].n = off.shape[0] - 1
        descs[i].m = idx.shape[0]
        descs[i].offsets = off.ctypes.data
        descs[i].indices = idx.ctypes.data
        descs[i].weights = None if w is None else w.ctypes.data
    h = ctypes.c_void_p()
    _check(load().lp_batch_create(len(graphs), descs,
                                  LP_FLAG_CHECK_SYMMETRIC if check_symmetric else 0, stream,
                                  ctypes.byref(h)))
    return h.value


def lp_batch_destroy(handle: Optional[int]) -> None:
    if handle:
        _check(load().lp_batch_destroy(handle))


def lp_batch_autotune(handle: int, params: Optional[lp_rak_params] = None, sweeps: int = 5,
                      **kw) -> lp_tune_result:
    """Pick the batch's bucket bounds by timing `sweeps` iterations of each
    candidate (keyword arguments as for make_params)."""
    if params is None:
        params, _ = make_params(**kw)
    out = lp_tune_result()
    _check(load().lp_batch_autotune(handle, ctypes.byref(params), int(sweeps), ctypes.byref(out)))
    return out


def lp_graph_autotune(handle: int, params: Optional[lp_rak_params] = None, sweeps: int = 5,
                      **kw) -> lp_tune_result:
    """Pick a graph's bucket bounds by timing `sweeps` iterations of each
    candidate (keyword arguments as for make_params)."""
    if params is None:
        params, _ = make_params(**kw)
    out = lp_tune_result()
    _check(load().lp_graph_autotune(handle, ctypes.byref(params), int(sweeps), ctypes.byref(out)))
    return out


def lp_graph_set_buckets(handle: int, max_degree) -> None:
    """Set the largest degree of the small / warp / cta / cta2 buckets."""
    arr = (ctypes.c_int32 * 4)(*[int(x) for x in max_degree])
    _check(load().lp_graph_set_buckets(handle, arr))


def lp_batch_set_buckets(handle: int, max_degree) -> None:
    """Set the largest degree of the small / warp / cta / cta2 buckets."""
    arr = (ctypes.c_int32 * 4)(*[int(x) for x in max_degree])
    _check(load().lp_batch_set_buckets(handle, arr))


def lp_batch_run(handle: int, count: int, params: Optional[lp_rak_params] = None, **kw):
    """Run every graph of a batch; returns the per-graph results."""
    if params is None:
        params, _ = make_params(**kw)
    res = (lp_rak_result * count)()
    _check(load().lp_batch_run(handle, ctypes.byref(params), res))
    return list(res)


def lp_batch_labels_get(handle: int, index: int, n: int, out=None):
    if out is None:
        out = np.empty(n, dtype=np.int32)
    ptr, on_dev, keep = _int32_buffer(out, "out")
    _check(load().lp_batch_labels_get(handle, index, ptr, 1 if on_dev else 0))
    return out


def lp_batch_modularity(handle: int, index: int) -> float:
    q = ctypes.c_double()
    _check(load().lp_batch_modularity(handle, index, ctypes.byref(q)))
    return q.value


# ---------------------------------------------------------------- serving
def lp_server_config_default() -> lp_server_config:
    c = lp_server_config()
    _check(load().lp_server_config_default(ctypes.byref(c)))
    return c


def lp_server_create(config: Optional[lp_server_config] = None,
                     params: Optional[lp_rak_params] = None, **kw) -> int:
    """Start a request server; ``kw`` are ``make_params`` arguments."""
    if config is None:
        config = lp_server_config_default()
    if params is None:
        params, _ = make_params(**kw)
    h = ctypes.c_void_p()
    _check(load().lp_server_create(ctypes.byref(config), ctypes.byref(params), ctypes.byref(h)))
    return h.value


def lp_server_submit(handle: int, request_id: int, offsets, indices, weights=None,
                     labels_out=None) -> None:
    """Queue a request (host arrays, kept alive by the caller until its
    result has been polled)."""
    po, _, ko = _int32_buffer(offsets, "offsets")
    pi, _, ki = _int32_buffer(indices, "indices")
    pw, _, _ = _int32_buffer(weights, "weights")
    pl, _, _ = _int32_buffer(labels_out, "labels_out")
    n = (ko.shape[0] if hasattr(ko, "shape") else len(ko)) - 1
    m = ki.shape[0] if hasattr(ki, "shape") else len(ki)
    _check(load().lp_server_submit(handle, int(request_id), int(n), int(m), po, pi, pw, pl))


def lp_server_poll(handle: int, capacity: int = 256, wait_ms: int = 0) -> list:
    out = (lp_serve_result * capacity)()
    cnt = ctypes.c_int32()
    st = load().lp_server_poll(handle, out, capacity, ctypes.byref(cnt), int(wait_ms))
    if st not in (LP_OK, LP_ENOTREADY):
        _check(st)
    return [out[i] for i in range(cnt.value)]


def lp_server_stats(handle: int) -> dict:
    """Cohorts formed so far, requests that ran in a cohort of two or more,
    and the largest cohort."""
    c, b, m = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().lp_server_stats(handle, ctypes.byref(c), ctypes.byref(b), ctypes.byref(m)))
    return {"cohorts": c.value, "batched_requests": b.value, "largest_cohort": m.value}


def lp_server_drain(handle: int) -> None:
    _check(load().lp_server_drain(handle))


def lp_server_destroy(handle: Optional[int]) -> None:
    if handle:
        _check(load().lp_server_destroy(handle))


def lp_profile_enable(on: bool = True) -> None:
    _check(load().lp_profile_enable(1 if on else 0))


def lp_profile_reset() -> None:
    _check(load().lp_profile_reset())


def lp_profile_read() -> dict:
    """Per-kernel sweep statistics: name -> dict(launches, total_ms, vertices,
    entries, bytes)."""
    stats = (lp_kernel_stat * 8)()
    cnt = ctypes.c_int32()
    _check(load().lp_profile_read(stats, 8, ctypes.byref(cnt)))
    return {st.name.decode(): {"launches": st.launches, "total_ms": st.total_ms,
                               "vertices": st.vertices, "entries": st.entries, "bytes": st.bytes}
            for st in stats[:cnt.value]}


def lp_rak_sweep_noalloc(offsets, indices, weights, labels_in, labels_out, strict=True, seed=0,
                         iteration=0, stream=None) -> int:
    """One synchronous sweep without any device allocation (CUDA tensors
    only); returns the number of vertices that changed label."""
    arrays = [_int32_buffer(x, nm) for x, nm in ((offsets, "offsets"), (indices, "indices"),
                                                 (weights, "weights"), (labels_in, "labels_in"),
                                                 (labels_out, "labels_out"))]
    if not all(on_dev for (ptr, on_dev, _), x in zip(arrays, (offsets, indices, weights, labels_in,
                                                              labels_out)) if x is not None):
        raise ValueError("lp_rak_sweep_noalloc takes device arrays")
    n = offsets.shape[0] - 1
    m = indices.shape[0]
    if stream is None:
        stream = _stream_of(offsets)
    changed = ctypes.c_int64()
    _check(load().lp_rak_sweep_noalloc(int(n), int(m), arrays[0][0], arrays[1][0], arrays[2][0],
                                       arrays[3][0], arrays[4][0], 1 if strict else 0,
                                       int(seed) & (2**64 - 1), int(iteration),
                                       ctypes.byref(changed), stream))
    return changed.value


def lp_last_error() -> str:
    return load().lp_last_error().decode(errors="replace")


def lp_copra_run(handle: int, max_labels=4, tolerance=0.01, max_iter=20, mode="async", waves=31,
                 strict=True, seed=0) -> lp_rak_result:
    """Run COPRA (Sec. 3.3) on a graph; its labels become the best labels."""
    p = lp_copra_params()
    _check(load().lp_copra_params_default(ctypes.byref(p)))
    p.max_labels = int(max_labels)
    p.tolerance = float(tolerance)
    p.max_iter = int(max_iter)
    p.mode = {"sync": LP_SYNC, "async": LP_ASYNC}[mode] if isinstance(mode, str) else int(mode)
    p.waves = int(waves)
    p.strict = 1 if strict else 0
    p.seed = int(seed) & (2**64 - 1)
    r = lp_rak_result()
    _check(load().lp_copra_run(handle, ctypes.byref(p), ctypes.byref(r)))
    return r


def lp_copra_sets_get(handle: int, max_labels: int):
    """(labels, belongings) of the last COPRA run as (n, max_labels) arrays."""
    n, _ = lp_graph_info(handle)
    lab = np.empty((n, max_labels), dtype=np.int32)
    bel = np.empty((n, max_labels), dtype=np.uint32)
    _check(load().lp_copra_sets_get(handle, lab.ctypes.data, bel.ctypes.data, 0))
    return lab, bel


def lp_slpa_run(handle: int, memory_size=20, tolerance=0.05, strict=True, seed=0) -> lp_rak_result:
    """Run SLPA (Sec. 3.4) on a graph; its labels become the communities."""
    p = lp_slpa_params()
    _check(load().lp_slpa_params_default(ctypes.byref(p)))
    p.memory_size = int(memory_size)
    p.tolerance = float(tolerance)
    p.strict = 1 if strict else 0
    p.seed = int(seed) & (2**64 - 1)
    r = lp_rak_result()
    _check(load().lp_slpa_run(handle, ctypes.byref(p), ctypes.byref(r)))
    return r


def lp_slpa_memory_get(handle: int, slots: int, out=None):
    """Memory slots 0 .. slots-1 of the last SLPA run as a (slots, n) array
    (numpy, or into a contiguous int32 ``out``, host or CUDA)."""
    n, _ = lp_graph_info(handle)
    if out is None:
        out = np.empty((slots, n), dtype=np.int32)
    ptr, on_dev, keep = _int32_buffer(out, "out")
    _check(load().lp_slpa_memory_get(handle, ptr, int(slots), 1 if on_dev else 0))
    del keep
    return out


def lp_probe_gather(n, indices, weights, labels, mode=1, repeats=20, stream=None) -> float:
    """Milliseconds per pass streaming indices and weights (mode 0), or also
    gathering labels[index] per entry (mode 1); CUDA tensors."""
    import torch

    sink = torch.zeros(2, dtype=torch.int32, device=indices.device)
    ms = ctypes.c_float()
    if stream is None:
        stream = _stream_of(indices)
    _check(load().lp_probe_gather(int(n), int(indices.shape[0]), indices.data_ptr(),
                                  None if weights is None else weights.data_ptr(),
                                  labels.data_ptr(), int(mode), int(repeats), sink.data_ptr(),
                                  ctypes.byref(ms), stream))
    return float(ms.value)


def lp_split_communities(handle: int) -> int:
    """Split the graph's communities into connected components in place (each
    named by its smallest vertex); returns the number of components."""
    k = ctypes.c_int64()
    _check(load().lp_split_communities(handle, ctypes.byref(k)))
    return k.value


def lp_selftest_barrier_timeout() -> bool:
    """True when a grid barrier that can never complete gave up after its
    poll limit and reported the timeout (the context stays usable)."""
    out = ctypes.c_int32()
    _check(load().lp_selftest_barrier_timeout(ctypes.byref(out)))
    return out.value == 1


def lp_launch_count() -> int:
    return int(load().lp_launch_count())


# ---------------------------------------------------------------- convenience
class Graph:
    """Owning wrapper of an ``lp_graph`` handle (destroyed on close / GC)."""

    def __init__(self, offsets, indices, weights=None, **kw):
        self._keep = (offsets, indices, weights) if kw.get("borrow") else None
        self.handle = lp_graph_create(offsets, indices, weights, **kw)
        self.n, self.m = lp_graph_info(self.handle)

    def rak(self, **kw) -> lp_rak_result:
        return lp_rak_run(self.handle, **kw)

    def split(self) -> int:
        return lp_split_communities(self.handle)

    def copra(self, **kw) -> lp_rak_result:
        self._copra_labels = kw.get("max_labels", 4)
        return lp_copra_run(self.handle, **kw)

    def copra_sets(self):
        return lp_copra_sets_get(self.handle, getattr(self, "_copra_labels", 4))

    def slpa(self, **kw) -> lp_rak_result:
        return lp_slpa_run(self.handle, **kw)

    def slpa_memory(self, slots: int, out=None):
        return lp_slpa_memory_get(self.handle, slots, out)

    def autotune(self, sweeps: int = 5, **kw) -> lp_tune_result:
        return lp_graph_autotune(self.handle, sweeps=sweeps, **kw)

    def set_buckets(self, max_degree) -> None:
        lp_graph_set_buckets(self.handle, max_degree)

    def labels(self, out=None):
        return lp_labels_get(self.handle, out)

    def history(self) -> np.ndarray:
        return lp_rak_history(self.handle)

    def modularity(self, labels=None) -> float:
        return lp_modularity(self.handle, labels)

    def close(self):
        if getattr(self, "handle", None):
            lp_graph_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
