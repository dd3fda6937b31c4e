"""CPU oracle for RAK label propagation and modularity (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_2301_09125_gb300`` never does: it shares no code, header or constant
with the C file compiled here (``rak_oracle.c``).

The functions are thin ctypes wrappers around the single-threaded C oracle,
which restates Sec. 3.2 of Sahu, arXiv 2301.09125 (RAK: strict / non-strict
tie rule, tolerance test), Sec. 3.3 (COPRA and the asynchronous update), Sec.
3.4 (SLPA) and Sec. 1 (Newman-Girvan modularity).  See the comment block at the top of
``rak_oracle.c`` for each reading of the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rak_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
             _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_mix64.restype = ctypes.c_uint64
        lib.oracle_mix64.argtypes = [ctypes.c_uint64]
        lib.oracle_tie_hash.restype = ctypes.c_uint64
        lib.oracle_tie_hash.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_int64]
        lib.oracle_choose_many.restype = ctypes.c_int
        lib.oracle_choose_many.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, _i32p,
                                           ctypes.c_int, ctypes.c_uint64, ctypes.c_int64,
                                           ctypes.c_int64, _i32p, _i32p]
        lib.oracle_rak.restype = ctypes.c_int
        lib.oracle_rak.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_double,
                                   ctypes.c_int32, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                   ctypes.c_int32, _i32p, ctypes.c_int32, _i32p, _i32p, _i32p,
                                   _i64p]
        lib.oracle_slpa_slot.restype = ctypes.c_int32
        lib.oracle_slpa_slot.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int64]
        lib.oracle_slpa.restype = ctypes.c_int
        lib.oracle_slpa.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_int32,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_uint64, _i32p, _i32p,
                                    ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int32), _i64p]
        lib.oracle_copra.restype = ctypes.c_int
        lib.oracle_copra.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_int32,
                                     ctypes.c_double, ctypes.c_int32, ctypes.c_int, ctypes.c_int32,
                                     ctypes.c_int, ctypes.c_uint64, _i32p,
                                     ctypes.POINTER(ctypes.c_uint32), _i32p,
                                     ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int32), _i64p]
        lib.oracle_split.restype = ctypes.c_int64
        lib.oracle_split.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, _i32p]
        lib.oracle_modularity.restype = ctypes.c_double
        lib.oracle_modularity.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, _i32p, _i64p,
                                          _i64p, _u64p]
        _lib = lib
    return _lib


def _arr(a, dtype=np.int32):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _ptr(a, ptype=_i32p):
    if a is None:
        return ctypes.cast(None, ptype)
    return a.ctypes.data_as(ptype)


def _check_csr(offsets, indices, weights):
    n = offsets.shape[0] - 1
    if n < 0 or offsets[0] != 0 or np.any(np.diff(offsets) < 0) or offsets[-1] != indices.shape[0]:
        raise ValueError("offsets are not a CSR row pointer")
    if indices.size and (indices.min() < 0 or indices.max() >= n):
        raise ValueError("indices out of range")
    if weights is not None and (weights.shape != indices.shape or np.any(weights <= 0)):
        raise ValueError("weights must be positive, one per entry")
    return n


def mix64(z: int) -> int:
    """SplitMix64 output function (Steele, Lea & Flood 2014)."""
    return int(_load().oracle_mix64(ctypes.c_uint64(z & (2**64 - 1))))


def tie_hash(seed: int, t: int, v: int, label: int) -> int:
    """Non-strict tie key of ``label`` at vertex ``v`` in global iteration ``t``."""
    return int(_load().oracle_tie_hash(ctypes.c_uint64(seed & (2**64 - 1)), t, v, label))


def rak(offsets, indices, weights=None, tolerance=0.05, max_iter=20, mode="sync",
        strict=True, seed=0, iter_offset=0, init_labels=None, waves=0):
    """Run RAK to convergence (Sec. 3.2).

    Returns ``(labels, iterations, converged, changed_per_iteration)``.
    ``mode`` is ``"sync"`` (double buffer) or ``"async"`` (in place, Sec. 3.3,
    in ``waves`` waves of vertices v mod W; 0 = every vertex its own wave,
    i.e. ascending vertex order).
    """
    offsets = _arr(offsets)
    indices = _arr(indices)
    weights = None if weights is None else _arr(weights)
    n = _check_csr(offsets, indices, weights)
    if mode not in ("sync", "async"):
        raise ValueError("mode must be 'sync' or 'async'")
    init = None if init_labels is None else _arr(init_labels)
    if init is not None and (init.shape != (n,) or (n and (init.min() < 0 or init.max() >= n))):
        raise ValueError("init_labels must be n vertex ids")
    labels = np.empty(n, dtype=np.int32)
    hist = np.zeros(max(int(max_iter), 1), dtype=np.int64)
    iters = ctypes.c_int32(0)
    conv = ctypes.c_int32(0)
    rc = _load().oracle_rak(n, _ptr(offsets), _ptr(indices), _ptr(weights), float(tolerance),
                            int(max_iter), 1 if mode == "async" else 0, 1 if strict else 0,
                            ctypes.c_uint64(seed & (2**64 - 1)), int(iter_offset), _ptr(init),
                            int(waves), _ptr(labels), ctypes.byref(iters), ctypes.byref(conv),
                            _ptr(hist, _i64p))
    if rc != 0:
        raise ValueError("oracle_rak rejected its arguments")
    return labels, int(iters.value), bool(conv.value), hist[: iters.value].copy()


def choose_many(offsets, indices, weights, cur, verts, strict=True, seed=0, t=0):
    """Label each vertex in ``verts`` adopts when reading labels ``cur`` in
    global iteration ``t`` (one RAK step, Sec. 3.2)."""
    offsets = _arr(offsets)
    indices = _arr(indices)
    weights = None if weights is None else _arr(weights)
    n = offsets.shape[0] - 1
    cur = _arr(cur)
    verts = _arr(verts)
    if cur.shape != (n,):
        raise ValueError("cur must hold n labels")
    if verts.size and (verts.min() < 0 or verts.max() >= n):
        raise ValueError("vertex out of range")
    out = np.empty(verts.shape[0], dtype=np.int32)
    rc = _load().oracle_choose_many(n, _ptr(offsets), _ptr(indices), _ptr(weights), _ptr(cur),
                                    1 if strict else 0, ctypes.c_uint64(seed & (2**64 - 1)),
                                    int(t), verts.shape[0], _ptr(verts), _ptr(out))
    if rc != 0:
        raise MemoryError("oracle_choose_many")
    return out


def slpa_slot(seed, t, v, pos):
    """The memory slot (0 .. t-1) a speaker speaks in iteration t to listener
    v through the entry at row position pos (Sec. 3.4's random speaker)."""
    return int(_load().oracle_slpa_slot(ctypes.c_uint64(seed & (2**64 - 1)), t, v, pos))


def slpa(offsets, indices, weights=None, memory_size=20, tolerance=0.05, strict=True, seed=0):
    """SLPA (Sec. 3.4): every vertex remembers itself, then in each iteration
    listens to one remembered label per neighbour and stores the heaviest.

    Returns ``(labels, memory, iterations, converged, changed_per_iteration)``
    with ``memory[t, v]`` the label v stored in iteration t (slot 0 = v).
    """
    offsets = _arr(offsets)
    indices = _arr(indices)
    weights = None if weights is None else _arr(weights)
    n = _check_csr(offsets, indices, weights)
    if memory_size < 1:
        raise ValueError("memory_size must be >= 1")
    memory = np.empty((memory_size, n), dtype=np.int32)
    labels = np.empty(n, dtype=np.int32)
    hist = np.zeros(max(memory_size - 1, 1), dtype=np.int64)
    iters = ctypes.c_int32(0)
    conv = ctypes.c_int32(0)
    rc = _load().oracle_slpa(n, _ptr(offsets), _ptr(indices), _ptr(weights), int(memory_size),
                             float(tolerance), 1 if strict else 0,
                             ctypes.c_uint64(seed & (2**64 - 1)), _ptr(memory), _ptr(labels),
                             ctypes.byref(iters), ctypes.byref(conv), _ptr(hist, _i64p))
    if rc != 0:
        raise ValueError("oracle_slpa rejected its arguments")
    it = int(iters.value)
    return labels, memory[: it + 1].copy(), it, bool(conv.value), hist[:it].copy()


COPRA_ONE = 65536  # belongings are integers in units of 2^-16 that sum to this


def copra(offsets, indices, weights=None, max_labels=4, tolerance=0.01, max_iter=20,
          mode="sync", waves=0, strict=True, seed=0):
    """COPRA (Sec. 3.3): every vertex keeps at most ``max_labels`` (label,
    belonging) pairs, belongings in units of 2^-16 summing to 2^16.

    Returns ``(labels, sets_l, sets_b, iterations, converged, changed)``:
    the best label of every vertex, the final sets as (n, max_labels) arrays
    (belonging 0 after a set's last pair), and the per-iteration counts of
    vertices whose best label changed.  ``waves`` as in :func:`rak`.
    """
    offsets = _arr(offsets)
    indices = _arr(indices)
    weights = None if weights is None else _arr(weights)
    n = _check_csr(offsets, indices, weights)
    if not 1 <= max_labels <= 64:
        raise ValueError("max_labels must lie in [1, 64]")
    L = int(max_labels)
    sets_l = np.empty((max(n, 1), L), dtype=np.int32)
    sets_b = np.empty((max(n, 1), L), dtype=np.uint32)
    labels = np.empty(max(n, 1), dtype=np.int32)
    hist = np.zeros(max_iter, dtype=np.int64)
    iters = ctypes.c_int32(0)
    conv = ctypes.c_int32(0)
    rc = _load().oracle_copra(n, _ptr(offsets), _ptr(indices), _ptr(weights), L,
                              float(tolerance), int(max_iter), 0 if mode == "sync" else 1,
                              int(waves), 1 if strict else 0, ctypes.c_uint64(seed & (2**64 - 1)),
                              _ptr(sets_l), sets_b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                              _ptr(labels), ctypes.byref(iters), ctypes.byref(conv),
                              _ptr(hist, _i64p))
    if rc != 0:
        raise ValueError("oracle_copra rejected its arguments")
    it = int(iters.value)
    return labels[:n].copy(), sets_l[:n].copy(), sets_b[:n].copy(), it, bool(conv.value), hist[:it].copy()


def split(offsets, indices, labels):
    """Split every community of ``labels`` into its connected components
    (only edges between two vertices of one community count); each component
    is labelled by its smallest vertex.  Returns ``(labels, components)``.
    The paper leaves this step out (end of Sec. 3.4)."""
    offsets = _arr(offsets)
    indices = _arr(indices)
    n = _check_csr(offsets, indices, None)
    labels = _arr(labels)
    if labels.shape != (n,):
        raise ValueError("labels must have one entry per vertex")
    out = np.empty(n, dtype=np.int32)
    k = _load().oracle_split(n, _ptr(offsets), _ptr(indices), _ptr(labels), _ptr(out))
    if k < 0:
        raise ValueError("oracle_split rejected its arguments")
    return out, int(k)


def modularity(offsets, indices, weights, labels, exact=False):
    """Newman-Girvan modularity of ``labels`` (Sec. 1).

    With ``exact=True`` also returns the exact integers ``(L, 2m, S)`` it is
    formed from (S = sum_c K_c^2 as a Python int).
    """
    offsets = _arr(offsets)
    indices = _arr(indices)
    weights = None if weights is None else _arr(weights)
    n = _check_csr(offsets, indices, weights)
    labels = _arr(labels)
    if labels.shape != (n,) or (n and (labels.min() < 0 or labels.max() >= n)):
        raise ValueError("labels must be n vertex ids")
    l_in = ctypes.c_int64(0)
    two_m = ctypes.c_int64(0)
    s = (ctypes.c_uint64 * 2)()
    q = _load().oracle_modularity(n, _ptr(offsets), _ptr(indices), _ptr(weights), _ptr(labels),
                                  ctypes.byref(l_in), ctypes.byref(two_m),
                                  ctypes.cast(s, _u64p))
    if exact:
        return float(q), int(l_in.value), int(two_m.value), (int(s[0]) << 64) | int(s[1])
    return float(q)
