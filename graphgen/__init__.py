"""Seeded synthetic graph inputs (shared by the tests, the benchmark and the
oracle checks; holds no label-propagation or modularity arithmetic).

The C generators in ``graphgen.c`` are built with gcc (+OpenMP) into
``graphgen/libgraphgen.so``.  Every graph is a symmetric int32 CSR
(``offsets[n+1]``, ``indices[m]``, ``weights[m]`` or ``None`` for unit
weights), rows sorted, no self-loops, no duplicate entries.

``workload(name)`` builds the named benchmark inputs, which stand in for the
SuiteSparse graphs of the paper's Table 1 (not available offline):

* ``sbm10k``   planted partition, 10,000 vertices, 20 blocks, p_in 0.02,
               p_out 0.0005, unit weights (collaboration-like)
* ``rmat22``   R-MAT scale 22, edge factor 16, a/b/c = .57/.19/.19, integer
               weights 1-4, random vertex permutation (web/social-like)
* ``road4096`` 4096 x 4096 grid, 15% of edges deleted, 1% shortcuts within
               radius 8, integer weights 1-16 (road-like)
* ``kmer8m``   8M vertices on random paths plus 5% branch edges (k-mer-like)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import NamedTuple, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None


class CSR(NamedTuple):
    offsets: np.ndarray
    indices: np.ndarray
    weights: Optional[np.ndarray]

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.indices.shape[0])


def build(force: bool = False) -> str:
    """Compile ``graphgen.c`` into ``graphgen/libgraphgen.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp = ctypes.c_void_p
        lib.gg_sbm_planted.restype = vp
        lib.gg_sbm_planted.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64, ctypes.c_int32,
                                       ctypes.c_int32]
        lib.gg_sbm_mixing.restype = vp
        lib.gg_sbm_mixing.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_uint64, ctypes.c_int32,
                                      ctypes.c_int32]
        lib.gg_rmat.restype = vp
        lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                ctypes.c_int32, ctypes.c_int32, ctypes.c_int]
        lib.gg_grid_road.restype = vp
        lib.gg_grid_road.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32,
                                     ctypes.c_int32]
        lib.gg_kmer_like.restype = vp
        lib.gg_kmer_like.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                     ctypes.c_uint64]
        lib.gg_n.restype = ctypes.c_int32
        lib.gg_n.argtypes = [vp]
        lib.gg_m.restype = ctypes.c_int64
        lib.gg_m.argtypes = [vp]
        lib.gg_has_weights.restype = ctypes.c_int
        lib.gg_has_weights.argtypes = [vp]
        lib.gg_copy_out.restype = None
        lib.gg_copy_out.argtypes = [vp, vp, vp, vp]
        lib.gg_free.restype = None
        lib.gg_free.argtypes = [vp]
        lib.gg_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _take(h) -> CSR:
    lib = _load()
    if not h:
        raise ValueError("graph generator rejected its parameters (or ran out of memory)")
    try:
        n, m = lib.gg_n(h), lib.gg_m(h)
        off = np.empty(n + 1, dtype=np.int32)
        idx = np.empty(m, dtype=np.int32)
        w = np.empty(m, dtype=np.int32) if lib.gg_has_weights(h) else None
        lib.gg_copy_out(h, off.ctypes.data, idx.ctypes.data, None if w is None else w.ctypes.data)
    finally:
        lib.gg_free(h)
    return CSR(off, idx, w)


def _u64(seed: int) -> ctypes.c_uint64:
    return ctypes.c_uint64(int(seed) & (2**64 - 1))


def sbm_planted(n, k, p_in, p_out, seed=1, wmin=1, wmax=1) -> CSR:
    """Planted-partition SBM: k equal blocks, edge probability p_in inside a
    block and p_out between blocks."""
    return _take(_load().gg_sbm_planted(n, k, p_in, p_out, _u64(seed), wmin, wmax))


def sbm_mixing(n, k, avg_degree, mu, seed=1, wmin=1, wmax=1) -> CSR:
    """Planted partition with expected degree ``avg_degree`` and a fraction
    ``mu`` of each vertex's edges leaving its block."""
    return _take(_load().gg_sbm_mixing(n, k, avg_degree, mu, _u64(seed), wmin, wmax))


def rmat(scale, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1, wmin=1, wmax=4,
         permute=True) -> CSR:
    """R-MAT graph, symmetrised, self-loops and duplicates removed."""
    return _take(_load().gg_rmat(scale, edge_factor, a, b, c, _u64(seed), wmin, wmax,
                                 1 if permute else 0))


def grid_road(side, delete_frac=0.15, shortcut_frac=0.01, radius=8, seed=1, wmin=1,
              wmax=16) -> CSR:
    """Road-like 2-D grid with deleted edges and short-range shortcuts."""
    return _take(_load().gg_grid_road(side, delete_frac, shortcut_frac, radius, _u64(seed),
                                      wmin, wmax))


def kmer_like(n, mean_path=1000, branch_frac=0.05, seed=1) -> CSR:
    """Random paths plus a few short branch edges (de-Bruijn-like), unit weights."""
    return _take(_load().gg_kmer_like(n, mean_path, branch_frac, _u64(seed)))


def num_threads() -> int:
    return int(_load().gg_num_threads())


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

WORKLOADS = {
    "sbm10k": dict(kind="sbm_planted", n=10_000, k=20, p_in=0.02, p_out=0.0005, seed=1),
    "rmat22": dict(kind="rmat", scale=22, edge_factor=16, seed=1, wmin=1, wmax=4),
    "rmat21": dict(kind="rmat", scale=21, edge_factor=16, seed=1, wmin=1, wmax=4),
    "road4096": dict(kind="grid_road", side=4096, seed=1, wmin=1, wmax=16),
    "kmer8m": dict(kind="kmer_like", n=8 * 1024 * 1024, seed=1),
}


def workload(name: str, **override) -> CSR:
    """Build one named benchmark input (see the module docstring)."""
    spec = dict(WORKLOADS[name])
    spec.update(override)
    kind = spec.pop("kind")
    return globals()[kind](**spec)


def with_self_loops(g: CSR, weight: int = 1) -> CSR:
    """The graph with a self-loop of the given weight added to every vertex
    (Sec. 3.1 adds one to every vertex of its inputs), stored last in its row.
    Weights become explicit when they were unit."""
    n, m = g.n, g.m
    deg = np.diff(g.offsets.astype(np.int64))
    off = (g.offsets.astype(np.int64) + np.arange(n + 1)).astype(np.int32)
    loop_at = off[1:].astype(np.int64) - 1
    keep = np.ones(m + n, dtype=bool)
    keep[loop_at] = False
    idx = np.empty(m + n, dtype=np.int32)
    idx[keep] = g.indices
    idx[loop_at] = np.arange(n, dtype=np.int32)
    w = np.empty(m + n, dtype=np.int32)
    w[keep] = 1 if g.weights is None else g.weights
    w[loop_at] = weight
    assert int(deg.sum()) == m
    return CSR(off, idx, w)


def batch_sbm_params(count=4096, seed=1000, n_lo=1_000, n_hi=200_000, k_lo=5, k_hi=500,
                     d_lo=8.0, d_hi=32.0, mu=0.3):
    """Parameters of the batched-SBM workload: per graph i, n log-uniform in
    [n_lo, n_hi], k log-uniform in [k_lo, k_hi] clamped to n/(2d), d uniform in
    [d_lo, d_hi], mixing mu, seed ``seed + i``.  Returns a list of dicts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        k = int(round(math.exp(rng.uniform(math.log(k_lo), math.log(k_hi)))))
        d = float(rng.uniform(d_lo, d_hi))
        k = max(1, min(k, int(n / (2 * d))))
        out.append(dict(n=n, k=k, avg_degree=d, mu=mu, seed=seed + i))
    return out


def batch_sbm(params) -> list:
    """Generate every graph of ``batch_sbm_params`` (unit weights)."""
    return [sbm_mixing(p["n"], p["k"], p["avg_degree"], p["mu"], seed=p["seed"]) for p in params]
