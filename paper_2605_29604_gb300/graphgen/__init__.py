"""Seeded synthetic graph generators (inputs only).

Every function returns ``(n, row_ptr, col_idx)`` with ``row_ptr`` an int32
array of length n+1 and ``col_idx`` an int32 array of length row_ptr[n]: an
undirected, unweighted graph stored as symmetric CSR with sorted rows, no
duplicate arcs and no self-loops (the input class of the paper, Sec. 4.1.2).

The heavy families (Erdos-Renyi, R-MAT, grid with diagonals, random geometric,
relabelling) run in ``graphgen.c`` (compiled on first use with gcc); the
small closed-form families used by tests (complete, star, complete bipartite,
path, cycle, empty, disjoint union) are written here with numpy.  Nothing in
this module computes any part of the MIS method.

The synthetic families stand in for the paper's SuiteSparse graphs (Table 1),
which are not available offline: R-MAT for the skewed social/web graphs,
the grid with diagonals for the road / Delaunay meshes, Erdos-Renyi and
random geometric graphs for the uniform sparse cases.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

GOLDEN_RATIO_64 = 0x9E3779B97F4A7C15


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so beside it (gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
             "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        ptr32 = ctypes.POINTER(ctypes.c_int32)
        lib.gg_free.argtypes = [P]
        lib.gg_n.argtypes = [P]
        lib.gg_n.restype = i32
        lib.gg_arcs.argtypes = [P]
        lib.gg_arcs.restype = i64
        lib.gg_copy.argtypes = [P, ptr32, ptr32]
        lib.gg_from_edges.argtypes = [i32, i64, ptr32, ptr32]
        lib.gg_from_edges.restype = P
        lib.gg_er_gnm.argtypes = [i32, i64, u64]
        lib.gg_er_gnm.restype = P
        lib.gg_rmat.argtypes = [i32, i64, dbl, dbl, dbl, u64]
        lib.gg_rmat.restype = P
        lib.gg_grid_diag.argtypes = [i32, i64, u64]
        lib.gg_grid_diag.restype = P
        lib.gg_rgg.argtypes = [i32, dbl, u64]
        lib.gg_rgg.restype = P
        lib.gg_stencil27.argtypes = [i32, i32, i32]
        lib.gg_stencil27.restype = P
        lib.gg_permute.argtypes = [P, u64]
        lib.gg_permute.restype = P
        lib.gg_stream.argtypes = [u64, u64]
        lib.gg_stream.restype = u64
        _lib = lib
        return lib


def _take(h):
    lib = _load()
    if not h:
        raise MemoryError("graph generation failed (bad parameters or out of memory)")
    try:
        n = lib.gg_n(h)
        arcs = lib.gg_arcs(h)
        rp = np.empty(n + 1, dtype=np.int32)
        col = np.empty(max(arcs, 1), dtype=np.int32)
        lib.gg_copy(h, rp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                    col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        return n, rp, col[:arcs]
    finally:
        lib.gg_free(h)


def _as_handle(n, rp, col):
    """Temporary C graph built from an existing CSR (via its edge list)."""
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    src = np.repeat(np.arange(n, dtype=np.int32), np.diff(rp))
    keep = src < col
    u = np.ascontiguousarray(src[keep])
    v = np.ascontiguousarray(col[keep])
    lib = _load()
    p32 = ctypes.POINTER(ctypes.c_int32)
    return lib.gg_from_edges(n, len(u), u.ctypes.data_as(p32), v.ctypes.data_as(p32))


def stream(seed: int, index: int) -> int:
    """The index-th output of the splitmix64 stream started at `seed`."""
    return int(_load().gg_stream(seed & (2**64 - 1), index))


def from_edges(n: int, u, v):
    """Symmetric, deduplicated, loop-free CSR from an undirected edge list."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.int32))
    v = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
    if len(u) != len(v):
        raise ValueError("u and v differ in length")
    if len(u) and (u.min() < 0 or v.min() < 0 or u.max() >= n or v.max() >= n):
        raise ValueError("vertex id out of range")
    lib = _load()
    p32 = ctypes.POINTER(ctypes.c_int32)
    return _take(lib.gg_from_edges(n, len(u), u.ctypes.data_as(p32), v.ctypes.data_as(p32)))


def er_gnm(n: int, m: int, seed: int):
    """Erdos-Renyi G(n, m): exactly m distinct undirected edges, uniform."""
    return _take(_load().gg_er_gnm(n, m, seed & (2**64 - 1)))


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int,
         permute: bool = True):
    """R-MAT graph on 2**scale vertices from edge_factor * 2**scale generated
    edges (a, b, c, d=1-a-b-c), symmetrised, deduplicated, self-loops dropped,
    then (by default) uniformly relabelled."""
    lib = _load()
    h = lib.gg_rmat(scale, edge_factor << scale, a, b, c, seed & (2**64 - 1))
    if not permute:
        return _take(h)
    if not h:
        raise MemoryError("R-MAT generation failed")
    try:
        h2 = lib.gg_permute(h, stream(seed, 1))
    finally:
        lib.gg_free(h)
    return _take(h2)


def grid_diag(width: int, diag_frac: float, seed: int, permute: bool = False):
    """width x width 4-neighbour grid plus floor(diag_frac * grid_edges)
    distinct random diagonals; optionally uniformly relabelled."""
    grid_edges = 2 * width * (width - 1)
    ndiag = int(math.floor(diag_frac * grid_edges))
    lib = _load()
    h = lib.gg_grid_diag(width, ndiag, seed & (2**64 - 1))
    if not permute:
        return _take(h)
    if not h:
        raise MemoryError("grid generation failed")
    try:
        h2 = lib.gg_permute(h, stream(seed, 1))
    finally:
        lib.gg_free(h)
    return _take(h2)


def rgg(n: int, avg_degree: float, seed: int):
    """Random geometric graph in the unit square with radius
    sqrt(avg_degree / (pi n)); ids in cell-sorted order."""
    r = math.sqrt(avg_degree / (math.pi * max(n, 1)))
    return _take(_load().gg_rgg(n, r, seed & (2**64 - 1)))


def stencil27(nx: int, ny: int, nz: int):
    """nx x ny x nz lattice with the 27-point stencil (every vertex adjacent
    to the up to 26 others within one step in each axis), natural ids
    (z * ny + y) * nx + x."""
    return _take(_load().gg_stencil27(nx, ny, nz))


def permute(n: int, row_ptr, col_idx, seed: int):
    """Uniform random relabelling of an existing graph."""
    lib = _load()
    h = _as_handle(n, row_ptr, col_idx)
    if not h:
        raise MemoryError("permute failed")
    try:
        h2 = lib.gg_permute(h, seed & (2**64 - 1))
    finally:
        lib.gg_free(h)
    return _take(h2)


# ---------------------------------------------------------------- small families

def empty(n: int):
    return n, np.zeros(n + 1, dtype=np.int32), np.zeros(0, dtype=np.int32)


def complete(n: int):
    iu = np.triu_indices(n, 1)
    return from_edges(n, iu[0], iu[1])


def star(k: int):
    """K_{1,k}: centre 0, leaves 1..k."""
    return from_edges(k + 1, np.zeros(k, dtype=np.int32), np.arange(1, k + 1))


def complete_bipartite(a: int, b: int):
    """K_{a,b}: side A = 0..a-1, side B = a..a+b-1."""
    uu, vv = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return from_edges(a + b, uu.ravel(), vv.ravel())


def path(n: int):
    return from_edges(n, np.arange(n - 1), np.arange(1, n))


def cycle(n: int):
    return from_edges(n, np.arange(n), (np.arange(n) + 1) % n)


def disjoint_union(graphs):
    """Block-diagonal union of (n, row_ptr, col_idx) graphs, ids concatenated."""
    us, vs, off = [], [], 0
    for n, rp, col in graphs:
        src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
        keep = src < col
        us.append(src[keep] + off)
        vs.append(col[keep].astype(np.int64) + off)
        off += n
    u = np.concatenate(us) if us else np.zeros(0, np.int64)
    v = np.concatenate(vs) if vs else np.zeros(0, np.int64)
    return from_edges(off, u, v)


def random_small(n: int, p: float, seed: int):
    """G(n, p) for small test graphs (numpy Generator seeded with `seed`)."""
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    keep = rng.random(len(iu[0])) < p
    return from_edges(n, iu[0][keep], iu[1][keep])


# ---------------------------------------------------------------- workloads

def er_10k_deg8(seed: int = 1):
    """Plain single solve: G(n=10,000, m=40,000), average degree 8."""
    return er_gnm(10_000, 40_000, seed)


def rmat22(seed: int = 22, scale: int = 22):
    """R-MAT scale 22, edge factor 16, (0.57, 0.19, 0.19, 0.05), permuted."""
    return rmat(scale, 16, 0.57, 0.19, 0.19, seed, permute=True)


def grid2048(seed: int = 3, permute_ids: bool = False, width: int = 2048):
    """2048 x 2048 grid plus 5% random diagonals, natural or permuted ids."""
    return grid_diag(width, 0.05, seed, permute=permute_ids)


def stencil160():
    """160 x 160 x 160 lattice, 27-point stencil, natural ids: 4,096,000
    vertices, 26 neighbours inside the box."""
    return stencil27(160, 160, 160)


def batch_mixed(count: int, seed: int, nmin: int = 64, nmax: int = 65_536, threads: int = 0):
    """`count` graphs with n log-uniform in [nmin, nmax]: even index ER with
    average degree uniform in [6, 32], odd index random geometric with average
    degree 10.  Per-graph parameters come from the splitmix64 stream of `seed`.
    Generated in parallel threads (the C generator releases the GIL)."""
    specs = []
    for i in range(count):
        r0 = stream(seed, 3 * i) >> 11
        r1 = stream(seed, 3 * i + 1) >> 11
        s = stream(seed, 3 * i + 2)
        u0 = r0 * 2.0 ** -53
        n = int(round(math.exp(math.log(nmin) + u0 * (math.log(nmax) - math.log(nmin)))))
        n = min(max(n, nmin), nmax)
        if i % 2 == 0:
            d = 6.0 + 26.0 * (r1 * 2.0 ** -53)
            m = int(n * d / 2)
            m = min(m, n * (n - 1) // 2)
            specs.append(("er", n, m, s))
        else:
            specs.append(("rgg", n, 10.0, s))

    def one(spec):
        kind, n, p, s = spec
        return er_gnm(n, p, s) if kind == "er" else rgg(n, p, s)

    workers = threads or min(32, (os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(one, specs))
