"""ctypes binding of libtcmis.so (the C ABI declared in include/tcmis.h).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  The functions keep the C names (``mis_create``, ``mis_solve``, ...);
the ``Graph`` class wraps a handle for convenience.  If the compiled library
is missing this module raises instead of falling back to anything else.

Device buffers and streams for the ``*_ex`` entry points come from PyTorch
(``tensor.data_ptr()``, ``torch.cuda.current_stream().cuda_stream``); host
buffers are numpy arrays.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtcmis.so")

MIS_OK = 0
MIS_EINVAL = -1
MIS_ENOMEM = -2
MIS_EBUSY = -3
MIS_ETIMEDOUT = -4
MIS_EDEVICE = -5
MIS_EINTERNAL = -6
MIS_ENOTREADY = -7

MIS_PATH_AUTO = 0
MIS_PATH_CSR = 1
MIS_PATH_TILE = 2
MIS_PATH_TILE_TC = 3
MIS_PATH_PUSH = 4
MIS_PATH_CLUSTER = 5
MIS_PATH_ROWS_TC = 6  # reported by mis_get_stats for the tensor-core multi-seed form
MIS_MULTI_ROWS = 0
MIS_MULTI_ROWS_TC = 1
MIS_PRIORITY_EQ1 = 0
MIS_PRIORITY_HASH = 1
MIS_PRIORITY_EQ1_Q8 = 2

ERROR_NAMES = {0: "MIS_OK", -1: "MIS_EINVAL", -2: "MIS_ENOMEM", -3: "MIS_EBUSY",
               -4: "MIS_ETIMEDOUT", -5: "MIS_EDEVICE", -6: "MIS_EINTERNAL", -7: "MIS_ENOTREADY"}


class MisError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class mis_options(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("threads_per_row", ctypes.c_int32),
                ("check_symmetry", ctypes.c_int32), ("build_tiles", ctypes.c_int32),
                ("spin_cap", ctypes.c_int64), ("device", ctypes.c_int32),
                ("max_slots", ctypes.c_int32), ("hbm_budget", ctypes.c_int64),
                ("serve_blocks", ctypes.c_int32), ("order_rows", ctypes.c_int32),
                ("priority", ctypes.c_int32)]


class mis_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("path", ctypes.c_int32),
                ("threads_per_row", ctypes.c_int32), ("status", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("csr_pending", ctypes.c_int32), ("ntiles", ctypes.c_int64),
                ("alive_sum", ctypes.c_int64), ("mis_size", ctypes.c_int64),
                ("alive_per_round", ctypes.c_int64 * 64), ("init_ns", ctypes.c_int64),
                ("select_ns", ctypes.c_int64 * 64), ("exclude_ns", ctypes.c_int64 * 64),
                ("sure_in", ctypes.c_int64), ("sure_out", ctypes.c_int64),
                ("tested_arcs", ctypes.c_int64), ("keyed", ctypes.c_int64),
                ("tested_rows", ctypes.c_int64), ("tested_prefix_arcs", ctypes.c_int64),
                ("tile_payload", ctypes.c_int32)]


class mis_tuning(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("param", ctypes.c_int32),
                ("bounds", ctypes.c_int32 * 4), ("grid", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("ms", ctypes.c_float),
                ("csr_pending", ctypes.c_int32),
                ("arcs_per_tile", ctypes.c_double), ("csr_range0", ctypes.c_int32),
                ("tile_payload", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libtcmis.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2605_29604_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        L.mis_options_init.argtypes = [ctypes.POINTER(mis_options)]
        L.mis_options_init.restype = None
        L.mis_create.argtypes = [i32, P, P]
        L.mis_create.restype = P
        L.mis_create_ex.argtypes = [i32, P, P, i32, ctypes.POINTER(mis_options), P]
        L.mis_create_ex.restype = P
        L.mis_create_batch.argtypes = [i32, P, P, P, ctypes.POINTER(mis_options)]
        L.mis_create_batch.restype = P
        L.mis_graph_count.argtypes = [P]
        L.mis_graph_count.restype = i32
        L.mis_result_size.argtypes = [P]
        L.mis_result_size.restype = i64
        L.mis_footprint.argtypes = [P]
        L.mis_footprint.restype = i64
        L.mis_solve.argtypes = [P, u64, P]
        L.mis_solve.restype = ctypes.c_int
        L.mis_solve_ex.argtypes = [P, P, P, P]
        L.mis_solve_ex.restype = ctypes.c_int
        L.mis_get_stats.argtypes = [P, ctypes.POINTER(mis_stats)]
        L.mis_get_stats.restype = ctypes.c_int
        L.mis_keys_ex.argtypes = [P, P, P, P]
        L.mis_keys_ex.restype = ctypes.c_int
        L.mis_set_path.argtypes = [P, i32, i32]
        L.mis_set_path.restype = ctypes.c_int
        L.mis_autotune.argtypes = [P, i32, ctypes.POINTER(mis_tuning)]
        L.mis_autotune.restype = ctypes.c_int
        L.mis_set_grid.argtypes = [P, i32]
        L.mis_set_grid.restype = ctypes.c_int
        L.mis_get_grid.argtypes = [P]
        L.mis_get_grid.restype = i32
        L.mis_tiles_ex.argtypes = [P, P, P, P, P]
        L.mis_tiles_ex.restype = ctypes.c_int
        L.mis_set_csr_bins.argtypes = [P, P]
        L.mis_set_csr_bins.restype = ctypes.c_int
        L.mis_solve_multi_ex.argtypes = [P, i32, P, P, P]
        L.mis_solve_multi_ex.restype = ctypes.c_int
        L.mis_capture.argtypes = [P, P, P, ctypes.POINTER(P)]
        L.mis_capture.restype = ctypes.c_int
        L.mis_replay_launch.argtypes = [P, P]
        L.mis_replay_launch.restype = ctypes.c_int
        L.mis_replay_destroy.argtypes = [P]
        L.mis_replay_destroy.restype = None
        L.mis_set_csr_pending.argtypes = [P, i32]
        L.mis_set_csr_pending.restype = ctypes.c_int
        L.mis_cluster_max_vertices.argtypes = []
        L.mis_cluster_max_vertices.restype = i32
        L.mis_tile_payload_ex.argtypes = [P, i32, P, P]
        L.mis_tile_payload_ex.restype = ctypes.c_int
        L.mis_set_tile_payload.argtypes = [P, i32]
        L.mis_set_tile_payload.restype = ctypes.c_int
        L.mis_set_multi_form.argtypes = [P, i32]
        L.mis_set_multi_form.restype = ctypes.c_int
        L.mis_autotune_multi.argtypes = [P, i32, i32, ctypes.POINTER(ctypes.c_int32)]
        L.mis_autotune_multi.restype = ctypes.c_int
        L.mis_set_csr_range0.argtypes = [P, i32]
        L.mis_set_csr_range0.restype = ctypes.c_int
        L.mis_destroy.argtypes = [P]
        L.mis_destroy.restype = None
        L.mis_update_edges.argtypes = [P, i64, P, i64, P, P]
        L.mis_update_edges.restype = ctypes.c_int
        L.mis_repair.argtypes = [P, u64, i64, P, P, ctypes.POINTER(i64), ctypes.POINTER(i32), P]
        L.mis_repair.restype = ctypes.c_int
        L.mis_add_vertices.argtypes = [P, i32, P]
        L.mis_add_vertices.restype = ctypes.c_int
        L.mis_repair.restype = ctypes.c_int
        L.mis_submit.argtypes = [P, u64, P, ctypes.POINTER(i64)]
        L.mis_submit.restype = ctypes.c_int
        L.mis_poll.argtypes = [i64]
        L.mis_poll.restype = ctypes.c_int
        L.mis_poll_ex.argtypes = [i64, ctypes.POINTER(i64)]
        L.mis_poll_ex.restype = ctypes.c_int
        L.mis_wait.argtypes = [i64, i64]
        L.mis_wait.restype = ctypes.c_int
        L.mis_serve_configure.argtypes = [ctypes.POINTER(mis_options)]
        L.mis_serve_configure.restype = ctypes.c_int
        L.mis_serve_shutdown.argtypes = []
        L.mis_serve_shutdown.restype = None
        L.mis_solve_noalloc.argtypes = [i32, P, P, u64, P, P]
        L.mis_solve_noalloc.restype = ctypes.c_int
        L.mis_last_error.argtypes = [ctypes.POINTER(ctypes.c_char_p)]
        L.mis_last_error.restype = ctypes.c_int
        L.mis_version.argtypes = []
        L.mis_version.restype = ctypes.c_char_p
        _lib = L
        # drain and stop the serving thread before the CUDA runtime unloads
        atexit.register(L.mis_serve_shutdown)
        return L


# header-declared entry points (checked by the CPU test suite)
EXPORTED = [
    "mis_options_init", "mis_create", "mis_create_ex", "mis_create_batch", "mis_graph_count",
    "mis_result_size", "mis_solve", "mis_solve_ex", "mis_get_stats", "mis_keys_ex",
    "mis_set_path", "mis_set_csr_bins", "mis_set_csr_pending", "mis_set_csr_range0", "mis_set_tile_payload", "mis_set_multi_form", "mis_autotune_multi", "mis_tile_payload_ex", "mis_cluster_max_vertices", "mis_capture", "mis_replay_launch", "mis_replay_destroy", "mis_solve_multi_ex", "mis_tiles_ex", "mis_set_grid", "mis_get_grid", "mis_autotune", "mis_footprint", "mis_destroy", "mis_submit", "mis_poll", "mis_poll_ex", "mis_wait",
    "mis_serve_configure", "mis_serve_shutdown", "mis_last_error", "mis_version",
    "mis_solve_noalloc", "mis_update_edges", "mis_repair", "mis_add_vertices",
]


def last_error():
    msg = ctypes.c_char_p()
    code = lib().mis_last_error(ctypes.byref(msg))
    return code, (msg.value or b"").decode()


def _check(rc):
    if rc != MIS_OK:
        code, msg = last_error()
        raise MisError(rc, msg)
    return rc


def options(**kw) -> mis_options:
    o = mis_options()
    lib().mis_options_init(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


# ------------------------------------------------------------ thin wrappers (C names)

def mis_create(n, row_ptr, col_idx):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col_idx, dtype=np.int32)
    h = lib().mis_create(n, _ptr(rp), _ptr(col) if len(col) else None)
    if not h:
        code, msg = last_error()
        raise MisError(code, msg)
    return h


def mis_create_ex(n, row_ptr, col_idx, on_device=0, opt=None, stream=None):
    """row_ptr / col_idx: numpy arrays (host) or integer device pointers."""
    if on_device:
        rp, col = ctypes.c_void_p(row_ptr), ctypes.c_void_p(col_idx)
        keep = None
    else:
        rpa = np.ascontiguousarray(row_ptr, dtype=np.int32)
        cola = np.ascontiguousarray(col_idx, dtype=np.int32)
        rp, col = _ptr(rpa), (_ptr(cola) if len(cola) else None)
        keep = (rpa, cola)
    h = lib().mis_create_ex(n, rp, col, int(on_device),
                            ctypes.byref(opt) if opt is not None else None,
                            ctypes.c_void_p(stream) if stream else None)
    del keep
    if not h:
        code, msg = last_error()
        raise MisError(code, msg)
    return h


def mis_create_batch(graphs, opt=None):
    """graphs: list of (n, row_ptr, col_idx) host arrays."""
    count = len(graphs)
    ns = np.array([g[0] for g in graphs], dtype=np.int32)
    rps = [np.ascontiguousarray(g[1], dtype=np.int32) for g in graphs]
    cols = [np.ascontiguousarray(g[2], dtype=np.int32) for g in graphs]
    rp_ptrs = (ctypes.c_void_p * count)(*[r.ctypes.data for r in rps])
    col_ptrs = (ctypes.c_void_p * count)(*[c.ctypes.data if len(c) else None for c in cols])
    h = lib().mis_create_batch(count, _ptr(ns), rp_ptrs, col_ptrs,
                               ctypes.byref(opt) if opt is not None else None)
    if not h:
        code, msg = last_error()
        raise MisError(code, msg)
    return h


def mis_solve(h, seed, out_status=None):
    size = lib().mis_result_size(h)
    out = out_status if out_status is not None else np.empty(size, dtype=np.uint8)
    _check(lib().mis_solve(h, seed & (2**64 - 1), _ptr(out) if size else None))
    return out


def mis_solve_ex(h, seeds, out_ptr, stream=None):
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64).reshape(-1))
    return _check(lib().mis_solve_ex(h, _ptr(s), ctypes.c_void_p(out_ptr) if out_ptr else None,
                                     ctypes.c_void_p(stream) if stream else None))


def mis_get_stats(h):
    st = mis_stats()
    _check(lib().mis_get_stats(h, ctypes.byref(st)))
    return st


def mis_keys_ex(h, seeds, out_ptr, stream=None):
    s = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64).reshape(-1))
    return _check(lib().mis_keys_ex(h, _ptr(s), ctypes.c_void_p(out_ptr),
                                    ctypes.c_void_p(stream) if stream else None))


def mis_solve_noalloc(n, row_ptr_ptr, col_idx_ptr, seed, out_ptr, stream=None):
    """Allocation-free solve: device pointers in and out (see include/tcmis.h)."""
    return _check(lib().mis_solve_noalloc(n, ctypes.c_void_p(row_ptr_ptr),
                                          ctypes.c_void_p(col_idx_ptr), seed & (2**64 - 1),
                                          ctypes.c_void_p(out_ptr),
                                          ctypes.c_void_p(stream) if stream else None))


def mis_set_path(h, path, threads_per_row=0):
    return _check(lib().mis_set_path(h, path, threads_per_row))


def mis_set_csr_bins(h, bounds):
    b = np.ascontiguousarray(np.asarray(bounds, dtype=np.int32))
    return _check(lib().mis_set_csr_bins(h, _ptr(b)))


def mis_solve_multi_ex(h, seeds, out_ptr, stream=None):
    """k = len(seeds) solves of one graph in one launch; solve s's result at
    out_ptr + s * n (device)."""
    s = np.ascontiguousarray(np.atleast_1d(np.asarray(seeds, dtype=np.uint64)))
    return _check(lib().mis_solve_multi_ex(h, len(s), _ptr(s),
                                           ctypes.c_void_p(out_ptr) if out_ptr else None,
                                           ctypes.c_void_p(stream) if stream else None))


def _pairs(p):
    a = np.ascontiguousarray(np.asarray(p, dtype=np.int32).reshape(-1, 2))
    return a, len(a)


def mis_update_edges(h, ins=(), dels=(), stream=None):
    """Insert and delete undirected edges (host (m, 2) arrays of vertex pairs)."""
    a, na = _pairs(ins)
    d, nd = _pairs(dels)
    return _check(lib().mis_update_edges(h, na, _ptr(a) if na else None, nd,
                                         _ptr(d) if nd else None,
                                         ctypes.c_void_p(stream) if stream else None))


def mis_add_vertices(h, k, stream=None):
    """Append k isolated vertices (ids n .. n+k-1)."""
    return _check(lib().mis_add_vertices(h, int(k), ctypes.c_void_p(stream) if stream else None))


def mis_repair(h, seed, changed, out_ptr, stream=None):
    """Repair the device result at out_ptr (a solve with `seed` before the
    edges in `changed` were inserted or deleted); returns (|M|, rounds)."""
    c, nc = _pairs(changed)
    size = ctypes.c_int64()
    rounds = ctypes.c_int32()
    _check(lib().mis_repair(h, ctypes.c_uint64(int(seed)), nc, _ptr(c) if nc else None,
                            ctypes.c_void_p(out_ptr) if out_ptr else None, ctypes.byref(size),
                            ctypes.byref(rounds), ctypes.c_void_p(stream) if stream else None))
    return size.value, rounds.value


def mis_capture(h, seeds, out_status_dev):
    """Capture one solve of `h` (seeds: one per graph; out_status_dev: device
    pointer) into a replayable CUDA graph; returns the replay handle."""
    s = np.ascontiguousarray(np.atleast_1d(np.asarray(seeds, dtype=np.uint64)))
    r = ctypes.c_void_p()
    _check(lib().mis_capture(h, _ptr(s), ctypes.c_void_p(out_status_dev) if out_status_dev else None,
                             ctypes.byref(r)))
    return r


def mis_replay_launch(r, stream):
    return _check(lib().mis_replay_launch(r, ctypes.c_void_p(stream) if stream else None))


def mis_replay_destroy(r):
    lib().mis_replay_destroy(r)


def mis_set_csr_pending(h, pending):
    return _check(lib().mis_set_csr_pending(h, int(pending)))


MIS_TILE_BITS, MIS_TILE_BITS_B1, MIS_TILE_INT8, MIS_TILE_FP16 = 0, 1, 2, 3


def mis_tile_payload_ex(h, payload, out_ptr, stream=None):
    return _check(lib().mis_tile_payload_ex(h, int(payload), ctypes.c_void_p(out_ptr),
                                            ctypes.c_void_p(stream) if stream else None))


def mis_set_tile_payload(h, payload):
    return _check(lib().mis_set_tile_payload(h, int(payload)))


def mis_set_multi_form(h, form):
    return _check(lib().mis_set_multi_form(h, int(form)))


def mis_autotune_multi(h, k=8, reps=3):
    """Times the multi-seed forms with k seeds, keeps the faster; returns it."""
    form = ctypes.c_int32(-1)
    _check(lib().mis_autotune_multi(h, int(k), int(reps), ctypes.byref(form)))
    return int(form.value)


def mis_set_csr_range0(h, on):
    return _check(lib().mis_set_csr_range0(h, int(on)))


def mis_autotune(h, reps=3):
    t = mis_tuning()
    _check(lib().mis_autotune(h, reps, ctypes.byref(t)))
    return t


def mis_set_grid(h, blocks):
    return _check(lib().mis_set_grid(h, blocks))


def mis_get_grid(h):
    return lib().mis_get_grid(h)


def mis_tiles_ex(h, trp_ptr, tcol_ptr, tbits_ptr, stream=None):
    return _check(lib().mis_tiles_ex(h, ctypes.c_void_p(trp_ptr), ctypes.c_void_p(tcol_ptr),
                                     ctypes.c_void_p(tbits_ptr),
                                     ctypes.c_void_p(stream) if stream else None))


def mis_destroy(h):
    lib().mis_destroy(h)


def mis_submit(h, seed, out_status):
    t = ctypes.c_int64()
    _check(lib().mis_submit(h, seed & (2**64 - 1), _ptr(out_status), ctypes.byref(t)))
    return t.value


def mis_poll(ticket):
    """MIS_OK (done; ticket released), MIS_ENOTREADY, or a negative error."""
    return lib().mis_poll(ticket)


def mis_poll_ex(ticket):
    """(rc, latency_ns): rc as mis_poll; latency from submit to result (done only)."""
    lat = ctypes.c_int64(0)
    rc = lib().mis_poll_ex(ticket, ctypes.byref(lat))
    return rc, lat.value


def mis_wait(ticket, timeout_us=-1):
    """Wait for a request; same returns as mis_poll, MIS_ETIMEDOUT on expiry."""
    return lib().mis_wait(ticket, timeout_us)


def mis_serve_configure(opt=None):
    return _check(lib().mis_serve_configure(ctypes.byref(opt) if opt is not None else None))


def mis_serve_shutdown():
    lib().mis_serve_shutdown()


class Graph:
    """Owning wrapper of a mis_graph handle."""

    def __init__(self, n, row_ptr=None, col_idx=None, opt=None, batch=None):
        if batch is not None:
            self.h = mis_create_batch(batch, opt)
        else:
            self.h = mis_create_ex(n, row_ptr, col_idx, 0, opt)

    @property
    def result_size(self):
        return lib().mis_result_size(self.h)

    @property
    def count(self):
        return lib().mis_graph_count(self.h)

    def solve(self, seed):
        return mis_solve(self.h, seed)

    def stats(self):
        return mis_get_stats(self.h)

    def set_path(self, path, threads_per_row=0):
        mis_set_path(self.h, path, threads_per_row)

    def close(self):
        if self.h:
            mis_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
