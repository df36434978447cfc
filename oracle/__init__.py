"""CPU oracle for the TC-MIS hot path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The library's own code path never does,
and this package imports nothing from it: the oracle and the CUDA path share
no code.

What is here (each function cites the part of the paper it follows):

- ``keys``            Eq. 1 priorities, assigned once per solve (Sec. 2).
- ``rounds``          Algorithm 2's while-loop, phase by phase, snapshot per round.
- ``greedy``          sequential greedy in decreasing priority: the closed form
                      of the round iteration's result.
- ``check``           independence and maximality.
- ``min_degree_greedy`` quality yardstick (not parity).
- ``brute_force_mis`` every maximal independent set of a graph with n <= 20.
- ``eps`` / ``priority`` / ``splitmix64_mix``  the pieces of Eq. 1, exposed
                      so that tests can pin them separately.
- ``rounds_parallel`` / ``solve_parallel``  not the oracle: a second CPU
                      baseline, the same rounds over worklists on all host
                      cores (``cpu_parallel.c``, OpenMP), checked against
                      ``rounds`` by the tests and timed beside it by bench.py.

The arithmetic lives in ``tcmis_oracle.c`` (plain C, one thread, binary32
round-to-nearest with no FMA contraction); the brute force is pure Python.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tcmis_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i32, i64, u64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float
        P = ctypes.c_void_p
        lib.orc_splitmix64_mix.argtypes = [u64]
        lib.orc_splitmix64_mix.restype = u64
        lib.orc_eps.argtypes = [u64, i32]
        lib.orc_eps.restype = f32
        lib.orc_priority.argtypes = [f32, i32, f32]
        lib.orc_priority.restype = f32
        lib.orc_keys.argtypes = [i32, P, u64, P]
        lib.orc_keys.restype = None
        lib.orc_keys_mode.argtypes = [i32, P, u64, i32, P]
        lib.orc_keys_mode.restype = None
        lib.orc_rounds.argtypes = [i32, P, P, P, P, P, P, P, P, i32]
        lib.orc_rounds.restype = ctypes.c_int
        lib.orc_greedy.argtypes = [i32, P, P, P, P]
        lib.orc_greedy.restype = ctypes.c_int
        lib.orc_check.argtypes = [i32, P, P, P, P]
        lib.orc_check.restype = ctypes.c_int
        lib.orc_min_degree_greedy.argtypes = [i32, P, P, P]
        lib.orc_min_degree_greedy.restype = i64
        _lib = lib
        return lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _csr(row_ptr, col_idx):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(col_idx, dtype=np.int32)
    if len(col) == 0:
        col = np.zeros(1, dtype=np.int32)
    return rp, col


def splitmix64_mix(z: int) -> int:
    """splitmix64's 64-bit finaliser (Steele, Lea, Flood, OOPSLA 2014)."""
    return int(_load().orc_splitmix64_mix(z & (2**64 - 1)))


def eps(seed: int, v: int) -> float:
    """eps(v) of Eq. 1: (hi32(mix(mix(seed) ^ v)) >> 8) * 2^-24, in [0, 1)."""
    return float(_load().orc_eps(seed & (2**64 - 1), v))


def priority(dbar: float, deg: int, e: float) -> float:
    """Eq. 1 in binary32: dbar / ((dbar + deg) - eps)."""
    return float(_load().orc_priority(dbar, deg, e))


# Priority heuristics of Sec. 3.3 (the mode argument of keys/solve).
PRIORITY_EQ1 = 0  # H2/H3: Eq. 1, degree-aware
PRIORITY_HASH = 1  # H1: random priority hash(v)
PRIORITY_EQ1_Q8 = 2  # Eq. 1 discretised to 8 bits


def keys(n: int, row_ptr, seed: int, priority: int = PRIORITY_EQ1) -> np.ndarray:
    """uint32 priority keys (0xFFFFFFFF if isolated).  PRIORITY_EQ1: bits of
    binary32 P of Eq. 1; PRIORITY_HASH: 2^29 + (hi32(mix(mix(seed) ^ v)) >> 3);
    PRIORITY_EQ1_Q8: trunc(255 * P) in binary32."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    out = np.empty(max(n, 1), dtype=np.uint32)
    if priority == PRIORITY_EQ1:
        _load().orc_keys(n, _p(rp), seed & (2**64 - 1), _p(out))
    else:
        _load().orc_keys_mode(n, _p(rp), seed & (2**64 - 1), int(priority), _p(out))
    return out[:n]


class RoundsResult:
    def __init__(self, status, rounds, work, alive_sum, alive_per_round):
        self.status = status
        self.rounds = rounds
        self.work = work
        self.alive_sum = alive_sum
        self.alive_per_round = alive_per_round


def rounds(n: int, row_ptr, col_idx, key, max_rounds: int | None = None) -> RoundsResult:
    """Algorithm 2 simulated round by round on the CPU (see tcmis_oracle.c)."""
    rp, col = _csr(row_ptr, col_idx)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    if n == 0:
        return RoundsResult(np.zeros(0, np.uint8), 0, 0, 0, np.zeros(0, np.int64))
    cap = max_rounds if max_rounds is not None else n + 1
    st = np.empty(n, dtype=np.uint8)
    r = ctypes.c_int32()
    w = ctypes.c_int64()
    a = ctypes.c_int64()
    per = np.zeros(cap, dtype=np.int64)
    rc = _load().orc_rounds(n, _p(rp), _p(col), _p(k), _p(st), ctypes.byref(r), ctypes.byref(w),
                            ctypes.byref(a), _p(per), cap)
    if rc != 0:
        raise RuntimeError("oracle round simulation did not terminate within the round cap")
    return RoundsResult(st, r.value, w.value, a.value, per[:r.value].copy())


def greedy(n: int, row_ptr, col_idx, key) -> np.ndarray:
    """Sequential greedy in decreasing (key, id) order (lexicographically-first MIS)."""
    rp, col = _csr(row_ptr, col_idx)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    st = np.empty(max(n, 1), dtype=np.uint8)
    if _load().orc_greedy(n, _p(rp), _p(col), _p(k), _p(st)) != 0:
        raise MemoryError("oracle greedy")
    return st[:n]


def check(n: int, row_ptr, col_idx, status) -> tuple[int, int]:
    """(code, vertex): code 0 = independent and maximal, 1 = two adjacent members
    (at vertex), 2 = an uncovered non-member (at vertex)."""
    rp, col = _csr(row_ptr, col_idx)
    st = np.ascontiguousarray(status, dtype=np.uint8)
    if len(st) == 0:
        st = np.zeros(1, np.uint8)
    bad = ctypes.c_int32(-1)
    code = _load().orc_check(n, _p(rp), _p(col), _p(st), ctypes.byref(bad))
    return code, bad.value


def min_degree_greedy(n: int, row_ptr, col_idx) -> tuple[int, np.ndarray]:
    rp, col = _csr(row_ptr, col_idx)
    st = np.empty(max(n, 1), dtype=np.uint8)
    size = _load().orc_min_degree_greedy(n, _p(rp), _p(col), _p(st))
    if size < 0:
        raise MemoryError("oracle min-degree greedy")
    return int(size), st[:n]


def solve(n: int, row_ptr, col_idx, seed: int, priority: int = PRIORITY_EQ1) -> RoundsResult:
    """Keys (Eq. 1 or another heuristic of Sec. 3.3) then Algorithm 2's rounds:
    the full hot path on the CPU."""
    return rounds(n, row_ptr, col_idx, keys(n, row_ptr, seed, priority))


# ---- the second CPU baseline (cpu_parallel.c): the same rounds on all cores

_PAR_SRC = os.path.join(_HERE, "cpu_parallel.c")
_PAR_LIB = os.path.join(_HERE, "libcpupar.so")
_par = None


def build_parallel(force: bool = False) -> str:
    """Compile cpu_parallel.c with OpenMP where gcc has it, else without."""
    if (force or not os.path.exists(_PAR_LIB)
            or os.path.getmtime(_PAR_LIB) < os.path.getmtime(_PAR_SRC)):
        tmp = _PAR_LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-o", tmp, _PAR_SRC]
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _PAR_LIB)
    return _PAR_LIB


def _load_parallel():
    global _par
    with _lock:
        if _par is None:
            lib = ctypes.CDLL(build_parallel())
            P = ctypes.c_void_p
            lib.par_rounds.argtypes = [ctypes.c_int32, P, P, P, P, P, P, P, ctypes.c_int32,
                                       ctypes.c_int32]
            lib.par_rounds.restype = ctypes.c_int
            lib.par_threads.argtypes = []
            lib.par_threads.restype = ctypes.c_int
            _par = lib
        return _par


def parallel_threads() -> int:
    return int(_load_parallel().par_threads())


def rounds_parallel(n: int, row_ptr, col_idx, key, threads: int = 0) -> RoundsResult:
    """Algorithm 2's rounds on all host cores (cpu_parallel.c); the same
    result, rounds and alive sets as rounds().  work is not counted (0)."""
    rp, col = _csr(row_ptr, col_idx)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    if n == 0:
        return RoundsResult(np.zeros(0, np.uint8), 0, 0, 0, np.zeros(0, np.int64))
    cap = n + 1
    st = np.empty(n, dtype=np.uint8)
    r = ctypes.c_int32()
    a = ctypes.c_int64()
    per = np.zeros(cap, dtype=np.int64)
    rc = _load_parallel().par_rounds(n, _p(rp), _p(col), _p(k), _p(st), ctypes.byref(r),
                                     ctypes.byref(a), _p(per), cap, int(threads))
    if rc != 0:
        raise RuntimeError("parallel round simulation did not terminate within the round cap")
    return RoundsResult(st, r.value, 0, a.value, per[:r.value].copy())


def solve_parallel(n: int, row_ptr, col_idx, seed: int, priority: int = PRIORITY_EQ1,
                   threads: int = 0) -> RoundsResult:
    """keys() (sequential), then the rounds on all host cores."""
    return rounds_parallel(n, row_ptr, col_idx, keys(n, row_ptr, seed, priority), threads)


def brute_force_mis(n: int, row_ptr, col_idx) -> list[int]:
    """All maximal independent sets of a graph with n <= 20, as bitmasks.

    Plain enumeration: every independent subset is generated by deciding the
    vertices 0..n-1 in turn (a vertex may join only if no chosen vertex is
    adjacent), and a complete subset is kept when every non-member has a
    member neighbour.  No MIS algorithm is involved."""
    if n > 20:
        raise ValueError("brute force is limited to n <= 20")
    nb = [0] * n
    for v in range(n):
        for p in range(int(row_ptr[v]), int(row_ptr[v + 1])):
            nb[v] |= 1 << int(col_idx[p])
    full = (1 << n) - 1
    out = []

    def rec(v, chosen, covered):
        if v == n:
            if covered == full:
                out.append(chosen)
            return
        if not (nb[v] & chosen):
            rec(v + 1, chosen | (1 << v), covered | (1 << v) | nb[v])
        rec(v + 1, chosen, covered)

    rec(0, 0, 0)
    return out
