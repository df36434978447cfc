"""The allocation-free entry point, mis_solve_noalloc.

Callers that cannot allocate device memory (inside a custom allocator, with
all device memory reserved by a framework, or in loops that cannot take an
allocation's latency) use mis_solve_noalloc, which keeps its scratch in a
fixed array inside the library.  This file checks, through the C ABI, that
it returns exactly the set that the regular entry point (mis_solve_ex)
returns, on two calls in a row that share that scratch, and that it rejects
sizes beyond its fixed limit.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_2605_29604_gb300 import graphgen as gg
from paper_2605_29604_gb300 import native

pytestmark = pytest.mark.gpu

LIMIT = 262144


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_29604_gb300 import build as nbuild
    nbuild.build()
    native.lib()
    torch.cuda.set_device(0)


def _regular(g, seed):
    import torch
    n, rp, col = g
    h = native.mis_create_ex(n, rp, col, 0, native.options(), None)
    try:
        out = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
        native.mis_solve_ex(h, [seed], out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        native.mis_get_stats(h)
        return out[:n].cpu().numpy()
    finally:
        native.mis_destroy(h)


def _noalloc(g, seed):
    import torch
    n, rp, col = g
    drp = torch.from_numpy(rp).cuda()
    # an unpadded, odd-offset view: the entry point must not need padding or alignment
    dcol_store = torch.zeros(len(col) + 1, dtype=torch.int32, device="cuda")
    dcol_store[1:] = torch.from_numpy(col).cuda()
    dcol = dcol_store[1:]
    out = torch.full((max(n, 1),), 9, dtype=torch.uint8, device="cuda")
    native.mis_solve_noalloc(n, drp.data_ptr(), dcol.data_ptr() if len(col) else 0, seed,
                             out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return out[:n].cpu().numpy()


@pytest.mark.parametrize("make,seed", [
    (lambda: gg.rmat(16, 16, 0.57, 0.19, 0.19, 5, permute=True), 3),
    (lambda: gg.er_gnm(LIMIT, 4 * LIMIT, 2), 11),
    (lambda: gg.grid_diag(300, 0.05, 1, permute=True), 7),
])
def test_noalloc_matches_regular_entry_point_twice(make, seed):
    g = make()
    want = _regular(g, seed)
    first = _noalloc(g, seed)
    second = _noalloc(g, seed + 1)   # the shared scratch keeps the first call's contents
    third = _noalloc(g, seed)
    assert np.array_equal(first, want)  # bit-exact, the tolerance of every parity test here
    assert np.array_equal(third, want)
    assert np.array_equal(second, _regular(g, seed + 1))


def test_noalloc_limit_and_empty():
    import torch
    assert native.mis_solve_noalloc(0, 0, 0, 1, 0) == native.MIS_OK
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(native.MisError) as ei:
        native.mis_solve_noalloc(LIMIT + 1, dummy.data_ptr(), dummy.data_ptr(), 1,
                                 dummy.data_ptr())
    assert ei.value.code == native.MIS_EINVAL
    assert "262144" in str(ei.value)


def test_noalloc_allocates_nothing():
    # what the entry point exists for: after a warm-up call (which loads the
    # library's device code, the fixed array included), further calls leave
    # the device's free memory and the torch pool's bytes exactly as they were
    import torch
    g = gg.rmat(14, 16, 0.57, 0.19, 0.19, 9, permute=True)
    n, rp, col = g
    drp = torch.from_numpy(rp).cuda()
    dcol = torch.from_numpy(col).cuda()
    out = torch.empty(n, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    native.mis_solve_noalloc(n, drp.data_ptr(), dcol.data_ptr(), 1, out.data_ptr(), stream)
    torch.cuda.synchronize()
    import gc
    gc.collect()  # tensors of earlier tests freed now, not during the measured calls
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    allocated0 = torch.cuda.memory_allocated()
    for seed in (2, 3, 4):
        native.mis_solve_noalloc(n, drp.data_ptr(), dcol.data_ptr(), seed, out.data_ptr(), stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0
    # a call that allocated through the pool would raise this count
    assert torch.cuda.memory_allocated() <= allocated0
    assert np.array_equal(out.cpu().numpy(), _regular(g, 4))


def test_noalloc_null_col_idx():
    import torch
    # a graph without arcs may pass a null col_idx: every vertex is isolated
    n = 37
    drp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    out = torch.zeros(n, dtype=torch.uint8, device="cuda")
    native.mis_solve_noalloc(n, drp.data_ptr(), 0, 5, out.data_ptr())
    assert int(out.sum()) == n
    # with arcs, a null col_idx is refused before any launch
    rp = torch.from_numpy(np.arange(0, 2 * n + 1, 2, dtype=np.int32)).cuda()
    with pytest.raises(native.MisError) as ei:
        native.mis_solve_noalloc(n, rp.data_ptr(), 0, 5, out.data_ptr())
    assert ei.value.code == native.MIS_EINVAL
