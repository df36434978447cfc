"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times (the headline: full rows, no create-time decisions, autotuned kernel;
beside it the amortised graph with create-time degree order; the batch as a
captured and replayed launch; the grid's tile paths and 8-seed tensor-core
launch).  The oracle solves these graphs in
seconds, so every output is compared, with the round structure; independence
and maximality are checked on top."""
import numpy as np
import pytest

import oracle
from paper_2605_29604_gb300 import graphgen as gg
from paper_2605_29604_gb300 import native

from gpu_util import assert_same, ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    torch.cuda.set_device(0)


def _bench_handle(g, order_rows=2):
    """order_rows = 0: the headline solve (full rows, no create-time round-0
    decisions); 2: the amortised one (create-time structures)."""
    n, rp, col = g
    h = native.mis_create_ex(n, rp, col, 0,
                             native.options(check_symmetry=1, order_rows=order_rows), None)
    native.mis_autotune(h, 3)
    return h


def _solve(h, n, seeds):
    import torch
    out = torch.full((max(n, 1),), 7, dtype=torch.uint8, device="cuda")
    native.mis_solve_ex(h, np.asarray(seeds, dtype=np.uint64), out.data_ptr(),
                        torch.cuda.current_stream().cuda_stream)
    return out[:n].cpu().numpy(), native.mis_get_stats(h)


@pytest.mark.parametrize("order_rows", [0, 2])
@pytest.mark.parametrize("name", ["rmat22", "grid", "grid_perm"])
def test_full_size_single_graph(name, order_rows):
    g = {"rmat22": lambda: gg.rmat22(seed=22),
         "grid": lambda: gg.grid2048(seed=3),
         "grid_perm": lambda: gg.grid2048(seed=3, permute_ids=True)}[name]()
    n, rp, col = g
    h = _bench_handle(g, order_rows)
    try:
        for seed in (1, 2**63 + 11):
            got, st = _solve(h, n, [seed])
            assert_same(g, seed, got, st)
            assert oracle.check(n, rp, col, got)[0] == 0
    finally:
        native.mis_destroy(h)


def test_full_size_multi_seed_rmat22():
    """Eight seeds of R-MAT scale 22 in one launch: each equals its oracle solve."""
    import torch
    g = gg.rmat22(seed=22)
    n, rp, col = g
    h = _bench_handle(g)
    try:
        seeds = np.arange(1, 9, dtype=np.uint64)
        out = torch.empty(8 * n, dtype=torch.uint8, device="cuda")
        native.mis_solve_multi_ex(h, seeds, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        host = out.cpu().numpy()
        for s in (0, 7):
            want = oracle.solve(n, rp, col, int(seeds[s]))
            assert np.array_equal(host[s * n:(s + 1) * n], want.status), s
    finally:
        native.mis_destroy(h)


def test_full_size_batch4096_replayed():
    """The 4096-graph batch as bench.py times it: one captured launch,
    replayed; every graph's result equals its own oracle solve."""
    import torch
    parts = gg.batch_mixed(4096, seed=4096, nmin=64, nmax=65536)
    h = native.mis_create_batch(parts, native.options(check_symmetry=1, order_rows=2))
    try:
        native.mis_autotune(h, 3)
        size = native.lib().mis_result_size(h)
        out = torch.full((size,), 7, dtype=torch.uint8, device="cuda")
        seeds = np.arange(1, len(parts) + 1, dtype=np.uint64)
        r = native.mis_capture(h, seeds, out.data_ptr())
        try:
            s = torch.cuda.current_stream().cuda_stream
            native.mis_replay_launch(r, s)
            out.fill_(7)
            native.mis_replay_launch(r, s)  # the second replay must redo everything
            host = out.cpu().numpy()
        finally:
            native.mis_replay_destroy(r)
        off = 0
        for i, (n, rp, col) in enumerate(parts):
            want = oracle.solve(n, rp, col, int(seeds[i])).status
            assert np.array_equal(host[off:off + n], want), i
            off += n
        assert off == size
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("payload", [native.MIS_TILE_BITS, native.MIS_TILE_BITS_B1,
                                     native.MIS_TILE_INT8, native.MIS_TILE_FP16])
def test_full_size_grid_tensor_core_forms(payload):
    """The grid (natural ids) on the tensor-core tile path in every payload
    form, one seed and eight seeds per launch, as bench.py's tc leg runs it."""
    import torch
    g = gg.grid2048(seed=3)
    n, rp, col = g
    h = native.mis_create_ex(n, rp, col, 0, native.options(order_rows=0), None)
    try:
        native.mis_set_tile_payload(h, payload)
        native.mis_set_path(h, native.MIS_PATH_TILE_TC, 16)
        got, st = _solve(h, n, [5])
        assert_same(g, 5, got, st)
        seeds = np.arange(1, 9, dtype=np.uint64)
        out = torch.empty(8 * n, dtype=torch.uint8, device="cuda")
        native.mis_solve_multi_ex(h, seeds, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        host = out.cpu().numpy()
        for s in (0, 7):
            want = oracle.solve(n, rp, col, int(seeds[s]))
            assert np.array_equal(host[s * n:(s + 1) * n], want.status), s
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("name", ["grid", "stencil"])
def test_full_size_multi_rows_tc(name):
    """Eight seeds per launch with the selection on the CSR rows and the
    exclusion on tensor cores, as bench.py's tc legs time it (the 2048 x 2048
    grid and the 160^3 stencil lattice, natural ids, full-row graphs after the
    autotuner): every solve equals its oracle solve, and the summed rounds and
    alive sets match."""
    import torch
    g = gg.grid2048(seed=3) if name == "grid" else gg.stencil160()
    n, rp, col = g
    h = native.mis_create_ex(n, rp, col, 0, native.options(order_rows=0), None)
    try:
        native.mis_autotune(h, 3)
        native.mis_set_multi_form(h, native.MIS_MULTI_ROWS_TC)
        seeds = np.arange(1, 9, dtype=np.uint64)
        out = torch.empty(8 * n, dtype=torch.uint8, device="cuda")
        native.mis_solve_multi_ex(h, seeds, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        st = native.mis_get_stats(h)
        assert st.path == native.MIS_PATH_ROWS_TC
        host = out.cpu().numpy()
        wants = [oracle.solve(n, rp, col, int(s)) for s in seeds]
        for s, want in enumerate(wants):
            assert np.array_equal(host[s * n:(s + 1) * n], want.status), s
        assert st.rounds == max(w.rounds for w in wants)
        alive = np.zeros(st.rounds, dtype=np.int64)
        for w in wants:
            alive[:w.rounds] += np.asarray(w.alive_per_round[:w.rounds], dtype=np.int64)
        assert list(st.alive_per_round[:st.rounds]) == [int(x) for x in alive]
    finally:
        native.mis_destroy(h)
