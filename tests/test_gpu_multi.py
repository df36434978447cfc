"""Several solves of one graph in one launch (mis_solve_multi_ex): each
solve's set is bit-identical to the oracle's for its seed, and the summed
round statistics match the oracle's per-seed rounds."""
import numpy as np
import pytest

import oracle
from paper_2605_29604_gb300 import graphgen as gg
from paper_2605_29604_gb300 import native

from gpu_util import create, ensure_built, oracle_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    torch.cuda.set_device(0)


FAMILIES = {
    "er_10k": lambda: gg.er_10k_deg8(1),
    "rmat14": lambda: gg.rmat(14, 16, 0.57, 0.19, 0.19, 9, permute=True),
    "rmat14_natural": lambda: gg.rmat(14, 16, 0.57, 0.19, 0.19, 9, permute=False),
    "grid": lambda: gg.grid_diag(127, 0.05, 2),
    "grid_perm": lambda: gg.grid_diag(127, 0.05, 2, permute=True),
    "stencil27": lambda: gg.stencil27(23, 19, 17),  # ragged in every axis
    "star_hub": lambda: gg.disjoint_union([gg.star(150000), gg.er_gnm(5000, 20000, 3)]),
    "dense": lambda: gg.random_small(700, 0.3, 6),
    "k_ab": lambda: gg.complete_bipartite(40, 900),
    "path": lambda: gg.path(5001),
    "empty": lambda: gg.empty(1234),
    "edge": lambda: gg.path(2),
}

_cache = {}


def graph(name):
    if name not in _cache:
        _cache[name] = FAMILIES[name]()
    return _cache[name]


def multi_solve(h, n, seeds):
    import torch
    k = len(seeds)
    out = torch.full((max(k * n, 1),), 7, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    native.mis_solve_multi_ex(h, np.asarray(seeds, dtype=np.uint64), out.data_ptr(), stream)
    st = native.mis_get_stats(h)
    return out[:k * n].cpu().numpy().reshape(k, n), st


def check(g, seeds, got, st):
    n = g[0]
    wants = [oracle_solve(g, int(s)) for s in seeds]
    for s, want, row in zip(seeds, wants, got):
        bad = np.flatnonzero(row != want.status)
        assert len(bad) == 0, f"seed {s}: {len(bad)} vertices differ, first {bad[:10]}"
    rounds = max(w.rounds for w in wants)
    assert st.rounds == rounds
    alive = np.zeros(rounds, dtype=np.int64)
    for w in wants:
        alive[:w.rounds] += np.asarray(w.alive_per_round[:w.rounds], dtype=np.int64)
    r = min(rounds, 64)
    assert list(st.alive_per_round[:r]) == [int(x) for x in alive[:r]]
    assert st.alive_sum == int(sum(w.alive_sum for w in wants))
    assert st.mis_size == int(sum(int(w.status.sum()) for w in wants))


@pytest.mark.parametrize("name", sorted(FAMILIES))
@pytest.mark.parametrize("k", [1, 3, 8])
def test_multi_bit_exact(name, k):
    g = graph(name)
    h = create(g)
    try:
        seeds = [1 + 977 * i for i in range(k)]
        got, st = multi_solve(h, g[0], seeds)
        check(g, seeds, got, st)
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("order_rows", [0, 2])
def test_multi_orderings_and_repeats(order_rows):
    g = graph("rmat14")
    h = create(g, order_rows=order_rows)
    try:
        seeds = [5, 5, 2**63 + 11, 0, 17]
        got, st = multi_solve(h, g[0], seeds)
        check(g, seeds, got, st)
        assert np.array_equal(got[0], got[1])
        # the handle's plain solves still work after a multi-seed solve
        import torch
        out = torch.empty(g[0], dtype=torch.uint8, device="cuda")
        native.mis_solve_ex(h, [17], out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        native.mis_get_stats(h)
        assert np.array_equal(out.cpu().numpy(), got[4])
    finally:
        native.mis_destroy(h)


def test_multi_rejects_bad_arguments():
    import torch
    g = graph("path")
    h = create(g)
    out = torch.empty(9 * g[0], dtype=torch.uint8, device="cuda")
    try:
        for seeds in ([], list(range(9))):
            with pytest.raises(native.MisError):
                native.mis_solve_multi_ex(h, np.asarray(seeds, dtype=np.uint64), out.data_ptr())
    finally:
        native.mis_destroy(h)
    hb = native.mis_create_batch([gg.path(10), gg.path(20)])
    try:
        with pytest.raises(native.MisError):
            native.mis_solve_multi_ex(hb, np.asarray([1, 2], dtype=np.uint64), out.data_ptr())
    finally:
        native.mis_destroy(hb)


PAYLOADS = [native.MIS_TILE_BITS, native.MIS_TILE_BITS_B1, native.MIS_TILE_INT8,
            native.MIS_TILE_FP16]


@pytest.mark.parametrize("name", sorted(FAMILIES))
@pytest.mark.parametrize("payload", PAYLOADS)
@pytest.mark.parametrize("k", [1, 5, 8])
def test_multi_on_tiles_tensor_cores_bit_exact(name, payload, k):
    """The k solves as right-hand sides of the tensor-core exclusion on the
    16 x 16 tiles, in every payload form: each solve's set equals the
    oracle's, and the summed rounds match."""
    g = graph(name)
    h = create(g, order_rows=0)
    try:
        native.mis_set_tile_payload(h, payload)
        native.mis_set_path(h, native.MIS_PATH_TILE_TC, 16)
        seeds = [3 + 1013 * i for i in range(k)]
        got, st = multi_solve(h, g[0], seeds)
        assert st.path == native.MIS_PATH_TILE_TC
        check(g, seeds, got, st)
        # a second launch reuses the bit vectors and words
        seeds2 = [s + 1 for s in seeds]
        got2, st2 = multi_solve(h, g[0], seeds2)
        check(g, seeds2, got2, st2)
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("name", sorted(FAMILIES))
@pytest.mark.parametrize("k", [1, 6, 8])
def test_multi_rows_tc_bit_exact(name, k):
    """Selection test on the CSR rows, exclusion test as the single-bit MMA
    over the 16 x 16 bitmask tiles (MIS_MULTI_ROWS_TC): every solve's set
    equals the oracle's, and the summed rounds and alive sets match; a second
    launch on the same handle (kept tiles, in-set bits and words) too."""
    g = graph(name)
    h = create(g, order_rows=0)
    try:
        native.mis_set_multi_form(h, native.MIS_MULTI_ROWS_TC)
        seeds = [7 + 1009 * i for i in range(k)]
        got, st = multi_solve(h, g[0], seeds)
        assert st.path == native.MIS_PATH_ROWS_TC
        check(g, seeds, got, st)
        seeds2 = [s + 2 for s in seeds]
        got2, st2 = multi_solve(h, g[0], seeds2)
        check(g, seeds2, got2, st2)
        # the CSR-row form on the same handle gives the same sets
        native.mis_set_multi_form(h, native.MIS_MULTI_ROWS)
        got3, st3 = multi_solve(h, g[0], seeds2)
        assert st3.path == native.MIS_PATH_CSR
        assert np.array_equal(got3, got2)
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("priority", [native.MIS_PRIORITY_HASH, native.MIS_PRIORITY_EQ1_Q8])
def test_multi_rows_tc_priorities(priority):
    """The tensor-core multi-seed form under the other priority heuristics
    (H1 hash, Eq. 1 on 8 bits), where ties between neighbours are common."""
    g = graph("grid")
    h = create(g, order_rows=0, priority=priority)
    try:
        native.mis_set_multi_form(h, native.MIS_MULTI_ROWS_TC)
        seeds = [11, 12, 13, 14, 15, 16, 17, 18]
        got, st = multi_solve(h, g[0], seeds)
        n, rp, col = g
        for s, row in zip(seeds, got):
            want = oracle.solve(n, rp, col, s, priority)
            assert np.array_equal(row, want.status), f"seed {s}"
    finally:
        native.mis_destroy(h)


def test_multi_rows_tc_refusals():
    """The form needs a single graph without create-time round-0 structures;
    a graph on 8 x 8 tiles is refused at solve time."""
    import torch
    g = graph("grid")
    h = create(g, order_rows=1)
    try:
        with pytest.raises(native.MisError):
            native.mis_set_multi_form(h, native.MIS_MULTI_ROWS_TC)
        with pytest.raises(native.MisError):
            native.mis_set_multi_form(h, 5)
    finally:
        native.mis_destroy(h)
    hb = native.mis_create_batch([gg.path(10), gg.path(20)])
    try:
        with pytest.raises(native.MisError):
            native.mis_set_multi_form(hb, native.MIS_MULTI_ROWS_TC)
    finally:
        native.mis_destroy(hb)
    h = create(g, order_rows=0)
    out = torch.empty(2 * g[0], dtype=torch.uint8, device="cuda")
    try:
        native.mis_set_multi_form(h, native.MIS_MULTI_ROWS_TC)
        native.mis_set_path(h, native.MIS_PATH_TILE, 8)
        with pytest.raises(native.MisError):
            native.mis_solve_multi_ex(h, np.asarray([1, 2], dtype=np.uint64), out.data_ptr())
        native.mis_set_path(h, native.MIS_PATH_CSR, 0)
        got, st = multi_solve(h, g[0], [1, 2])
        check(g, [1, 2], got, st)
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("name", ["grid", "stencil27", "rmat14", "empty"])
def test_multi_autotune_form(name):
    """mis_autotune_multi times both multi-seed forms and keeps one; the
    solves that follow in that form are bit-exact, and a graph with
    create-time round-0 structures keeps the CSR-row form untimed."""
    g = graph(name)
    h = create(g, order_rows=0)
    try:
        form = native.mis_autotune_multi(h, 8, 2)
        assert form in (native.MIS_MULTI_ROWS, native.MIS_MULTI_ROWS_TC)
        seeds = [31 + i for i in range(8)]
        got, st = multi_solve(h, g[0], seeds)
        if g[0] > 0:
            assert st.path == (native.MIS_PATH_ROWS_TC if form == native.MIS_MULTI_ROWS_TC
                               else native.MIS_PATH_CSR)
        check(g, seeds, got, st)
    finally:
        native.mis_destroy(h)
    h = create(g, order_rows=1)
    try:
        assert native.mis_autotune_multi(h, 4, 1) == native.MIS_MULTI_ROWS
        with pytest.raises(native.MisError):
            native.mis_autotune_multi(h, 9, 1)
    finally:
        native.mis_destroy(h)
