"""GPU parity of the CSR round kernel against the CPU oracle.

Every comparison is bit-exact on the vertex set (the result is unique for a
given graph and seed), and the round structure of Algorithm 2 (rounds, alive
set size per round) must match too.
"""
import numpy as np
import pytest

import oracle
from paper_2605_29604_gb300 import graphgen as gg
from paper_2605_29604_gb300 import native

from gpu_util import assert_same, create, ensure_built, gpu_keys, gpu_solve, oracle_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    torch.cuda.set_device(0)


FAMILIES = {
    "er_small": lambda: gg.er_gnm(3000, 12000, 4),
    "er_10k": lambda: gg.er_10k_deg8(1),
    "rmat14": lambda: gg.rmat(14, 16, 0.57, 0.19, 0.19, 9, permute=True),
    "rmat14_natural": lambda: gg.rmat(14, 16, 0.57, 0.19, 0.19, 9, permute=False),
    "grid": lambda: gg.grid_diag(127, 0.05, 2),
    "grid_perm": lambda: gg.grid_diag(127, 0.05, 2, permute=True),
    "stencil27": lambda: gg.stencil27(23, 19, 17),  # ragged in every axis
    "rgg": lambda: gg.rgg(20000, 10.0, 3),
    "dense": lambda: gg.random_small(700, 0.3, 6),
    "star_hub": lambda: gg.disjoint_union([gg.star(150000), gg.er_gnm(5000, 20000, 3)]),
    "path": lambda: gg.path(5001),
    "cycle": lambda: gg.cycle(4099),
    "complete": lambda: gg.complete(300),
    "k_ab": lambda: gg.complete_bipartite(40, 900),
    "empty": lambda: gg.empty(1234),
    "single": lambda: gg.empty(1),
    "edge": lambda: gg.path(2),
}

_cache = {}


def graph(name):
    if name not in _cache:
        _cache[name] = FAMILIES[name]()
    return _cache[name]


@pytest.mark.parametrize("name", sorted(FAMILIES))
def test_keys_bit_exact(name):
    g = graph(name)
    n, rp, col = g
    h = create(g)
    try:
        for seed in (1, 2**63 + 5):
            got = gpu_keys(h, [seed])
            want = oracle.keys(n, rp, seed)
            assert np.array_equal(got, want)
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("name", sorted(FAMILIES))
@pytest.mark.parametrize("tpr", [0, 1, 4, 16, 32, 512])
def test_csr_solve_bit_exact(name, tpr):
    g = graph(name)
    h = create(g)
    try:
        for seed in (1, 7):
            got, st = gpu_solve(h, [seed], native.MIS_PATH_CSR, tpr)
            assert st.path == native.MIS_PATH_CSR and st.threads_per_row == tpr
            assert_same(g, seed, got, st)
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("name", sorted(FAMILIES))
@pytest.mark.parametrize("tpr", [0, 1, 4, 32, 512])
def test_csr_pending_list_bit_exact(name, tpr):
    """Phase 2 over Phase 1's pending list instead of a triage of W_r."""
    g = graph(name)
    h = create(g)
    try:
        native.mis_set_csr_pending(h, 1)
        for seed in (1, 7):
            got, st = gpu_solve(h, [seed], native.MIS_PATH_CSR, tpr)
            assert st.csr_pending == 1
            assert_same(g, seed, got, st)
        native.mis_set_csr_pending(h, 0)
        got, st = gpu_solve(h, [9], native.MIS_PATH_CSR, tpr)
        assert st.csr_pending == 0
        assert_same(g, 9, got, st)
    finally:
        native.mis_destroy(h)


def test_csr_pending_rejects_bad_mode():
    h = create(graph("path"))
    try:
        for bad in (-1, 2, 7):
            with pytest.raises(RuntimeError):
                native.mis_set_csr_pending(h, bad)
    finally:
        native.mis_destroy(h)


def _sure_sets(g):
    """Round-0 decisions that need no test, from their definition: a vertex
    whose neighbours all have degree >= deg + 2 outranks every neighbour under
    Eq. 1 (sure candidate); a vertex with such a neighbour is excluded."""
    n, rp, col = g
    rp = rp.astype(np.int64)
    deg = np.diff(rp)
    if len(col) == 0:
        return 0, 0
    src = np.repeat(np.arange(n), deg)
    outranked = (deg[col] >= deg[src] + 2)
    nz = deg > 0
    all_lower = np.zeros(n, dtype=bool)
    all_lower[nz] = np.logical_and.reduceat(outranked, rp[:-1][nz])
    sure_in = nz & all_lower
    has = np.zeros(n, dtype=bool)
    has[nz] = np.logical_or.reduceat(sure_in[col], rp[:-1][nz])
    sure_out = nz & ~sure_in & has
    return int(sure_in.sum()), int(sure_out.sum())


def _tested_arcs(g):
    """Arcs between vertices that are neither isolated nor decided at create
    time: the only ones the round-0 exclusion test and every later round can
    need, since every other vertex is decided by the end of round 0."""
    n, rp, col = g
    rp = rp.astype(np.int64)
    deg = np.diff(rp)
    if len(col) == 0:
        return 0
    src = np.repeat(np.arange(n), deg)
    outranked = (deg[col] >= deg[src] + 2)
    nz = deg > 0
    all_lower = np.zeros(n, dtype=bool)
    all_lower[nz] = np.logical_and.reduceat(outranked, rp[:-1][nz])
    has = np.zeros(n, dtype=bool)
    has[nz] = np.logical_or.reduceat(all_lower[col], rp[:-1][nz])
    tested = nz & ~has & ~all_lower
    return int((tested[src] & tested[col]).sum())


@pytest.mark.parametrize("order_rows", [0, 1, 2])
@pytest.mark.parametrize("name", ["rmat14", "star_hub", "er_10k", "k_ab", "grid", "path", "empty"])
def test_round0_sure_sets(name, order_rows):
    """Vertices decided at create time: counts match their definition, and
    the result, rounds and alive sets still match Algorithm 2."""
    g = graph(name)
    h = create(g, order_rows=order_rows)
    try:
        for pending in (0, 1):
            native.mis_set_csr_pending(h, pending)
            got, st = gpu_solve(h, [13], native.MIS_PATH_CSR, 0)
            assert_same(g, 13, got, st)
            want = _sure_sets(g) if order_rows else (0, 0)
            assert (st.sure_in, st.sure_out) == want
            # the tested subgraph is kept when it holds at most half the arcs
            t = _tested_arcs(g)
            want_t = t if order_rows and 2 * t <= len(g[2]) and g[0] > 0 else -1
            assert st.tested_arcs == want_t
    finally:
        native.mis_destroy(h)


def _keyed_count(g):
    """Vertices whose words a solve with the tested subgraph reads: the
    tested vertices and every vertex in one of their selection prefixes
    (neighbours of degree <= deg + 1)."""
    n, rp, col = g
    rp = rp.astype(np.int64)
    deg = np.diff(rp)
    src = np.repeat(np.arange(n), deg)
    outranked = (deg[col] >= deg[src] + 2)
    nz = deg > 0
    all_lower = np.zeros(n, dtype=bool)
    all_lower[nz] = np.logical_and.reduceat(outranked, rp[:-1][nz])
    has = np.zeros(n, dtype=bool)
    has[nz] = np.logical_or.reduceat(all_lower[col], rp[:-1][nz])
    tested = nz & ~has & ~all_lower
    need = tested.copy()
    in_prefix = tested[src] & ~outranked
    need[col[in_prefix]] = True
    return int(need.sum()), int(tested.sum()), int(in_prefix.sum())


@pytest.mark.parametrize("offset", [0, 1, 3, 16])
def test_keyed_result_any_alignment(offset):
    """With the keyed list a solve starts its result from create-time bytes
    and writes candidates as it selects them: every byte of the result is
    written at any alignment of the buffer, none around it, and successive
    seeds on one handle (stale words of vertices no test reads) agree with
    the oracle."""
    import torch
    for name in ("rmat14", "star_hub", "k_ab"):
        g = graph(name)
        n = g[0]
        h = create(g, order_rows=2)
        try:
            native.mis_set_path(h, native.MIS_PATH_CSR, 0)
            buf = torch.empty(n + 64, dtype=torch.uint8, device="cuda")
            stream = torch.cuda.current_stream().cuda_stream
            for pending in (0, 1):
                native.mis_set_csr_pending(h, pending)
                for seed in (5, 6, 2**63 + 1):
                    buf.fill_(7)
                    native.mis_solve_ex(h, np.array([seed], dtype=np.uint64),
                                        buf.data_ptr() + offset, stream)
                    st = native.mis_get_stats(h)
                    host = buf.cpu().numpy()
                    assert_same(g, seed, host[offset:offset + n], st)
                    assert (host[:offset] == 7).all() and (host[offset + n:] == 7).all()
                    if st.tested_arcs >= 0:
                        assert (st.keyed, st.tested_rows, st.tested_prefix_arcs) == _keyed_count(g)
        finally:
            native.mis_destroy(h)


@pytest.mark.parametrize("bounds", [(2, 5, 9, 20), (-1, 3, 3, 3), (0, 0, 100000, 100000),
                                    (1, 2, 3, 4), (-1, -1, -1, 2)])
def test_csr_custom_bins(bounds):
    for name in ("rmat14", "grid_perm", "star_hub"):
        g = graph(name)
        h = create(g)
        try:
            native.mis_set_csr_bins(h, bounds)
            got, st = gpu_solve(h, [5])
            assert st.threads_per_row == 0
            assert_same(g, 5, got, st)
        finally:
            native.mis_destroy(h)


@pytest.mark.parametrize("order_rows", [0, 1, 2])
@pytest.mark.parametrize("name", ["rmat14", "grid_perm", "star_hub", "dense", "k_ab", "cycle"])
def test_row_orderings_bit_exact(name, order_rows):
    g = graph(name)
    h = create(g, order_rows=order_rows)
    try:
        for pending in (0, 1):
            native.mis_set_csr_pending(h, pending)
            for tpr in (0, 1):
                got, st = gpu_solve(h, [3], native.MIS_PATH_CSR, tpr)
                assert_same(g, 3, got, st)
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("name", sorted(FAMILIES))
@pytest.mark.parametrize("priority", [0, 1, 2])
def test_range_round0_bit_exact(name, priority):
    """Graphs without round-0 classes (order_rows = 0, or H1 / 8-bit keys):
    round 0 reaches bin 0 by vertex ranges or through its list, with and
    without the pending list, at several bin-0 bounds (including every row
    in bin 0, hubs too)."""
    g = graph(name)
    h = create(g, order_rows=0, priority=priority)
    try:
        seed = 11
        want = oracle.solve(g[0], g[1], g[2], seed, priority)
        for bounds in ((8, 4096, 4096, 65536), (1, 2, 3, 4), (32, 64, 64, 64),
                       (2**31 - 2,) * 4):
            native.mis_set_csr_bins(h, bounds)
            for range0 in (1, 0):
                native.mis_set_csr_range0(h, range0)
                for pending in (0, 1):
                    native.mis_set_csr_pending(h, pending)
                    got, st = gpu_solve(h, [seed])
                    assert_same(g, seed, got, st, want)
    finally:
        native.mis_destroy(h)


def test_range_round0_rejects_bad_mode():
    h = create(graph("path"), order_rows=0)
    try:
        with pytest.raises(native.MisError):
            native.mis_set_csr_range0(h, 2)
    finally:
        native.mis_destroy(h)


def test_zero_vertices():
    h = create((0, np.zeros(1, np.int32), np.zeros(0, np.int32)))
    try:
        got, st = gpu_solve(h, [1])
        assert len(got) == 0 and st.rounds == 0
    finally:
        native.mis_destroy(h)


def test_repeated_solves_reuse_workspace():
    g = graph("rmat14")
    h = create(g)
    try:
        for seed in range(10, 16):
            got, st = gpu_solve(h, [seed])
            assert_same(g, seed, got, st)
    finally:
        native.mis_destroy(h)


def test_host_api_matches():
    g = graph("er_10k")
    n, rp, col = g
    h = native.mis_create(n, rp, col)
    try:
        got = native.mis_solve(h, 1)
        st = native.mis_get_stats(h)
        assert_same(g, 1, got, st)
    finally:
        native.mis_destroy(h)


def test_device_input_create():
    import torch
    g = graph("grid")
    n, rp, col = g
    drp = torch.from_numpy(rp).cuda()
    dcol = torch.from_numpy(col).cuda()
    s = torch.cuda.current_stream().cuda_stream
    h = native.mis_create_ex(n, drp.data_ptr(), dcol.data_ptr(), 1, None, s)
    try:
        got, st = gpu_solve(h, [3])
        assert_same(g, 3, got, st)
    finally:
        native.mis_destroy(h)


BAD = {
    "asymmetric": (3, [0, 1, 1, 1], [1]),
    "self_loop": (2, [0, 2, 3], [0, 1, 0]),
    "unsorted": (3, [0, 2, 3, 4], [2, 1, 0, 0]),
    "duplicate": (2, [0, 2, 3], [1, 1, 0]),
    "out_of_range": (2, [0, 1, 2], [5, 0]),
    "negative_col": (2, [0, 1, 2], [-1, 0]),
    "rowptr_decreasing": (3, [0, 2, 1, 2], [1, 2]),
    "rowptr_start": (2, [1, 2, 2], [1, 0]),
}


@pytest.mark.parametrize("name", sorted(BAD))
def test_invalid_graph_rejected(name):
    n, rp, col = BAD[name]
    with pytest.raises(native.MisError) as ei:
        create((n, np.array(rp, np.int32), np.array(col, np.int32)))
    assert ei.value.code == native.MIS_EINVAL


def test_unchecked_symmetry_accepted_when_disabled():
    n, rp, col = BAD["asymmetric"]
    h = create((n, np.array(rp, np.int32), np.array(col, np.int32)), check_symmetry=0)
    native.mis_destroy(h)


def test_barrier_timeout_reports_error_and_recovers():
    # A spin limit of one poll makes a grid barrier give up almost surely:
    # the kernel must record MIS_ETIMEDOUT and return, leaving the context
    # usable for the next (normal) solve on the same graph.
    g = graph("rmat14")
    h = create(g, spin_cap=1)
    try:
        seen = False
        for _ in range(5):
            try:
                gpu_solve(h, [1])
            except native.MisError as e:
                assert e.code == native.MIS_ETIMEDOUT
                seen = True
                break
        assert seen
    finally:
        native.mis_destroy(h)
    h = create(g)
    try:
        got, st = gpu_solve(h, [1])
        assert_same(g, 1, got, st)
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("count", [1, 5, 64])
def test_batch_union_equals_standalone(count):
    parts = gg.batch_mixed(count, seed=100 + count, nmin=16, nmax=5000)
    parts[0] = gg.empty(0) if count > 2 else parts[0]
    h = native.mis_create_batch(parts)
    try:
        seeds = np.arange(1000, 1000 + count, dtype=np.uint64)
        keys = gpu_keys(h, seeds)
        for pending in (0, 1):
            native.mis_set_csr_pending(h, pending)
            got, st = gpu_solve(h, seeds)
            off = 0
            for g, s in zip(parts, seeds):
                n = g[0]
                assert np.array_equal(keys[off:off + n], oracle.keys(n, g[1], int(s)))
                want = oracle_solve(g, int(s))
                assert np.array_equal(got[off:off + n], want.status)
                off += n
            assert off == len(got)
    finally:
        native.mis_destroy(h)


def test_large_host_upload_checks_every_piece():
    """Host graphs of many arcs go up in pieces, each checked as it lands
    (symmetry check off): a defect in the last piece is still rejected, and
    a clean copy solves to a valid maximal independent set."""
    n, rp, col = gg.rmat(20, 16, 0.57, 0.19, 0.19, 41, permute=True)
    assert rp[-1] > (16 << 20)  # at least two pieces
    for kind in ("range", "self", "order"):
        bad = col.copy()
        v = int(np.searchsorted(rp, len(col) - 1, side="right") - 1)  # row of the last arc
        if kind == "range":
            bad[-1] = n
        elif kind == "self":
            bad[-1] = v
        else:
            bad[-1] = bad[-2] if rp[v + 1] - rp[v] >= 2 else bad[-1]
            if rp[v + 1] - rp[v] < 2:
                continue
        with pytest.raises(native.MisError):
            native.mis_create_ex(n, rp, bad, 0, native.options(check_symmetry=0), None)
    h = native.mis_create_ex(n, rp, col, 0, native.options(check_symmetry=0), None)
    try:
        got, st = gpu_solve(h, [5])
        assert oracle.check(n, rp, col, got) == (0, -1)
        assert st.mis_size == int(got.sum())
    finally:
        native.mis_destroy(h)
