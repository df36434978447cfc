"""Dynamic graphs: edge insertions and deletions of a resident graph
(mis_update_edges), and incremental repair of an MIS after them (mis_repair).
After an update every solve is bit-identical to the oracle's on the new
graph, and a repaired result to a full solve of the new graph."""
import numpy as np
import pytest

import oracle
from paper_2605_29604_gb300 import graphgen as gg
from paper_2605_29604_gb300 import native

from gpu_util import assert_same, create, ensure_built, gpu_solve

pytestmark = pytest.mark.gpu

HASH = native.MIS_PRIORITY_HASH


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    torch.cuda.set_device(0)


FAMILIES = {
    "rmat14": lambda: gg.rmat(14, 16, 0.57, 0.19, 0.19, 9, permute=True),
    "er_10k": lambda: gg.er_10k_deg8(1),
    "grid": lambda: gg.grid_diag(127, 0.05, 2),
    "star_hub": lambda: gg.disjoint_union([gg.star(20000), gg.er_gnm(5000, 20000, 3)]),
}


def edges_of(g):
    """Undirected edges (u < v) of a CSR as int64 codes u * n + v."""
    n, rp, col = g
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp.astype(np.int64)))
    keep = src < col
    return src[keep] * n + col[keep].astype(np.int64)


def apply_changes(g, ins, dels):
    """The graph with the pairs `dels` removed and `ins` added (numpy)."""
    n = g[0]
    def codes(p):
        p = np.asarray(p, dtype=np.int64).reshape(-1, 2)
        return np.minimum(p[:, 0], p[:, 1]) * n + np.maximum(p[:, 0], p[:, 1])
    e = np.setdiff1d(edges_of(g), codes(dels))
    e = np.union1d(e, codes(ins))
    return gg.from_edges(n, (e // n).astype(np.int32), (e % n).astype(np.int32))


def random_changes(g, k_ins, k_del, rng):
    """k_del existing edges and k_ins random pairs (existing or not), plus a
    deletion of a pair that is no edge (a no-op)."""
    n = g[0]
    e = edges_of(g)
    dels = e[rng.choice(len(e), size=min(k_del, len(e)), replace=False)] if len(e) else e
    dels = np.stack([dels // n, dels % n], axis=1)
    u = rng.integers(0, n, size=k_ins)
    v = (u + rng.integers(1, n, size=k_ins)) % n
    ins = np.stack([u, v], axis=1)
    a = rng.integers(0, n)
    b = (a + 1 + rng.integers(0, n - 1)) % n
    if (min(a, b) * n + max(a, b)) not in set(e.tolist()):
        dels = np.concatenate([dels, [[a, b]]])
    return ins.astype(np.int32), dels.astype(np.int32)


@pytest.mark.parametrize("priority", [native.MIS_PRIORITY_EQ1, HASH])
@pytest.mark.parametrize("name", sorted(FAMILIES))
def test_update_then_solve(name, priority):
    """After updates, solves (CSR path, both kernel forms) match the oracle on
    the new graph: rounds, alive sets and result."""
    rng = np.random.default_rng(7)
    g = FAMILIES[name]()
    h = create(g, priority=priority, order_rows=2)
    try:
        for step in range(3):
            ins, dels = random_changes(g, 50 + 400 * step, 50 + 400 * step, rng)
            native.mis_update_edges(h, ins, dels)
            g = apply_changes(g, ins, dels)
            for pending in (0, 1):
                native.mis_set_path(h, native.MIS_PATH_CSR, 0)
                native.mis_set_csr_pending(h, pending)
                got, st = gpu_solve(h, [11 + step])
                n, rp, col = g
                want = oracle.solve(n, rp, col, 11 + step, priority)
                assert_same(g, 11 + step, got, st, want=want)
    finally:
        native.mis_destroy(h)


def _device_solve(h, n, seed):
    import torch
    out = torch.full((max(n, 1),), 7, dtype=torch.uint8, device="cuda")
    native.mis_solve_ex(h, np.array([seed], dtype=np.uint64), out.data_ptr(),
                        torch.cuda.current_stream().cuda_stream)
    return out


@pytest.mark.parametrize("name", sorted(FAMILIES))
def test_repair_equals_full_solve(name):
    """A result repaired after each batch of changes equals a full solve of
    the new graph (the oracle's), for batches of deletions only, insertions
    only, both, and none."""
    import torch
    rng = np.random.default_rng(3)
    g = FAMILIES[name]()
    n = g[0]
    seed = 2**63 + 5
    h = create(g, priority=HASH)
    try:
        out = _device_solve(h, n, seed)
        plans = [(0, 30), (30, 0), (200, 200), (0, 0), (2000, 1500), (1, 1)]
        for k_ins, k_del in plans:
            ins, dels = random_changes(g, k_ins, k_del, rng)
            if k_del == 0:
                dels = dels[:0]
            native.mis_update_edges(h, ins, dels)
            g = apply_changes(g, ins, dels)
            changed = np.concatenate([ins, dels]) if len(ins) + len(dels) else ins
            size, rounds = native.mis_repair(h, seed, changed, out.data_ptr(),
                                             torch.cuda.current_stream().cuda_stream)
            got = out[:n].cpu().numpy()
            want = oracle.solve(g[0], g[1], g[2], seed, HASH)
            bad = np.flatnonzero(got != want.status)
            assert len(bad) == 0, f"{len(bad)} vertices differ, first {bad[:10]}"
            assert size == int(want.status.sum())
            assert (rounds == 0) == (len(changed) == 0)
    finally:
        native.mis_destroy(h)


def test_repair_isolates_and_reconnects():
    """Deleting every edge of a vertex isolates it (it goes in); inserting
    edges to a hub reconnects it."""
    import torch
    g = gg.disjoint_union([gg.star(300), gg.path(50)])
    n = g[0]
    seed = 9
    h = create(g, priority=HASH)
    try:
        out = _device_solve(h, n, seed)
        none = np.zeros((0, 2), dtype=np.int32)
        spokes = np.array([[0, j] for j in range(1, 300)], dtype=np.int32)
        links = np.array([[1, 2], [300, 5], [0, 320]], dtype=np.int32)
        for ins, dels in ((none, spokes), (links, none), (none, links)):
            native.mis_update_edges(h, ins, dels)
            g = apply_changes(g, ins, dels)
            native.mis_repair(h, seed, np.concatenate([ins, dels]), out.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
            want = oracle.solve(g[0], g[1], g[2], seed, HASH)
            assert np.array_equal(out[:n].cpu().numpy(), want.status)
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("priority", [native.MIS_PRIORITY_EQ1, HASH])
def test_add_vertices_then_connect(priority):
    """Added vertices are isolated (in); once connected by inserted edges, a
    solve -- and, with H1 keys, a repair of the grown result -- equals the
    oracle's on the grown graph."""
    import torch
    rng = np.random.default_rng(5)
    g = gg.rmat(12, 8, 0.57, 0.19, 0.19, 4, permute=True)
    n, rp, col = g
    seed = 77
    h = create(g, priority=priority)
    try:
        out = _device_solve(h, n, seed)
        k = 300
        native.mis_add_vertices(h, k)
        assert native.lib().mis_result_size(h) == n + k
        grown = (n + k, np.concatenate([rp, np.full(k, rp[-1], dtype=rp.dtype)]), col)
        got, st = gpu_solve(h, [seed])
        assert np.array_equal(got, oracle.solve(*grown, seed, priority).status)
        assert (got[n:] == 1).all()
        # connect every new vertex to two old ones and to the next new one
        new = np.arange(n, n + k)
        ins = np.concatenate([np.stack([new, rng.integers(0, n, k)], 1),
                              np.stack([new, rng.integers(0, n, k)], 1),
                              np.stack([new[:-1], new[1:]], 1)]).astype(np.int32)
        native.mis_update_edges(h, ins, ())
        g2 = apply_changes(grown, ins, np.zeros((0, 2), np.int32))
        want = oracle.solve(g2[0], g2[1], g2[2], seed, priority)
        got, st = gpu_solve(h, [seed])
        assert np.array_equal(got, want.status)
        if priority == HASH:
            buf = torch.ones(n + k, dtype=torch.uint8, device="cuda")
            buf[:n] = out[:n]
            native.mis_repair(h, seed, ins, buf.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
            assert np.array_equal(buf.cpu().numpy(), want.status)
    finally:
        native.mis_destroy(h)


def test_dynamic_rejects_bad_input():
    import torch
    g = gg.er_10k_deg8(1)
    n = g[0]
    h = create(g, priority=HASH)
    heq = create(g)
    try:
        out = _device_solve(h, n, 1)
        s = torch.cuda.current_stream().cuda_stream
        for bad in ([[3, 3]], [[-1, 4]], [[0, n]]):
            with pytest.raises(RuntimeError):
                native.mis_update_edges(h, bad, ())
            with pytest.raises(RuntimeError):
                native.mis_update_edges(h, (), bad)
            with pytest.raises(RuntimeError):
                native.mis_repair(h, 1, bad, out.data_ptr(), s)
        # Eq. 1 keys move with every edge change: no repair
        with pytest.raises(RuntimeError):
            native.mis_repair(heq, 1, [[0, 1]], out.data_ptr(), s)
        # a failed update leaves the graph as it was
        got, st = gpu_solve(h, [4])
        assert np.array_equal(got, oracle.solve(g[0], g[1], g[2], 4, HASH).status)
        torch.cuda.synchronize()
        # nor a graph with a captured solve, until the replay is destroyed
        r = native.mis_capture(h, [3], out.data_ptr())
        with pytest.raises(RuntimeError):
            native.mis_update_edges(h, [[0, 1]], ())
        native.mis_replay_destroy(r)
        native.mis_update_edges(h, [[0, 1]], ())
        # a batch cannot be updated
        b = native.mis_create_batch([g, g])
        try:
            with pytest.raises(RuntimeError):
                native.mis_update_edges(b, [[0, 1]], ())
            with pytest.raises(RuntimeError):
                native.mis_add_vertices(b, 3)
        finally:
            native.mis_destroy(b)
    finally:
        native.mis_destroy(h)
        native.mis_destroy(heq)
