"""The rule behind incremental repair, checked on the CPU against the oracle.

With fixed keys, Algorithm 2's result is the greedy MIS in priority order: v
is in exactly when no neighbour that outranks it is in.  So after edge
changes only the lower endpoint of a changed edge can change directly, and a
vertex that flips can only change the neighbours it outranks.  Re-deciding
the lower endpoints, then pass by pass the lower neighbours of every vertex
that flipped, until nothing flips, must give the oracle's full solve of the
new graph.  This plain-Python restatement of the passes (no GPU) is compared
with the oracle on random graphs and random batches of changes.
"""
import numpy as np
import pytest

import oracle
from paper_2605_29604_gb300 import graphgen as gg

HASH = oracle.PRIORITY_HASH


def _adj(n, rp, col):
    return [col[rp[v]:rp[v + 1]].tolist() for v in range(n)]


def _outranks(keys, u, v):
    return keys[u] > keys[v] or (keys[u] == keys[v] and u > v)


def repair(n, rp, col, keys, state, changed):
    """The passes of the repair, sequentially: returns the new states."""
    adj = _adj(n, rp, col)
    state = state.copy()
    todo = {b if _outranks(keys, a, b) else a for a, b in changed}
    while todo:
        # re-decide the listed vertices by the greedy rule, highest key first
        # (the rounds reach the same fixpoint; order only saves iterations)
        old = {v: state[v] for v in todo}
        for v in sorted(todo, key=lambda x: (keys[x], x), reverse=True):
            state[v] = 0 if any(state[u] and _outranks(keys, u, v) for u in adj[v]) else 1
        todo = {u for v in old if state[v] != old[v] for u in adj[v]
                if _outranks(keys, v, u)}
    return state


def hash_keys(n, seed):
    """H1 keys of every vertex, as the repair uses them.  The oracle gives an
    isolated vertex the largest key instead (it has no neighbour to compare
    with, so either choice gives the same result); keys taken on a cycle, where
    no vertex is isolated, are the seed hash of every id."""
    cn, crp, _ = gg.cycle(n)
    return oracle.keys(cn, crp, seed, HASH)


def _edit(n, rp, col, ins, dels):
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp.astype(np.int64)))
    keep = src < col
    e = set(zip(src[keep].tolist(), col[keep].tolist()))
    for a, b in dels:
        e.discard((min(a, b), max(a, b)))
    for a, b in ins:
        e.add((min(a, b), max(a, b)))
    e = sorted(e)
    u = np.array([x for x, _ in e], dtype=np.int32)
    v = np.array([y for _, y in e], dtype=np.int32)
    return gg.from_edges(n, u, v)


def _random_changes(rng, n, rp, col, k):
    src = np.repeat(np.arange(n), np.diff(rp))
    keep = np.flatnonzero(src < col)
    pick = rng.choice(keep, size=min(k, len(keep)), replace=False) if len(keep) else keep
    dels = [(int(src[p]), int(col[p])) for p in pick]
    ins = []
    while len(ins) < k:
        a, b = (int(x) for x in rng.integers(0, n, 2))
        if a != b:
            ins.append((a, b))
    return ins, dels


@pytest.mark.parametrize("family", ["er", "rmat", "grid", "star"])
def test_flip_propagation_equals_full_solve(family):
    rng = np.random.default_rng(11)
    make = {
        "er": lambda s: gg.er_gnm(300, 1200, s),
        "rmat": lambda s: gg.rmat(9, 8, 0.57, 0.19, 0.19, s, permute=True),
        "grid": lambda s: gg.grid_diag(17, 0.1, s),
        "star": lambda s: gg.disjoint_union([gg.star(60), gg.er_gnm(100, 300, s)]),
    }[family]
    for trial in range(6):
        n, rp, col = make(trial + 1)
        seed = 1000 + trial
        keys = hash_keys(n, seed)
        state = oracle.solve(n, rp, col, seed, HASH).status.astype(np.int64)
        for step in range(4):
            k = [1, 3, 20, 60][step]
            ins, dels = _random_changes(rng, n, rp, col, k)
            n2, rp2, col2 = _edit(n, rp, col, ins, dels)
            # keys depend on the seed and the id only (isolated vertices aside)
            live = np.diff(rp2) > 0
            assert np.array_equal(oracle.keys(n2, rp2, seed, HASH)[live], keys[live])
            got = repair(n2, rp2, col2, keys, state, ins + dels)
            want = oracle.solve(n2, rp2, col2, seed, HASH).status
            assert np.array_equal(got, want), (family, trial, step)
            n, rp, col, state = n2, rp2, col2, got


def test_only_the_lower_endpoint_is_seeded():
    """A changed edge seeds its lower endpoint; with no flip nothing else
    moves (an edge between two out vertices changes nothing)."""
    n, rp, col = gg.path(6)
    seed = 3
    keys = hash_keys(n, seed)
    state = oracle.solve(n, rp, col, seed, HASH).status.astype(np.int64)
    outs = [v for v in range(n) if state[v] == 0]
    a, b = outs[0], outs[-1]
    if a + 1 != b:  # a new edge between two out vertices
        n2, rp2, col2 = _edit(n, rp, col, [(a, b)], [])
        got = repair(n2, rp2, col2, keys, state, [(a, b)])
        assert np.array_equal(got, state)
        assert np.array_equal(got, oracle.solve(n2, rp2, col2, seed, HASH).status)
