"""The push/decrement form of the rounds (MIS_PATH_PUSH): same set, same
rounds and alive sets as Algorithm 2 (the oracle), on every graph family,
priority heuristic and batch."""
import numpy as np
import pytest

import oracle
from paper_2605_29604_gb300 import graphgen as gg
from paper_2605_29604_gb300 import native

from gpu_util import assert_same, create, ensure_built, gpu_solve, oracle_solve

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


@pytest.mark.parametrize("order_rows", [0, 1])
@pytest.mark.parametrize("name", sorted(FAMILIES))
def test_push_bit_exact(name, order_rows):
    g = graph(name)
    h = create(g, order_rows=order_rows)
    try:
        native.mis_set_path(h, native.MIS_PATH_PUSH, 0)
        for seed in (1, 7, 2**63 + 3):
            got, st = gpu_solve(h, [seed])
            assert st.path == native.MIS_PATH_PUSH
            assert_same(g, seed, got, st)
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("mode", [native.MIS_PRIORITY_HASH, native.MIS_PRIORITY_EQ1_Q8])
@pytest.mark.parametrize("name", ["rmat14", "grid", "dense", "star_hub"])
def test_push_other_heuristics(name, mode):
    g = graph(name)
    h = create(g, priority=mode)
    try:
        native.mis_set_path(h, native.MIS_PATH_PUSH, 0)
        got, st = gpu_solve(h, [5])
        assert_same(g, 5, got, st, want=oracle.solve(g[0], g[1], g[2], 5, mode))
    finally:
        native.mis_destroy(h)


def test_push_batch():
    parts = gg.batch_mixed(24, seed=61, nmin=16, nmax=5000)
    h = native.mis_create_batch(parts)
    try:
        native.mis_set_path(h, native.MIS_PATH_PUSH, 0)
        seeds = np.arange(70, 70 + len(parts), dtype=np.uint64)
        got, st = gpu_solve(h, seeds)
        off = 0
        for g, s in zip(parts, seeds):
            n = g[0]
            assert np.array_equal(got[off:off + n], oracle_solve(g, int(s)).status)
            off += n
    finally:
        native.mis_destroy(h)


def test_push_capture_replay():
    import torch
    g = graph("rmat14")
    h = create(g)
    rep = None
    try:
        native.mis_set_path(h, native.MIS_PATH_PUSH, 0)
        out = torch.full((g[0],), 7, dtype=torch.uint8, device="cuda")
        rep = native.mis_capture(h, [9], out.data_ptr())
        native.mis_replay_launch(rep, torch.cuda.current_stream().cuda_stream)
        st = native.mis_get_stats(h)
        assert_same(g, 9, out.cpu().numpy(), st)
    finally:
        if rep is not None:
            native.mis_replay_destroy(rep)
        native.mis_destroy(h)
