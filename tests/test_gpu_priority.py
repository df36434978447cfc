"""The other priority heuristics of Sec. 3.3 on every path: H1 (random
priority hash(v)) and Eq. 1 discretised to 8 bits.  Keys and sets are
bit-identical to the oracle's for the same heuristic."""
import numpy as np
import pytest

import oracle
from paper_2605_29604_gb300 import graphgen as gg
from paper_2605_29604_gb300 import native

from gpu_util import assert_same, create, ensure_built, gpu_keys, gpu_solve

pytestmark = pytest.mark.gpu

MODES = [native.MIS_PRIORITY_HASH, native.MIS_PRIORITY_EQ1_Q8]


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
    "grid": lambda: gg.grid_diag(127, 0.05, 2),
    "star_hub": lambda: gg.disjoint_union([gg.star(150000), gg.er_gnm(5000, 20000, 3)]),
    "dense": lambda: gg.random_small(700, 0.3, 6),
    "k_ab": lambda: gg.complete_bipartite(40, 900),
    "path": lambda: gg.path(5001),
    "empty": lambda: gg.empty(1234),
}
_cache = {}


def graph(name):
    if name not in _cache:
        _cache[name] = FAMILIES[name]()
    return _cache[name]


def want(g, seed, mode):
    n, rp, col = g
    return oracle.solve(n, rp, col, seed, mode)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", sorted(FAMILIES))
def test_keys_bit_exact(name, mode):
    g = graph(name)
    h = create(g, priority=mode)
    try:
        got = gpu_keys(h, [21])
        assert np.array_equal(got, oracle.keys(g[0], g[1], 21, mode))
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("name", sorted(FAMILIES))
@pytest.mark.parametrize("path", ["csr0", "csr1", "csr_pending", "tile8", "tile_tc"])
def test_solve_bit_exact(name, mode, path):
    g = graph(name)
    h = create(g, priority=mode)
    try:
        if path == "tile8":
            native.mis_set_path(h, native.MIS_PATH_TILE, 8)
        elif path == "tile_tc":
            native.mis_set_path(h, native.MIS_PATH_TILE_TC, 16)
        else:
            native.mis_set_path(h, native.MIS_PATH_CSR, 1 if path == "csr1" else 0)
            native.mis_set_csr_pending(h, 1 if path == "csr_pending" else 0)
        for seed in (3, 2**40 + 1):
            got, st = gpu_solve(h, [seed])
            assert_same(g, seed, got, st, want=want(g, seed, mode))
            assert st.sure_in == 0 and st.sure_out == 0
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("mode", MODES)
def test_multi_seed(mode):
    import torch
    g = graph("rmat14")
    n = g[0]
    h = create(g, priority=mode)
    try:
        seeds = [4, 5, 6, 7]
        out = torch.full((4 * n,), 7, dtype=torch.uint8, device="cuda")
        native.mis_solve_multi_ex(h, np.asarray(seeds, dtype=np.uint64), out.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
        native.mis_get_stats(h)
        got = out.cpu().numpy().reshape(4, n)
        for s, row in zip(seeds, got):
            assert np.array_equal(row, want(g, s, mode).status)
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("mode", MODES)
def test_batch(mode):
    parts = gg.batch_mixed(16, seed=31, nmin=16, nmax=3000)
    h = native.mis_create_batch(parts, native.options(priority=mode))
    try:
        seeds = np.arange(40, 40 + len(parts), dtype=np.uint64)
        keys = gpu_keys(h, seeds)
        got, st = gpu_solve(h, seeds)
        off = 0
        for g, s in zip(parts, seeds):
            n = g[0]
            assert np.array_equal(keys[off:off + n], oracle.keys(n, g[1], int(s), mode))
            assert np.array_equal(got[off:off + n], want(g, int(s), mode).status)
            off += n
    finally:
        native.mis_destroy(h)


def test_bad_priority_rejected():
    g = graph("path")
    with pytest.raises(native.MisError):
        create(g, priority=3)
