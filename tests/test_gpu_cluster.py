"""GPU parity of the thread-block-cluster solve (MIS_PATH_CLUSTER): vertex
words in distributed shared memory, cluster barriers between the phases of
Algorithm 2.  Bit-exact on the vertex set and on the round structure, for
graphs with one vertex per thread (rows cached in registers) and with
several vertices per thread (rows read from memory each round)."""
import numpy as np
import pytest

import oracle
from paper_2605_29604_gb300 import graphgen as gg
from paper_2605_29604_gb300 import native

from gpu_util import assert_same, create, ensure_built, gpu_solve

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
    "er_small": lambda: gg.er_gnm(3000, 12000, 4),
    "rmat14": lambda: gg.rmat(14, 16, 0.57, 0.19, 0.19, 9, permute=True),
    "grid": lambda: gg.grid_diag(127, 0.05, 2),
    "stencil27": lambda: gg.stencil27(23, 19, 17),  # ragged in every axis
    "rgg": lambda: gg.rgg(20000, 10.0, 3),
    "dense": lambda: gg.random_small(700, 0.3, 6),
    "star": lambda: gg.star(5000),
    "path": lambda: gg.path(5001),
    "cycle": lambda: gg.cycle(4099),
    "complete": lambda: gg.complete(300),
    "k_ab": lambda: gg.complete_bipartite(40, 900),
    "empty": lambda: gg.empty(1234),
    "single": lambda: gg.empty(1),
    "edge": lambda: gg.path(2),
    # several vertices per thread
    "rmat18": lambda: gg.rmat(18, 8, 0.57, 0.19, 0.19, 4, permute=True),
    "star_hub": lambda: gg.disjoint_union([gg.star(150000), gg.er_gnm(5000, 20000, 3)]),
    "er_300k": lambda: gg.er_gnm(300000, 1200000, 8),
}
_cache = {}


def graph(name):
    if name not in _cache:
        _cache[name] = FAMILIES[name]()
    return _cache[name]


@pytest.mark.parametrize("name", sorted(FAMILIES))
@pytest.mark.parametrize("priority", [0, 1, 2])
def test_cluster_solve_bit_exact(name, priority):
    g = graph(name)
    assert g[0] <= native.lib().mis_cluster_max_vertices()
    h = create(g, order_rows=0, priority=priority)
    try:
        for seed in (1, 2**63 + 3):
            want = oracle.solve(g[0], g[1], g[2], seed, priority)
            got, st = gpu_solve(h, [seed], native.MIS_PATH_CLUSTER, 0)
            assert st.path == native.MIS_PATH_CLUSTER
            assert_same(g, seed, got, st, want)
    finally:
        native.mis_destroy(h)


def test_cluster_limit_and_batch_rejected():
    limit = native.lib().mis_cluster_max_vertices()
    assert limit >= 131072
    g = gg.empty(limit + 1)
    h = create(g)
    try:
        with pytest.raises(native.MisError):
            native.mis_set_path(h, native.MIS_PATH_CLUSTER, 0)
    finally:
        native.mis_destroy(h)
    hb = native.mis_create_batch([gg.path(10), gg.path(20)])
    try:
        with pytest.raises(native.MisError):
            native.mis_set_path(hb, native.MIS_PATH_CLUSTER, 0)
    finally:
        native.mis_destroy(hb)


def test_cluster_solve_captured_and_replayed():
    import torch
    g = graph("er_10k")
    n = g[0]
    h = create(g, order_rows=0)
    try:
        native.mis_set_path(h, native.MIS_PATH_CLUSTER, 0)
        out = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        rep = native.mis_capture(h, [5], out.data_ptr())
        stream = torch.cuda.current_stream().cuda_stream
        for _ in range(3):
            out.fill_(7)
            native.mis_replay_launch(rep, stream)
            st = native.mis_get_stats(h)
            assert_same(g, 5, out.cpu().numpy(), st)
        native.mis_replay_destroy(rep)
    finally:
        native.mis_destroy(h)
