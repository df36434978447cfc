"""Captured solves (mis_capture / mis_replay_launch): every replay is a full
solve, bit-identical to the oracle, with the seeds fixed at capture time."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("path", ["csr", "csr_pending", "tile8", "tile_tc"])
def test_replay_equals_oracle(path):
    import torch
    g = gg.grid_diag(127, 0.05, 2) if path.startswith("tile") else gg.rmat(14, 16, 0.57, 0.19,
                                                                           0.19, 9, permute=True)
    h = create(g)
    rep = None
    try:
        if path == "csr_pending":
            native.mis_set_csr_pending(h, 1)
        elif path == "tile8":
            native.mis_set_path(h, native.MIS_PATH_TILE, 8)
        elif path == "tile_tc":
            native.mis_set_path(h, native.MIS_PATH_TILE_TC, 16)
        size = native.lib().mis_result_size(h)
        out = torch.full((size,), 7, dtype=torch.uint8, device="cuda")
        rep = native.mis_capture(h, [11], out.data_ptr())
        stream = torch.cuda.current_stream().cuda_stream
        for _ in range(3):
            out.fill_(7)
            native.mis_replay_launch(rep, stream)
            st = native.mis_get_stats(h)
            assert_same(g, 11, out.cpu().numpy(), st)
    finally:
        if rep is not None:
            native.mis_replay_destroy(rep)
        native.mis_destroy(h)


def test_replay_keeps_captured_seeds():
    """A plain solve with other seeds between replays does not change what a
    replay computes."""
    import torch
    g = gg.er_gnm(5000, 30000, 8)
    h = create(g)
    rep = None
    try:
        out = torch.zeros(g[0], dtype=torch.uint8, device="cuda")
        rep = native.mis_capture(h, [3], out.data_ptr())
        stream = torch.cuda.current_stream().cuda_stream
        got, st = gpu_solve(h, [4])
        assert_same(g, 4, got, st)
        native.mis_replay_launch(rep, stream)
        st = native.mis_get_stats(h)
        assert_same(g, 3, out.cpu().numpy(), st)
    finally:
        if rep is not None:
            native.mis_replay_destroy(rep)
        native.mis_destroy(h)


def test_batch_replay_equals_standalone():
    import torch
    parts = gg.batch_mixed(48, seed=77, nmin=16, nmax=4000)
    h = native.mis_create_batch(parts)
    rep = None
    try:
        seeds = np.arange(500, 500 + len(parts), dtype=np.uint64)
        size = native.lib().mis_result_size(h)
        out = torch.full((size,), 7, dtype=torch.uint8, device="cuda")
        rep = native.mis_capture(h, seeds, out.data_ptr())
        stream = torch.cuda.current_stream().cuda_stream
        for _ in range(2):
            out.fill_(7)
            native.mis_replay_launch(rep, stream)
            native.mis_get_stats(h)
            got = out.cpu().numpy()
            off = 0
            for g, s in zip(parts, seeds):
                n = g[0]
                assert np.array_equal(got[off:off + n], oracle_solve(g, int(s)).status)
                off += n
            assert off == size
    finally:
        if rep is not None:
            native.mis_replay_destroy(rep)
        native.mis_destroy(h)


def test_capture_rejects_null_arguments():
    h = create(gg.path(100))
    try:
        with pytest.raises(native.MisError):
            native.mis_capture(h, [1], 0)  # null output for a non-empty graph
    finally:
        native.mis_destroy(h)
    with pytest.raises(native.MisError):
        native.mis_replay_launch(None, None)
