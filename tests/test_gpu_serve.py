"""Serving (continuous batching): mis_submit / mis_poll / mis_wait.

Each served result must equal the graph's standalone result (the CPU
oracle's, bit-exact), whether the request ran alone or among others that
were admitted while it was on the device.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2605_29604_gb300 import graphgen as gg
from paper_2605_29604_gb300 import native

from gpu_util import create, ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    torch.cuda.set_device(0)
    yield
    native.mis_serve_shutdown()


@pytest.fixture(scope="module")
def pool():
    graphs = [gg.er_gnm(300, 900, 1), gg.rmat(12, 8, 0.57, 0.19, 0.19, 2),
              gg.rgg(5000, 10.0, 3), gg.er_gnm(16000, 64000, 4),
              gg.rmat(15, 16, 0.57, 0.19, 0.19, 5), gg.grid_diag(150, 0.05, 6, permute=True),
              gg.er_gnm(40000, 400000, 7), gg.empty(33)]
    handles = [create(g) for g in graphs]
    yield graphs, handles
    for h in handles:
        native.mis_destroy(h)


def _want(g, seed):
    return oracle.solve(g[0], g[1], g[2], seed).status


def test_served_equals_standalone(pool):
    graphs, handles = pool
    reqs = []
    for k in range(48):
        i = (k * 5) % len(graphs)
        out = np.full(graphs[i][0], 9, dtype=np.uint8)
        t = native.mis_submit(handles[i], 100 + k, out)
        reqs.append((t, i, 100 + k, out))
    for t, i, seed, out in reqs:
        assert native.mis_wait(t, -1) == native.MIS_OK
        assert np.array_equal(out, _want(graphs[i], seed)), (i, seed)


def test_requests_join_while_others_run(pool):
    graphs, handles = pool
    first = []
    for k in range(10):
        i = 4 + (k % 3)  # the larger graphs
        out = np.empty(graphs[i][0], dtype=np.uint8)
        first.append((native.mis_submit(handles[i], 7 + k, out), i, 7 + k, out))
    time.sleep(0.0005)
    second = []
    for k in range(20):
        i = k % 4  # small graphs arriving while the large ones run
        out = np.empty(graphs[i][0], dtype=np.uint8)
        second.append((native.mis_submit(handles[i], 70 + k, out), i, 70 + k, out))
    for t, i, seed, out in first + second:
        assert native.mis_wait(t, -1) == native.MIS_OK
        assert np.array_equal(out, _want(graphs[i], seed))


def test_poll_and_ticket_release(pool):
    graphs, handles = pool
    out = np.empty(graphs[6][0], dtype=np.uint8)
    t = native.mis_submit(handles[6], 3, out)
    deadline = time.time() + 30
    rc, lat = native.mis_poll_ex(t)
    while rc == native.MIS_ENOTREADY and time.time() < deadline:
        time.sleep(0.0002)
        rc, lat = native.mis_poll_ex(t)
    assert rc == native.MIS_OK
    assert 0 < lat < 30e9
    assert np.array_equal(out, _want(graphs[6], 3))
    assert native.mis_poll(t) == native.MIS_EINVAL  # released
    assert native.mis_wait(123456789, 0) == native.MIS_EINVAL


def test_wait_with_timeout(pool):
    graphs, handles = pool
    out = np.empty(graphs[6][0], dtype=np.uint8)
    t = native.mis_submit(handles[6], 11, out)
    rc = native.mis_wait(t, 0)
    assert rc in (native.MIS_OK, native.MIS_ETIMEDOUT)
    if rc == native.MIS_ETIMEDOUT:
        assert native.mis_wait(t, -1) == native.MIS_OK
    assert np.array_equal(out, _want(graphs[6], 11))


def test_destroy_while_in_flight():
    g = gg.er_gnm(50000, 300000, 12)
    h = create(g)
    outs = []
    for k in range(4):
        out = np.empty(g[0], dtype=np.uint8)
        outs.append((native.mis_submit(h, k, out), k, out))
    native.mis_destroy(h)  # deferred until the requests retire
    for t, k, out in outs:
        assert native.mis_wait(t, -1) == native.MIS_OK
        assert np.array_equal(out, _want(g, k))


def test_small_budget_still_serves_everything(pool):
    graphs, handles = pool
    native.mis_serve_shutdown()
    native.mis_serve_configure(native.options(max_slots=3, hbm_budget=1 << 20))
    try:
        reqs = []
        for k in range(12):
            i = k % len(graphs)
            out = np.empty(graphs[i][0], dtype=np.uint8)
            reqs.append((native.mis_submit(handles[i], 500 + k, out), i, 500 + k, out))
        for t, i, seed, out in reqs:
            assert native.mis_wait(t, -1) == native.MIS_OK
            assert np.array_equal(out, _want(graphs[i], seed))
    finally:
        native.mis_serve_shutdown()
        native.mis_serve_configure(native.options())


def test_served_barrier_timeout_is_reported():
    # a graph above the one-block size runs on the cooperative grid; a spin
    # limit of one poll makes its barriers give up: the request must finish
    # with MIS_ETIMEDOUT and later requests must still be served
    g = gg.rmat(16, 16, 0.57, 0.19, 0.19, 3)
    h = create(g, spin_cap=1)
    try:
        seen = False
        for k in range(6):
            out = np.empty(g[0], dtype=np.uint8)
            rc = native.mis_wait(native.mis_submit(h, k, out), -1)
            assert rc in (native.MIS_OK, native.MIS_ETIMEDOUT)
            seen |= rc == native.MIS_ETIMEDOUT
            if seen:
                break
        assert seen
    finally:
        native.mis_destroy(h)
    g2 = gg.er_gnm(2000, 8000, 1)
    h2 = create(g2)
    try:
        out = np.empty(g2[0], dtype=np.uint8)
        assert native.mis_wait(native.mis_submit(h2, 5, out), -1) == native.MIS_OK
        assert np.array_equal(out, _want(g2, 5))
    finally:
        native.mis_destroy(h2)


def test_same_graph_requests_ride_together():
    """Requests queued on the same large graph are solved together (several
    seeds per launch); each result must still be its own seed's set, and a
    graph on the tile path (solved alone) must not be affected."""
    g = gg.rmat(15, 16, 0.57, 0.19, 0.19, 21)
    gt = gg.grid_diag(150, 0.05, 8)
    h = create(g)
    ht = create(gt)
    native.mis_set_path(ht, native.MIS_PATH_TILE, 8)
    try:
        reqs = []
        seeds = [1000 + k for k in range(20)] + [1003, 1003, 2**64 - 1, 0]
        for k, s in enumerate(seeds):
            out = np.full(g[0], 9, dtype=np.uint8)
            reqs.append((native.mis_submit(h, s, out), g, s, out))
            if k % 6 == 0:
                o2 = np.full(gt[0], 9, dtype=np.uint8)
                reqs.append((native.mis_submit(ht, s, o2), gt, s, o2))
        for t, gg_, s, out in reqs:
            assert native.mis_wait(t, -1) == native.MIS_OK
            assert np.array_equal(out, _want(gg_, s)), s
    finally:
        native.mis_destroy(h)
        native.mis_destroy(ht)
