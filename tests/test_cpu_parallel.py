"""The second CPU baseline (OpenMP rounds, oracle/cpu_parallel.c) gives the
oracle's result, rounds and alive sets, at any thread count (CPU only)."""
import numpy as np
import pytest

import oracle
from paper_2605_29604_gb300 import graphgen as gg

GRAPHS = {
    "er": lambda: gg.er_gnm(3000, 15000, 5),
    "rmat": lambda: gg.rmat(12, 16, 0.57, 0.19, 0.19, 6, permute=True),
    "grid": lambda: gg.grid_diag(63, 0.05, 4),
    "star_union": lambda: gg.disjoint_union([gg.star(500), gg.path(40), gg.empty(7)]),
    "empty": lambda: gg.empty(10),
}


@pytest.mark.parametrize("threads", [1, 3, 0])
@pytest.mark.parametrize("priority", [oracle.PRIORITY_EQ1, oracle.PRIORITY_HASH])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_parallel_rounds_equal_oracle(name, priority, threads):
    n, rp, col = GRAPHS[name]()
    want = oracle.solve(n, rp, col, 17, priority)
    got = oracle.solve_parallel(n, rp, col, 17, priority, threads)
    assert np.array_equal(got.status, want.status)
    assert got.rounds == want.rounds
    assert got.alive_sum == want.alive_sum
    assert np.array_equal(got.alive_per_round, want.alive_per_round)


def test_thread_count_reported():
    assert oracle.parallel_threads() >= 1
