"""The 27-point stencil generator against its definition (brute force over
all vertex pairs) and the closed-form arc count.  The generator is input
plumbing shared by the oracle tests and the GPU tests; it holds none of the
method's arithmetic."""
import itertools

import numpy as np
import pytest

from paper_2605_29604_gb300 import graphgen as gg


def _brute(nx, ny, nz):
    n = nx * ny * nz
    coords = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]
    rows = []
    for i, (x, y, z) in enumerate(coords):
        row = [j for j, (a, b, c) in enumerate(coords)
               if j != i and abs(a - x) <= 1 and abs(b - y) <= 1 and abs(c - z) <= 1]
        rows.append(sorted(row))
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([u for r in rows for u in r], dtype=np.int64)
    return n, rp, col


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 1, 1), (1, 3, 1), (1, 1, 4), (3, 4, 5),
                                  (5, 3, 2), (4, 4, 4)])
def test_stencil27_matches_definition(dims):
    n, rp, col = gg.stencil27(*dims)
    bn, brp, bcol = _brute(*dims)
    assert n == bn
    assert np.array_equal(rp.astype(np.int64), brp)
    assert np.array_equal(col.astype(np.int64), bcol)


def test_stencil27_arc_count_closed_form():
    # each of the 13 forward offsets (dx, dy, dz) contributes
    # (nx - |dx|)(ny - |dy|)(nz - |dz|) edges, each stored as two arcs
    nx, ny, nz = 23, 19, 17
    n, rp, col = gg.stencil27(nx, ny, nz)
    want = 0
    for dx, dy, dz in itertools.product((-1, 0, 1), repeat=3):
        if (dx, dy, dz) != (0, 0, 0):
            want += (nx - abs(dx)) * (ny - abs(dy)) * (nz - abs(dz))
    assert int(rp[-1]) == want
    deg = np.diff(rp)
    assert deg.max() == 26 and deg.min() == 7
    # an interior vertex's row: the 26 ids at offsets dz*ny*nx + dy*nx + dx
    x, y, z = 5, 6, 7
    v = (z * ny + y) * nx + x
    offs = sorted(dz * ny * nx + dy * nx + dx
                  for dx, dy, dz in itertools.product((-1, 0, 1), repeat=3)
                  if (dx, dy, dz) != (0, 0, 0))
    assert list(col[rp[v]:rp[v + 1]]) == [v + o for o in offs]
