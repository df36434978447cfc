"""The autotuner: measured choice per density class, cached, result unchanged."""
import os

import numpy as np
import pytest

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


@pytest.mark.parametrize("name,make,dense", [
    ("grid", lambda: gg.grid_diag(300, 0.05, 2), True),
    ("grid_perm", lambda: gg.grid_diag(300, 0.05, 2, permute=True), False),
    ("rmat", lambda: gg.rmat(15, 16, 0.57, 0.19, 0.19, 4), False),
    ("er", lambda: gg.er_gnm(20000, 80000, 3), False),
])
def test_autotune_keeps_result(name, make, dense, tmp_path):
    os.environ["TCMIS_TUNE_CACHE"] = str(tmp_path / "tune.txt")
    g = make()
    h = create(g)
    try:
        t = native.mis_autotune(h, 2)
        assert t.candidates >= 7 and t.ms > 0
        if dense:
            assert t.arcs_per_tile > 3.0 and t.candidates >= 10
        else:
            assert t.arcs_per_tile < 2.5
        got, st = gpu_solve(h, [4])
        assert st.path == t.path
        assert_same(g, 4, got, st)
        lines = open(tmp_path / "tune.txt").read().split("\n")
        assert any(l.strip() for l in lines)
    finally:
        native.mis_destroy(h)
        del os.environ["TCMIS_TUNE_CACHE"]


def test_auto_create_uses_class_choice():
    g = gg.grid_diag(200, 0.05, 8)
    h = create(g)
    try:
        t = native.mis_autotune(h, 2)
    finally:
        native.mis_destroy(h)
    g2 = gg.grid_diag(201, 0.05, 9)  # same density class
    h2 = create(g2)  # default options: MIS_PATH_AUTO
    try:
        got, st = gpu_solve(h2, [2])
        assert st.path == t.path
        assert_same(g2, 2, got, st)
    finally:
        native.mis_destroy(h2)
