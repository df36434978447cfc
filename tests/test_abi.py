"""The C-ABI library loads and exports every entry point include/tcmis.h declares.

CPU only: no call here touches a GPU.
"""
import ctypes
import os
import re

import pytest

from paper_2605_29604_gb300 import build as nbuild
from paper_2605_29604_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    nbuild.build()
    return native.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "tcmis.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(mis_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["mis_create", "mis_solve", "mis_submit", "mis_poll", "mis_destroy",
                     "mis_last_error", "mis_wait"]:
        assert required in names
    assert sorted(native.EXPORTED) == names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_options_defaults_and_version(lib):
    o = native.options()
    assert o.path == native.MIS_PATH_AUTO
    assert o.check_symmetry == 1
    assert o.build_tiles == -1
    assert b"sm_103a" in lib.mis_version()


def test_null_arguments_rejected_without_device(lib):
    # argument checks happen before any CUDA call
    assert lib.mis_solve(None, 1, None) == native.MIS_EINVAL
    code, msg = native.last_error()
    assert code == native.MIS_EINVAL and msg
    assert lib.mis_create_ex(-1, None, None, 0, None, None) is None
    assert native.last_error()[0] == native.MIS_EINVAL
    o = native.options(threads_per_row=8)
    assert lib.mis_create_ex(0, None, None, 0, ctypes.byref(o), None) is None
    assert native.last_error()[0] == native.MIS_EINVAL
    # the dynamic-graph entry points check their arguments first too
    assert lib.mis_update_edges(None, 0, None, 0, None, None) == native.MIS_EINVAL
    assert lib.mis_update_edges(None, -1, None, 0, None, None) == native.MIS_EINVAL
    assert lib.mis_repair(None, 1, 0, None, None, None, None, None) == native.MIS_EINVAL
    assert lib.mis_add_vertices(None, 1, None) == native.MIS_EINVAL
    assert native.last_error()[0] == native.MIS_EINVAL


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2605_29604_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "tcmis_oracle" not in text and "liboracle" not in text, f


def _header_fields(struct):
    text = open(os.path.join(ROOT, "include", "tcmis.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (struct, struct), text, flags=re.S)
    assert body, struct
    sizes = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
             "float": ctypes.c_float, "double": ctypes.c_double}
    out = []
    for ty, name, _, count in re.findall(
            r"(int32_t|int64_t|uint64_t|float|double)\s+(\w+)(\[(\d+)\])?;", body.group(1)):
        out.append((name, sizes[ty] * int(count) if count else sizes[ty]))
    return out


@pytest.mark.parametrize("struct", ["mis_options", "mis_stats", "mis_tuning"])
def test_binding_structs_match_the_header(struct):
    """The ctypes mirrors have the header's fields, in order, with its types
    (so offsets and sizes agree on every platform ctypes knows)."""
    want = _header_fields(struct)
    got = getattr(native, struct)._fields_
    assert [n for n, _ in got] == [n for n, _ in want]
    for (n, t), (_, w) in zip(got, want):
        assert ctypes.sizeof(t) == ctypes.sizeof(w), n
        assert getattr(t, "_type_", t) == getattr(w, "_type_", w), n
