"""GPU parity of the tile-CSR converter and the tile round kernels.

The converter is checked entry by entry against a tile-CSR built here with
numpy from the CSR; the tile kernels (CUDA-core popc, 8x8 and 16x16, and the
tensor-core exclusion test, 16x16) against the CPU oracle, bit-exact on the
vertex set and on the round structure of Algorithm 2.
"""
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


FAMILIES = {
    "er_10k": lambda: gg.er_10k_deg8(1),
    "rmat14": lambda: gg.rmat(14, 16, 0.57, 0.19, 0.19, 9, permute=True),
    "grid": lambda: gg.grid_diag(131, 0.05, 2),
    "grid_perm": lambda: gg.grid_diag(131, 0.05, 2, permute=True),
    "stencil27": lambda: gg.stencil27(23, 19, 17),  # ragged in every axis
    "rgg": lambda: gg.rgg(20001, 10.0, 3),
    "dense": lambda: gg.random_small(300, 0.5, 6),
    "star_hub": lambda: gg.disjoint_union([gg.star(40000), gg.er_gnm(5000, 20000, 3)]),
    "path_ragged": lambda: gg.path(1037),
    "complete": lambda: gg.complete(70),
    "empty": lambda: gg.empty(77),
    "single": lambda: gg.empty(1),
}
_cache = {}


def graph(name):
    if name not in _cache:
        _cache[name] = FAMILIES[name]()
    return _cache[name]


def numpy_tiles(n, rp, col, T):
    """Tile-CSR of a CSR graph, written directly from its definition."""
    nrb = (n + T - 1) // T
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    dst = col.astype(np.int64)
    key = (src // T) * nrb + dst // T
    order = np.argsort(key, kind="stable")
    key, src, dst = key[order], src[order], dst[order]
    uniq, first, inv = np.unique(key, return_index=True, return_inverse=True)
    words = T * T // 64
    bits = np.zeros((len(uniq), words), dtype=np.uint64)
    pos = (src % T) * T + dst % T
    np.bitwise_or.at(bits, (inv, pos // 64), np.left_shift(np.uint64(1), (pos % 64).astype(np.uint64)))
    rows = uniq // nrb
    trp = np.searchsorted(rows, np.arange(nrb + 1)).astype(np.int32)
    return trp, (uniq % nrb).astype(np.int32), bits.reshape(-1)


@pytest.mark.parametrize("name", ["er_10k", "rmat14", "grid", "grid_perm", "stencil27", "path_ragged", "empty"])
@pytest.mark.parametrize("T", [8, 16])
def test_converter_matches_definition(name, T):
    import torch
    g = graph(name)
    n, rp, col = g
    h = create(g)
    try:
        native.mis_set_path(h, native.MIS_PATH_TILE, T)
        st = native.mis_get_stats(h)
        want_trp, want_col, want_bits = numpy_tiles(n, rp, col, T)
        assert st.tile == T and st.ntiles == len(want_col)
        nrb = (n + T - 1) // T
        trp = torch.zeros(nrb + 1, dtype=torch.int32, device="cuda")
        tcol = torch.zeros(max(st.ntiles, 1), dtype=torch.int32, device="cuda")
        tbits = torch.zeros(max(st.ntiles * T * T // 64, 1), dtype=torch.int64, device="cuda")
        native.mis_tiles_ex(h, trp.data_ptr(), tcol.data_ptr(), tbits.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.array_equal(trp.cpu().numpy(), want_trp)
        assert np.array_equal(tcol.cpu().numpy()[:st.ntiles], want_col)
        got_bits = tbits.cpu().numpy().view(np.uint64)[:st.ntiles * T * T // 64]
        assert np.array_equal(got_bits, want_bits)
        # the bits hold exactly the arcs (no loss, no extras)
        assert int(sum(bin(int(x)).count("1") for x in got_bits)) == int(rp[-1])
    finally:
        native.mis_destroy(h)


PAYLOADS = [native.MIS_TILE_BITS, native.MIS_TILE_BITS_B1, native.MIS_TILE_INT8,
            native.MIS_TILE_FP16]


@pytest.mark.parametrize("name", ["er_10k", "rmat14", "grid", "grid_perm", "stencil27", "path_ragged", "empty",
                                  "complete"])
@pytest.mark.parametrize("payload", PAYLOADS)
def test_payload_matches_definition(name, payload):
    """Each payload form of the 16 x 16 tiles against the tile-CSR built here
    from the definition: the bitmask bit for bit, the int8 and fp16 forms
    entry by entry (1 exactly where the arc is, 0 elsewhere)."""
    import torch
    g = graph(name)
    n, rp, col = g
    h = create(g)
    try:
        native.mis_tile_payload_ex(h, payload, 0)
        st = native.mis_get_stats(h)
        _, _, bits = numpy_tiles(n, rp, col, 16)
        nt = st.ntiles
        assert nt == len(bits) // 4
        per = {native.MIS_TILE_INT8: 256, native.MIS_TILE_FP16: 512}.get(payload, 32)
        buf = torch.zeros(max(nt * per, 16), dtype=torch.uint8, device="cuda")
        native.mis_tile_payload_ex(h, payload, buf.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = buf.cpu().numpy()[:nt * per]
        # entry (t, i, j) of the definition
        ent = np.zeros((nt, 16, 16), dtype=np.uint8)
        w = bits.reshape(nt, 4)
        for i in range(16):
            row = (w[:, i // 4] >> np.uint64(16 * (i % 4))) & np.uint64(0xFFFF)
            for j in range(16):
                ent[:, i, j] = ((row >> np.uint64(j)) & np.uint64(1)).astype(np.uint8)
        if payload in (native.MIS_TILE_BITS, native.MIS_TILE_BITS_B1):
            assert np.array_equal(got.view(np.uint64), bits)
        elif payload == native.MIS_TILE_INT8:
            assert np.array_equal(got.reshape(nt, 16, 16), ent)
        else:
            halves = got.view(np.float16).reshape(nt, 16, 16)
            assert np.array_equal(halves, ent.astype(np.float16))
        assert int(ent.sum()) == int(rp[-1])
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("name", sorted(FAMILIES))
@pytest.mark.parametrize("payload", PAYLOADS)
def test_tile_tc_payloads_bit_exact(name, payload):
    """The tensor-core exclusion in every payload form."""
    g = graph(name)
    h = create(g)
    try:
        native.mis_set_tile_payload(h, payload)
        for seed in (1, 9):
            got, st = gpu_solve(h, [seed], native.MIS_PATH_TILE_TC, 16)
            assert st.path == native.MIS_PATH_TILE_TC and st.tile_payload == payload
            assert_same(g, seed, got, st)
    finally:
        native.mis_destroy(h)


@pytest.mark.parametrize("name", sorted(FAMILIES))
@pytest.mark.parametrize("path,T", [(native.MIS_PATH_TILE, 8), (native.MIS_PATH_TILE, 16),
                                    (native.MIS_PATH_TILE_TC, 16)])
def test_tile_solve_bit_exact(name, path, T):
    g = graph(name)
    h = create(g)
    try:
        for seed in (1, 9):
            got, st = gpu_solve(h, [seed], path, T)
            assert st.path == path and st.tile == T
            assert_same(g, seed, got, st)
    finally:
        native.mis_destroy(h)


def test_paths_agree_on_one_handle():
    g = graph("rgg")
    h = create(g)
    try:
        outs = []
        for path, p in [(native.MIS_PATH_CSR, 0), (native.MIS_PATH_TILE, 8),
                        (native.MIS_PATH_TILE_TC, 16), (native.MIS_PATH_TILE, 16),
                        (native.MIS_PATH_CSR, 4)]:
            got, st = gpu_solve(h, [3], path, p)
            outs.append(got)
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
    finally:
        native.mis_destroy(h)


def test_batch_on_tiles():
    parts = gg.batch_mixed(12, seed=5, nmin=16, nmax=3000)
    h = native.mis_create_batch(parts)
    try:
        seeds = np.arange(50, 62, dtype=np.uint64)
        for path, T in [(native.MIS_PATH_TILE, 8), (native.MIS_PATH_TILE_TC, 16)]:
            got, st = gpu_solve(h, seeds, path, T)
            off = 0
            import oracle
            for g, s in zip(parts, seeds):
                want = oracle.solve(g[0], g[1], g[2], int(s))
                assert np.array_equal(got[off:off + g[0]], want.status)
                off += g[0]
    finally:
        native.mis_destroy(h)


def test_tile_size_rejected():
    g = graph("er_10k")
    h = create(g)
    try:
        with pytest.raises(native.MisError):
            native.mis_set_path(h, native.MIS_PATH_TILE, 12)
        with pytest.raises(native.MisError):
            native.mis_set_path(h, native.MIS_PATH_TILE_TC, 8)
    finally:
        native.mis_destroy(h)
