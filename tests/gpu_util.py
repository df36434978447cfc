"""Helpers for the GPU tests: run the library through its C ABI with device
buffers from PyTorch, and the CPU oracle beside it."""
import numpy as np

import oracle
from paper_2605_29604_gb300 import native


def ensure_built():
    from paper_2605_29604_gb300 import build as nbuild
    nbuild.build()
    native.lib()


def create(g, **opt):
    n, rp, col = g
    o = native.options(**opt)
    return native.mis_create_ex(n, rp, col, 0, o, None)


def gpu_solve(h, seeds, path=None, tpr=0):
    """Solve through mis_solve_ex (device output on the current torch stream);
    returns (status bytes, stats)."""
    import torch
    if path is not None:
        native.mis_set_path(h, path, tpr)
    size = native.lib().mis_result_size(h)
    out = torch.full((max(size, 1),), 7, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    native.mis_solve_ex(h, np.atleast_1d(np.asarray(seeds, dtype=np.uint64)), out.data_ptr(),
                        stream)
    st = native.mis_get_stats(h)
    return out[:size].cpu().numpy(), st


def gpu_keys(h, seeds):
    import torch
    size = native.lib().mis_result_size(h)
    out = torch.zeros(max(size, 1), dtype=torch.int64, device="cuda")  # 8-byte aligned
    k = torch.zeros(max(size, 1), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    native.mis_keys_ex(h, np.atleast_1d(np.asarray(seeds, dtype=np.uint64)), k.data_ptr(), stream)
    torch.cuda.synchronize()
    del out
    return k[:size].cpu().numpy().view(np.uint32)


def oracle_solve(g, seed):
    n, rp, col = g
    return oracle.solve(n, rp, col, seed)


def assert_same(g, seed, got, st, want=None):
    """Bit-exact result, plus the round structure of Algorithm 2."""
    n, rp, col = g
    want = want or oracle_solve(g, seed)
    assert got.dtype == np.uint8 and len(got) == n
    bad = np.flatnonzero(got != want.status)
    assert len(bad) == 0, f"{len(bad)} vertices differ, first {bad[:10]}"
    assert st.rounds == want.rounds
    r = min(want.rounds, 64)
    assert list(st.alive_per_round[:r]) == [int(x) for x in want.alive_per_round[:r]]
    assert st.alive_sum == want.alive_sum
    assert st.mis_size == int(want.status.sum())
    return want
