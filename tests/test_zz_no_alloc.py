"""ans_window_quantities_noalloc: the allocation-free entry point.

It exists for callers that cannot allocate device memory while they run (a
process whose device memory is all owned by another framework's allocator, or
a latency-critical loop that cannot absorb cudaMalloc's synchronisation).  This
test calls it through the C ABI on calls in a row that reuse the same static
scratch -- a large window, a smaller one (stale contents from the first call
must not leak), the maximum size, a single packet and an empty window -- and
checks each result exactly against the CPU oracle and against the regular
entry point (ans_build_window).  It also checks the promise in the name: once
the first call has looked up the scratch array, further calls change neither
torch's allocated bytes nor the device's free memory.  It lives in a file that
pytest collects last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes
import gc

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_PACKETS = 65536


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _noalloc(lib, src, dst, n, out=None, status=True):
    if out is None:
        out = torch.zeros(9, dtype=torch.int64, device="cuda")
    st = torch.full((1,), 7, dtype=torch.int32, device="cuda") if status else None
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.ans_window_quantities_noalloc(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), n,
                                           ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(st.data_ptr() if st is not None else None),
                                           ctypes.c_void_p(stream))
    return rc, out, st


def test_noalloc_matches_oracle_and_build_window_on_consecutive_calls():
    from paper_2510_14050_gb300 import ans, synth
    lib = ans.load()
    ctx = ans.Context(0)
    try:
        sizes = [60000, 9000, MAX_PACKETS, 1, 0]
        w = synth.generate(5, sizes=sizes)
        for i, n in enumerate(sizes):
            s, d = w.window(i)
            ds, dd = _dev(s if n else [0]), _dev(d if n else [0])
            rc, out, status = _noalloc(lib, ds, dd, n)
            assert rc == ans.OK, lib.ans_last_error(None)
            torch.cuda.synchronize()
            got = ans.quantities_from_tensor(out)[0]
            assert got == oracle.window_quantities(s, d), f"call {i} (n={n}) against the oracle"
            m = ctx.build_window(ds, dd, n)
            assert got == m.quantities(), f"call {i} (n={n}) against ans_build_window"
            assert int(status.item()) == 0
            m.free()
    finally:
        ctx.close()


def test_noalloc_allocates_nothing():
    from paper_2510_14050_gb300 import ans, synth
    lib = ans.load()
    w = synth.generate(2, sizes=[MAX_PACKETS, 30000])
    wins = [(_dev(w.window(i)[0]), _dev(w.window(i)[1])) for i in range(2)]
    outs = [torch.zeros(9, dtype=torch.int64, device="cuda") for _ in range(2)]
    # the first call looks up the scratch array and loads the kernels
    rc, _, _ = _noalloc(lib, *wins[0], MAX_PACKETS, out=outs[0], status=False)
    assert rc == ans.OK
    # memory that earlier tests' objects still hold is released first, so that
    # only this call's behaviour is measured
    gc.collect()
    torch.cuda.synchronize()
    torch_bytes = torch.cuda.memory_allocated()
    free_before = torch.cuda.mem_get_info()[0]
    for (s, d), n, out in zip(wins, [MAX_PACKETS, 30000], outs):
        rc, _, _ = _noalloc(lib, s, d, n, out=out, status=False)  # d_status = NULL
        assert rc == ans.OK
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == torch_bytes
    assert torch.cuda.mem_get_info()[0] == free_before
    for i, out in enumerate(outs):
        assert ans.quantities_from_tensor(out)[0] == oracle.window_quantities(*w.window(i))


def test_noalloc_rejects_oversized_windows():
    from paper_2510_14050_gb300 import ans
    lib = ans.load()
    ds = _dev(np.zeros(MAX_PACKETS + 1, np.uint32))
    rc, _, _ = _noalloc(lib, ds, ds, MAX_PACKETS + 1)
    assert rc == ans.ERR_INVALID_ARG
    assert b"65536" in lib.ans_last_error(None)
