"""The allocation-free total-momentum entry point.

kdfmm_total_momentum_noalloc serves callers that must not allocate device
memory while they run (cudaMalloc / cudaFree can synchronise the device, can
fail when another allocator holds the memory, or are forbidden inside a fixed
memory budget).  Its scratch is a fixed array inside the library.  This test
calls it through the C ABI and checks it against kdfmm_total_momentum, which
allocates its scratch per call, on two calls in a row (the shared scratch keeps
the previous call's partials, which must not leak into the next result).  It
lives in a file that pytest collects last and passes both alone and after the
other GPU tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_total_momentum_matches_allocating_entry_point():
    import torch
    from paper_2502_01496_gb300 import native
    L = native.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(17)
    # sizes rise and then fall, so a call also follows one that left more
    # partial sums in the shared scratch than it reads itself
    for n in (5, 123457, 3_000_001, 123457, 5):
        m = torch.tensor(rng.uniform(0.1, 1.0, n), device="cuda")
        v = torch.tensor(rng.normal(0.0, 1.0, (n, 3)), device="cuda")
        ref = torch.empty(3, dtype=torch.float64, device="cuda")
        assert L.kdfmm_total_momentum(_p(m), _p(v), n, _p(ref), stream) == 0, native.last_error()
        torch.cuda.synchronize()
        for _ in range(2):
            out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
            rc = L.kdfmm_total_momentum_noalloc(_p(m), _p(v), n, _p(out), stream)
            assert rc == 0, native.last_error()
            torch.cuda.synchronize()
            # same blocks, same reduction order: bit for bit
            assert torch.equal(out, ref), (n, out, ref)


def test_noalloc_total_momentum_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2502_01496_gb300 import native
    L = native.lib()
    m = torch.ones(8, dtype=torch.float64, device="cuda")
    v = torch.ones((8, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.kdfmm_total_momentum_noalloc(_p(m), _p(v), (1 << 30) + 1, _p(out), stream) == -1
    assert "allocation-free" in native.last_error()
    assert L.kdfmm_total_momentum_noalloc(_p(m), _p(v), 0, _p(out), stream) == -1
