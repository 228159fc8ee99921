"""The allocation-free entry point, xe_correlate_noalloc.

It exists for callers that cannot call cudaMalloc (a real-time pipeline that forbids
allocation once running, or a host application whose own pool owns all device memory): it
takes its scratch from a fixed array inside libxe.so.  This file checks, through the C ABI,
that two calls in a row give exactly the visibilities of the allocating entry point
(xe_correlate_async, same kernels: tolerance 0 for these exact integers), and that requests
beyond the fixed array are refused with a clear error.  It is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2005_09481_gb300 import synth

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_09481_gb300 import xe
    return xe.load()


def _vis(N, C):
    return torch.empty((C, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point_twice_in_a_row(lib):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(64, 1024, 1, 1), (300, 2000, 2, 2), (1100, 3000, 1, 3)]
    ins = [torch.from_numpy(synth.gauss_plane(N, T, C, seed=s)).cuda() for (N, T, C, s) in cases]
    got = [_vis(N, C) for (N, T, C, _) in cases]
    ref = [_vis(N, C) for (N, T, C, _) in cases]
    for (N, T, C, _), x, g in zip(cases, ins, got):     # calls back to back on one stream
        rc = lib.xe_correlate_noalloc(ctypes.c_void_p(x.data_ptr()), N, T, C,
                                      ctypes.c_void_p(g.data_ptr()), stream)
        assert rc == 0, lib.xe_last_error()
    for (N, T, C, _), x, r in zip(cases, ins, ref):
        rc = lib.xe_correlate_async(ctypes.c_void_p(x.data_ptr()), N, T, C,
                                    ctypes.c_void_p(r.data_ptr()), 1, stream)
        assert rc == 0, lib.xe_last_error()
    torch.cuda.synchronize()
    for g, r in zip(got, ref):
        assert torch.equal(g, r)
    # the first case is small enough to check against its closed-form size too
    assert got[0].shape == (1, 2080, 2)


@pytest.mark.gpu
def test_noalloc_refuses_sizes_beyond_the_fixed_scratch(lib):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    x = torch.zeros(16, dtype=torch.uint8, device="cuda")
    v = torch.zeros(16, dtype=torch.int32, device="cuda")
    for (N, T, C) in [(2048, 131072, 1), (2048, 4096, 3), (64, 131073, 1)]:
        rc = lib.xe_correlate_noalloc(ctypes.c_void_p(x.data_ptr()), N, T, C,
                                      ctypes.c_void_p(v.data_ptr()), stream)
        assert rc == -1
        assert b"noalloc" in lib.xe_last_error()
