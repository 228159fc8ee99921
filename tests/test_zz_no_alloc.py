"""The allocation-free entry point, xe_correlate_noalloc, and its status query.

It exists for callers that cannot call cudaMalloc (a real-time pipeline that forbids
allocation once running, or a host application whose own pool owns all device memory): it
takes its scratch from a fixed array inside libxe.so.  Through the C ABI, this file checks
that two calls in a row give exactly the visibilities of the CPU oracle and of the
allocating entry point (xe_correlate_async; tolerance 0 for these exact integers), up to the
full-array size (several windows of staged operands) and the most tiles the array admits;
that a timed-out call is reported by xe_noalloc_status even after a later call; and that
requests beyond the fixed array are refused with a clear error.  It is collected last on
purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2005_09481_gb300 import synth

torch = pytest.importorskip("torch")

XE_ETIMEOUT, XE_EINVAL, XE_EOVERFLOW = -6, -1, -2


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_09481_gb300 import xe
    return xe.load()


def _vis(N, C):
    return torch.empty((C, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _noalloc(lib, x, N, T, C, out):
    return lib.xe_correlate_noalloc(ctypes.c_void_p(x.data_ptr()), N, T, C,
                                    ctypes.c_void_p(out.data_ptr()), _stream())


@pytest.mark.gpu
def test_noalloc_matches_oracle_and_allocating_entry_point_twice_in_a_row(lib):
    # The last case is the full array: N=2048, T=32768 runs as five windows of staged
    # operands (4 x 8128 + 256 samples), each added into the visibilities.
    cases = [(64, 1024, 1, 1), (300, 2000, 2, 2), (1100, 3000, 1, 3), (2048, 32768, 1, 4)]
    host = [synth.gauss_plane(N, T, C, seed=s) for (N, T, C, s) in cases]
    want = [oracle.correlate_dense(h, N, T, C) for h, (N, T, C, _) in zip(host, cases)]
    ins = [torch.from_numpy(h).cuda() for h in host]
    ref = [_vis(N, C) for (N, T, C, _) in cases]
    for (N, T, C, _), x, r in zip(cases, ins, ref):
        rc = lib.xe_correlate_async(ctypes.c_void_p(x.data_ptr()), N, T, C,
                                    ctypes.c_void_p(r.data_ptr()), 1, _stream())
        assert rc == 0, lib.xe_last_error()
    for _ in range(2):                                   # two rounds of calls in a row
        got = [_vis(N, C) for (N, T, C, _) in cases]
        for (N, T, C, _), x, g in zip(cases, ins, got):
            assert _noalloc(lib, x, N, T, C, g) == 0, lib.xe_last_error()
        assert lib.xe_noalloc_status(_stream()) == 0, lib.xe_last_error()
        for g, r, w in zip(got, ref, want):
            assert torch.equal(g, r)
            np.testing.assert_array_equal(g.cpu().numpy(), w)


@pytest.mark.gpu
def test_noalloc_at_the_tile_limit(lib):
    # 56 channels of N=2048 are 4032 triangle tiles (at most 4096 fit the tile table): one
    # CTA per tile, several waves.
    N, T, C = 2048, 128, 56
    h = synth.uniform(N, T, C, seed=77)
    x = torch.from_numpy(h).cuda()
    g = _vis(N, C)
    assert _noalloc(lib, x, N, T, C, g) == 0, lib.xe_last_error()
    assert lib.xe_noalloc_status(_stream()) == 0, lib.xe_last_error()
    np.testing.assert_array_equal(g.cpu().numpy(), oracle.correlate_dense(h, N, T, C))


@pytest.mark.gpu
def test_noalloc_timeout_is_reported_after_a_later_call(lib):
    # The test hook makes the producer issue no copies, so the MMA warp's bounded wait runs
    # out (about a second).  A second call before the status query must not erase the
    # evidence; the query reports it once, and the next call is exact again.
    from paper_2005_09481_gb300 import xe
    N, T, C = 64, 1024, 1
    h = synth.uniform(N, T, C, seed=5)
    x = torch.from_numpy(h).cuda()
    g = _vis(N, C)
    xe.set_option("inject_stall", 1)
    assert _noalloc(lib, x, N, T, C, g) == 0, lib.xe_last_error()
    assert _noalloc(lib, x, N, T, C, g) == 0, lib.xe_last_error()
    assert lib.xe_noalloc_status(_stream()) == XE_ETIMEOUT
    assert b"earlier call" in lib.xe_last_error()
    assert lib.xe_noalloc_status(_stream()) == 0
    assert _noalloc(lib, x, N, T, C, g) == 0, lib.xe_last_error()
    assert lib.xe_noalloc_status(_stream()) == 0
    np.testing.assert_array_equal(g.cpu().numpy(), oracle.correlate(h, N, T, C))


@pytest.mark.gpu
def test_noalloc_refuses_sizes_beyond_the_fixed_scratch(lib):
    x = torch.zeros(16, dtype=torch.uint8, device="cuda")
    v = torch.zeros(16, dtype=torch.int32, device="cuda")
    for (N, T, C, code, what) in [(2048, 64, 200, XE_EINVAL, b"staged operands"),
                                  (16384, 64, 1, XE_EINVAL, b"tiles"),
                                  (64, 16777216, 1, XE_EOVERFLOW, b"XE_MAX_T")]:
        assert _noalloc(lib, x, N, T, C, v) == code
        assert what in lib.xe_last_error()
    assert lib.xe_noalloc_status(_stream()) == 0
