"""Guard canaries around every output buffer (the stand-in for an out-of-bounds checker).

Each output is a view into a larger buffer whose words before and after it hold a sentinel;
after ragged-shape calls of every entry point that writes device (or host) memory, the
sentinels must be untouched and the outputs must equal the CPU oracle.  An out-of-bounds
store into a caching allocator's slack would pass the parity tests but fails here.  Outputs
sit at a 4096-byte offset and at an offset that is only as aligned as the entry point
requires (8 bytes for visibilities, 4 for counts, beams and pre-sums, 1 for frames).
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2005_09481_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SENT32 = 0x5A5A5A5A
SENT8 = 0x5A
GUARD = 1024            # sentinel words (or bytes) on each side


@pytest.fixture(scope="module")
def xe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_09481_gb300 import xe as m
    m.load()
    return m


class Guarded:
    """A view of n elements inside a sentinel-filled buffer, `off` extra elements in."""

    def __init__(self, n, dtype=torch.int32, off=0, device="cuda", pin=False):
        sent = SENT32 if dtype == torch.int32 else SENT8
        self.lo = GUARD + off
        self.n = n
        total = self.lo + n + GUARD
        if device == "cuda":
            self.buf = torch.full((total,), sent, dtype=dtype, device="cuda")
        else:
            self.buf = torch.full((total,), sent, dtype=dtype).pin_memory() if pin else \
                torch.full((total,), sent, dtype=dtype)
        self.sent = sent
        self.view = self.buf[self.lo:self.lo + n]

    def check(self):
        b = self.buf.cpu() if self.buf.is_cuda else self.buf
        head, tail = b[:self.lo], b[self.lo + self.n:]
        assert bool((head == self.sent).all()), "store before the output buffer"
        assert bool((tail == self.sent).all()), "store after the output buffer"


RAGGED = [(300, 1000, 2), (129, 640, 1), (17, 65, 3), (2048, 192, 1), (1, 1, 1)]


@pytest.mark.parametrize("algo", ["tc", "imma"])
@pytest.mark.parametrize("off", [0, 2])
def test_correlate_stays_inside_vis(xe, algo, off):
    for q, (N, T, C) in enumerate(RAGGED):
        p = synth.uniform(N, T, C, seed=700 + q)
        g = Guarded(C * N * (N + 1), off=off)
        xe.correlate(torch.from_numpy(p).cuda(), N, T, C, out=g.view.view(C, N * (N + 1) // 2, 2), algo=algo)
        torch.cuda.synchronize()
        xe.device_status()
        g.check()
        np.testing.assert_array_equal(g.view.cpu().numpy().reshape(C, -1, 2), oracle.correlate(p, N, T, C))


def test_batch_and_accumulate_stay_inside_vis(xe):
    shapes = [(300, 1000, 2), (129, 640, 1), (17, 65, 3), (520, 200, 1)]
    ins = [synth.uniform(N, T, C, seed=720 + q) for q, (N, T, C) in enumerate(shapes)]
    gs = [Guarded(C * N * (N + 1), off=2 * (q % 2)) for q, (N, T, C) in enumerate(shapes)]
    jobs = [(torch.from_numpy(p).cuda(), g.view.view(C, -1, 2), N, T, C)
            for p, g, (N, T, C) in zip(ins, gs, shapes)]
    xe.correlate_batch(jobs)
    xe.correlate_accumulate(jobs)
    torch.cuda.synchronize()
    xe.device_status()
    for p, g, (N, T, C) in zip(ins, gs, shapes):
        g.check()
        np.testing.assert_array_equal(g.view.cpu().numpy().reshape(C, -1, 2), 2 * oracle.correlate(p, N, T, C))


@pytest.mark.parametrize("off", [0, 1])
def test_masked_stays_inside_vis_and_counts(xe, off):
    for q, (N, T, C) in enumerate([(300, 1000, 2), (129, 640, 1), (17, 65, 3)]):
        p = synth.uniform(N, T, C, seed=740 + q)
        f = synth.flags(N, T, C, p_bad=0.1, seed=741 + q, burst=16)
        gv = Guarded(C * N * (N + 1), off=2 * off)
        gc = Guarded(C * N * (N + 1) // 2, off=off)
        xe.correlate_masked(torch.from_numpy(synth.to_offset_binary(p)).cuda(), torch.from_numpy(f).cuda(),
                            N, T, C, encoding="offset", out=gv.view.view(C, -1, 2), counts=gc.view.view(C, -1))
        torch.cuda.synchronize()
        xe.device_status()
        gv.check()
        gc.check()
        np.testing.assert_array_equal(gv.view.cpu().numpy().reshape(C, -1, 2), oracle.correlate_masked(p, f, N, T, C))
        np.testing.assert_array_equal(gc.view.cpu().numpy().reshape(C, -1), oracle.flag_counts(f, N, T, C))


@pytest.mark.parametrize("off", [0, 1])
def test_beamform_stays_inside_beams(xe, off):
    for q, (N, T, C, B) in enumerate([(300, 1000, 2, 10), (129, 130, 1, 3), (64, 128, 1, 65)]):
        p = synth.uniform(N, T, C, seed=760 + q)
        w = synth.beam_weights(B, N, seed=761 + q)
        g = Guarded(C * T * B * 2, off=off)
        xe.beamform(torch.from_numpy(p).cuda(), torch.from_numpy(w).cuda(), N, T, C, out=g.view.view(C, T, B, 2))
        torch.cuda.synchronize()
        xe.device_status()
        g.check()
        np.testing.assert_array_equal(g.view.cpu().numpy().reshape(C, T, B, 2), oracle.beamform(p, w, N, T, C, B))


@pytest.mark.parametrize("off", [0, 3])
def test_corner_turn_stays_inside_frames_and_presums(xe, off):
    L = xe.load()
    for (n_cyl, n_freq, n_in, T) in [(3, 2, 5, 9), (4, 4, 512, 300), (2, 3, 32, 257)]:
        N = n_cyl * n_in
        frames = synth.uniform(N, T, n_freq, seed=780 + T)
        bundles = synth.bundles_of(frames, n_cyl)
        gf = Guarded(n_freq * T * N, dtype=torch.uint8, off=off)
        gp = Guarded(n_freq * N * 2, off=off)
        b = torch.from_numpy(np.ascontiguousarray(bundles)).cuda()
        s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = L.xe_corner_turn(ctypes.c_void_p(b.data_ptr()), n_cyl, n_freq, n_in, T,
                              ctypes.c_void_p(gf.view.data_ptr()), ctypes.c_void_p(gp.view.data_ptr()), s)
        assert rc == 0, L.xe_last_error()
        torch.cuda.synchronize()
        gf.check()
        gp.check()
        np.testing.assert_array_equal(gf.view.cpu().numpy().reshape(n_freq, T, N), frames.reshape(n_freq, T, N))
        np.testing.assert_array_equal(gp.view.cpu().numpy().reshape(n_freq, N, 2), oracle.presum(frames, N, T, n_freq))


def test_host_entry_point_stays_inside_host_vis(xe):
    for q, (N, T, C) in enumerate([(300, 1000, 2), (17, 65, 3)]):
        p = synth.uniform(N, T, C, seed=800 + q)
        g = Guarded(C * N * (N + 1), off=2, device="cpu", pin=True)
        xe.correlate_host(torch.from_numpy(p), N, T, C, out=g.view.view(C, -1, 2))
        g.check()
        np.testing.assert_array_equal(g.view.numpy().reshape(C, -1, 2), oracle.correlate(p, N, T, C))


def test_noalloc_stays_inside_vis(xe):
    for q, (N, T, C) in enumerate([(300, 1000, 2), (17, 65, 3), (2048, 9000, 1)]):
        p = synth.uniform(N, T, C, seed=820 + q)
        g = Guarded(C * N * (N + 1), off=2)
        xe.correlate_noalloc(torch.from_numpy(p).cuda(), N, T, C, out=g.view.view(C, -1, 2))
        xe.noalloc_status()
        g.check()
        want = oracle.correlate_dense(p, N, T, C) if N > 256 else oracle.correlate(p, N, T, C)
        np.testing.assert_array_equal(g.view.cpu().numpy().reshape(C, -1, 2), want)
