"""Phased-array beams on the GPU against the CPU oracle, element by element (tolerance 0:
the beams are exact integers).  Every call goes through the C ABI (xe_beamform)."""
import numpy as np
import pytest

import oracle
from paper_2005_09481_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_09481_gb300 import xe as _xe
    _xe.load()
    return _xe


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(xe, packed, w, N, T, C):
    y = xe.beamform(dev(packed), dev(w), N, T, C)
    torch.cuda.synchronize()
    xe.device_status()
    return y.cpu().numpy()


def check(xe, packed, w, N, T, C, B, dense=False):
    got = run(xe, packed, w, N, T, C)
    want = (oracle.beamform_dense if dense else oracle.beamform)(packed, w, N, T, C, B)
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{len(bad)} mismatches, first {bad[:4].tolist()}"


def test_ten_beams_small(xe):
    N, T, B = 64, 1024, 10
    check(xe, synth.uniform(N, T, 1), synth.beam_weights(B, N), N, T, 1, B)


@pytest.mark.parametrize("N,T,C,B", [(1, 1, 1, 1), (5, 127, 1, 3), (64, 128, 2, 8), (100, 129, 1, 10),
                                     (130, 300, 3, 16), (257, 1000, 1, 17), (48, 64, 1, 128),
                                     (1000, 515, 1, 33)])
def test_ragged_shapes(xe, N, T, C, B):
    # N % 16 != 0 takes the byte-load path; N % 64 != 0 ends inside a stage; T % 128 != 0
    # leaves a partial tile; B crosses the 16-column MMA granularity.
    p = synth.uniform(N, T, C, seed=N + 7 * T)
    w = synth.beam_weights(B, N, seed=B * N)
    check(xe, p, w, N, T, C, B)


def test_extreme_values_at_the_exactness_bound(xe):
    # x = -8-8i everywhere; weights (-128, 127) make every input contribute 2040 to Re and
    # 8 to Im: 8192 inputs reach 16,711,680 < 2^24 in one accumulation window.
    N, T, B = 8192, 256, 2
    p = synth.constant(N, T, -8, -8)
    w = np.zeros((B, N, 2), np.int8)
    w[0, :, 0], w[0, :, 1] = -128, 127
    w[1, :, 0], w[1, :, 1] = 127, -128
    check(xe, p, w, N, T, 1, B, dense=True)


def test_input_windows_beyond_8192(xe):
    # N > 8192: several exact windows add into the beams.
    N, T, B = 20000, 256, 4
    p = synth.uniform(N, T, 1, seed=3)
    check(xe, p, synth.beam_weights(B, N, seed=4), N, T, 1, B, dense=True)


def test_unaligned_input_pointer(xe):
    N, T, B = 256, 500, 10
    p = synth.uniform(N, T, 1, seed=5)
    buf = torch.zeros(p.size + 16, dtype=torch.uint8, device="cuda")
    view = buf[1:1 + p.size]
    view.copy_(dev(p.reshape(-1)))
    w = synth.beam_weights(B, N, seed=6)
    y = xe.beamform(view, dev(w), N, T, 1)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), oracle.beamform(p, w, N, T, 1, B))


def test_coherent_gain_on_gpu(xe):
    # A quarter-turn phase ramp undone by the weights: y = N s(t) exactly.
    N, T = 2048, 384
    rng = np.random.default_rng(1)
    s = rng.integers(-1, 2, size=(T, 2))
    unit = [1, 1j, -1, -1j]
    x = np.empty((T, N), np.complex128)
    for i in range(N):
        x[:, i] = (s[:, 0] + 1j * s[:, 1]) * unit[(3 * i) % 4]
    p = synth.pack(np.rint(x.real).astype(int), np.rint(x.imag).astype(int)).reshape(1, T, N)
    w = np.zeros((1, N, 2), np.int8)
    for i in range(N):
        u = unit[(-3 * i) % 4]
        w[0, i] = (int(u.real), int(u.imag))
    y = run(xe, p, w, N, T, 1)[0, :, 0]
    assert np.array_equal(y[:, 0], N * s[:, 0]) and np.array_equal(y[:, 1], N * s[:, 1])


def test_full_size_ten_beams(xe):
    # The pulsar workload at full size: N = 2048, T = 32768, 10 beams.
    N, T, B = 2048, 32768, 10
    p = synth.gauss_plane(N, T, 1)
    check(xe, p, synth.beam_weights(B, N), N, T, 1, B, dense=True)


def test_rejects_bad_arguments(xe):
    p = dev(synth.uniform(8, 8, 1))
    with pytest.raises(xe.XeError):
        xe.beamform(p, torch.zeros((129, 8, 2), dtype=torch.int8, device="cuda"), 8, 8, 1)
