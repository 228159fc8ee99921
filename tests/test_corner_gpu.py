"""Corner turn, pre-sums and the fused bundle-view correlation on the GPU, against the CPU
oracle (tolerance 0: bytes and integers).  Every call goes through the C ABI."""
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


@pytest.fixture(autouse=True)
def _default_options(xe):
    yield
    xe.set_option("exact_chunk_t", 131072)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def random_bundles(n_cyl, n_freq, n_in, T, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(n_cyl, T, n_freq, n_in)).astype(np.uint8)


@pytest.mark.parametrize("n_cyl,n_freq,n_in,T", [(4, 4, 512, 1000), (3, 2, 5, 77), (4, 1, 16, 33),
                                                 (2, 4, 64, 4096), (1, 1, 1, 1), (4, 4, 24, 300)])
def test_corner_turn_and_presums(xe, n_cyl, n_freq, n_in, T):
    b = random_bundles(n_cyl, n_freq, n_in, T, seed=n_in + T)
    frames, ps = xe.corner_turn(dev(b), n_cyl, n_freq, n_in, T)
    torch.cuda.synchronize()
    want = oracle.corner_turn(b, n_cyl, n_freq, n_in, T)
    assert np.array_equal(frames.cpu().numpy(), want)
    assert np.array_equal(ps.cpu().numpy(), oracle.presum(want, n_cyl * n_in, T, n_freq))


@pytest.mark.parametrize("n_cyl,n_freq,n_in,T", [(4, 4, 64, 1024), (3, 2, 20, 300), (4, 2, 128, 777)])
def test_bundle_view_correlation(xe, n_cyl, n_freq, n_in, T):
    # n_in = 20 is not a multiple of 16: the staging kernel's byte-load path.
    b = random_bundles(n_cyl, n_freq, n_in, T, seed=7 * T)
    vis = xe.correlate_bundles(dev(b), n_cyl, n_freq, n_in, T)
    torch.cuda.synchronize()
    xe.device_status()
    frames = oracle.corner_turn(b, n_cyl, n_freq, n_in, T)
    assert np.array_equal(vis.cpu().numpy(), oracle.correlate(frames, n_cyl * n_in, T, n_freq))


def test_bundle_view_windows(xe):
    # Several exact windows: the view's time offset t0 > 0.
    xe.set_option("exact_chunk_t", 256)
    n_cyl, n_freq, n_in, T = 4, 2, 64, 1000
    b = random_bundles(n_cyl, n_freq, n_in, T, seed=3)
    vis = xe.correlate_bundles(dev(b), n_cyl, n_freq, n_in, T)
    torch.cuda.synchronize()
    frames = oracle.corner_turn(b, n_cyl, n_freq, n_in, T)
    assert np.array_equal(vis.cpu().numpy(), oracle.correlate(frames, n_cyl * n_in, T, n_freq))


def test_plain_view_equals_plain_call(xe):
    N, T, C = 300, 500, 2
    p = synth.uniform(N, T, C, seed=11)
    v = xe.View(T * N, N, N, 0)
    got = xe.correlate_view(dev(p), v, N, T, C)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), oracle.correlate(p, N, T, C))


def test_full_array_from_chime_bundles(xe):
    # The CHIME node shape: 4 cylinders x 512 inputs, 4 frequencies (N = 2048).
    n_cyl, n_freq, n_in, T = 4, 4, 512, 8192
    frames = synth.gauss_plane(n_cyl * n_in, T, n_freq)
    b = synth.bundles_of(frames, n_cyl)
    d_b = dev(b)
    vis = xe.correlate_bundles(d_b, n_cyl, n_freq, n_in, T)
    fr, ps = xe.corner_turn(d_b, n_cyl, n_freq, n_in, T)
    torch.cuda.synchronize()
    xe.device_status()
    assert np.array_equal(fr.cpu().numpy(), frames)
    assert np.array_equal(vis.cpu().numpy(), oracle.correlate_dense(frames, n_cyl * n_in, T, n_freq))
    assert np.array_equal(ps.cpu().numpy(), oracle.presum(frames, n_cyl * n_in, T, n_freq))
