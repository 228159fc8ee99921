"""Device-side descriptor checks (option "checks"): with the checks on, valid launches of
every kind stay bit-exact against the oracle, and corrupted descriptors (a test hook that
alters only values no kernel addresses through before the check has run) are reported as
XE_ECHECK with the outputs untouched; the next call on the same context is exact."""
import time

import numpy as np
import pytest

import oracle
from paper_2005_09481_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SENTINEL = 0x5A5A5A5A


@pytest.fixture(scope="module")
def xe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_09481_gb300 import xe as _xe
    _xe.load()
    return _xe


@pytest.fixture(autouse=True)
def _checks_off_after(xe):
    yield
    xe.set_option("check_corrupt", 0)
    xe.set_option("checks", 0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_valid_launches_pass_the_checks(xe):
    xe.set_option("checks", 1)
    # One call, two channels, ragged N and T.
    N, T, C = 300, 5000, 2
    p = synth.uniform(N, T, C, seed=11)
    out = xe.correlate(dev(p), N, T, C)
    xe.device_status()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.correlate_dense(p, N, T, C))
    # A batch of three shapes in one persistent launch, through a CUDA graph.
    shapes = [(64, 2048), (520, 3000), (256, 700)]
    ins = [synth.uniform(n, t, 1, seed=20 + k) for k, (n, t) in enumerate(shapes)]
    outs = [xe.empty_vis(n, 1) for n, _ in shapes]
    xe.correlate_batch([(dev(a), o, n, t, 1) for a, o, (n, t) in zip(ins, outs, shapes)], use_graph=True)
    xe.device_status()
    for a, o, (n, t) in zip(ins, outs, shapes):
        np.testing.assert_array_equal(o.cpu().numpy(), oracle.correlate_dense(a, n, t, 1))
    # Masked with counts: data and count launches, each checked.
    N, T = 200, 3000
    p = synth.uniform(N, T, 1, seed=5)
    f = synth.flags(N, T, 1, p_bad=0.1, seed=6)
    vis, cnt = xe.correlate_masked(dev(p), dev(f), N, T, 1)
    xe.device_status()
    np.testing.assert_array_equal(vis.cpu().numpy(), oracle.correlate_masked_dense(p, f, N, T, 1, 0))
    np.testing.assert_array_equal(cnt.cpu().numpy(), oracle.flag_counts_dense(f, N, T, 1))
    # Host buffers (copies inside the call).
    N, T = 128, 4096
    p = synth.uniform(N, T, 1, seed=8)
    got = xe.correlate_host(torch.from_numpy(p), N, T, 1)
    np.testing.assert_array_equal(got.numpy(), oracle.correlate_dense(p, N, T, 1))


def test_stream_batches_pass_the_checks(xe):
    # The streaming server's batches run implicit plans (tiles decoded in the kernel).
    xe.set_option("checks", 1)
    N, fT, F = 136, 1024, 2
    data = {c: synth.gauss_plane(N, F * fT, 1, seed=60 + c)[0].reshape(F, fT, N) for c in range(3)}
    with xe.Stream(N, fT, F * fT, max_chan=4, hbm_budget=1 << 30, ring_frames=2) as st:
        for c in range(3):
            assert st.admit(c) == 0
        for k in range(F):
            for c in range(3):
                while st.push(c, torch.from_numpy(data[c][k]), k) == xe.XE_EAGAIN:
                    time.sleep(0.001)
        got = []
        t0 = time.time()
        while len(got) < 3 and time.time() - t0 < 20:
            r = st.poll(timeout_ms=100)
            if r is not None:
                got.append(r)
    assert len(got) == 3
    for meta, vis in got:
        want = oracle.correlate_dense(data[meta["chan"]].reshape(1, F * fT, N), N, F * fT, 1)[0]
        np.testing.assert_array_equal(vis, want)


@pytest.mark.parametrize("corrupt", [1, 2])
def test_corrupt_descriptors_are_reported_and_nothing_is_written(xe, corrupt):
    N, T = 256, 2048
    p = synth.uniform(N, T, 1, seed=70 + corrupt)
    inp = dev(p)
    out = xe.empty_vis(N, 1)
    out.fill_(SENTINEL)
    xe.set_option("checks", 1)
    xe.set_option("check_corrupt", corrupt)
    xe.correlate(inp, N, T, 1, out=out)
    with pytest.raises(xe.XeError) as e:
        xe.device_status()
    assert e.value.code == xe.XE_ECHECK
    assert bool((out == SENTINEL).all())
    xe.set_option("check_corrupt", 0)
    xe.correlate(inp, N, T, 1, out=out)
    xe.device_status()
    np.testing.assert_array_equal(out.cpu().numpy(), oracle.correlate_dense(p, N, T, 1))
