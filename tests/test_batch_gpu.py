"""Batched persistent launches: every job of a batch equals its solo launch and the oracle
(exactly), for uneven N and T, every schedule and tile width, CUDA-graph replay with fresh
pointers, the autotuner, and the full-size 16-channel and 64-instance workloads."""
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
def _reset(xe):
    yield
    for k, v in (("sched", -1), ("tile_n", 0), ("autotune", 0), ("n_cta", 0)):
        xe.set_option(k, v)


def make_batch(shapes, seed=0):
    host = [synth.uniform(N, T, C, seed=seed + 17 * q) for q, (N, T, C) in enumerate(shapes)]
    dev = [torch.from_numpy(h).cuda() for h in host]
    return host, dev


def run_batch(xe, shapes, dev, use_graph=False):
    outs = [xe.empty_vis(N, C) for (N, T, C) in shapes]
    xe.correlate_batch([(d, o, N, T, C) for d, o, (N, T, C) in zip(dev, outs, shapes)], use_graph=use_graph)
    torch.cuda.synchronize()
    xe.device_status()
    return [o.cpu().numpy() for o in outs]


UNEVEN = [(64, 100, 1), (200, 1000, 2), (256, 4096, 1), (512, 64, 3), (130, 3000, 1),
          (700, 777, 1), (1, 5, 2), (257, 2048, 1)]


def test_uneven_batch_equals_oracle_and_solo(xe):
    host, dev = make_batch(UNEVEN, seed=1)
    got = run_batch(xe, UNEVEN, dev)
    for (N, T, C), h, g, d in zip(UNEVEN, host, got, dev):
        np.testing.assert_array_equal(g, oracle.correlate_dense(h, N, T, C))
        solo = xe.correlate(d, N, T, C)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(g, solo.cpu().numpy())


@pytest.mark.parametrize("sched", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("tile_n", [128, 256])
def test_every_schedule_and_tile_width_is_exact(xe, sched, tile_n):
    shapes = [(300, 1000, 2), (520, 2000, 1), (64, 64, 1)]
    host, dev = make_batch(shapes, seed=2)
    xe.set_option("sched", sched)
    xe.set_option("tile_n", tile_n)
    got = run_batch(xe, shapes, dev)
    for (N, T, C), h, g in zip(shapes, host, got):
        np.testing.assert_array_equal(g, oracle.correlate_dense(h, N, T, C))


def test_graph_replay_with_new_pointers(xe):
    shapes = [(256, 2048, 2), (384, 1000, 1)]
    host_a, dev_a = make_batch(shapes, seed=3)
    host_b, dev_b = make_batch(shapes, seed=4)
    for host, dev in ((host_a, dev_a), (host_b, dev_b), (host_a, dev_a)):
        got = run_batch(xe, shapes, dev, use_graph=True)
        for (N, T, C), h, g in zip(shapes, host, got):
            np.testing.assert_array_equal(g, oracle.correlate_dense(h, N, T, C))


def test_autotune_picks_a_plan_and_stays_exact(xe):
    shapes = [(640, 4096, 3)]
    host, dev = make_batch(shapes, seed=5)
    xe.set_option("autotune", 1)
    got = run_batch(xe, shapes, dev)
    n_cta, tile_n, sched = xe.last_config()
    assert tile_n in (128, 256) and 0 <= sched <= 4 and n_cta > 0   # schedules 0..4 (xe_plan_dump)
    np.testing.assert_array_equal(got[0], oracle.correlate_dense(host[0], 640, 4096, 3))


def test_config3_sixteen_channels_batched(xe):
    # 16 channels x N=2048 x T=16384, quantised Gaussian + plane wave, one persistent launch
    # (channels as one 16-channel job, and as 16 jobs in a graph): every channel's full output
    # equals the oracle, and the two batch forms and per-channel solo launches agree.
    N, T, C = 2048, 16384, 16
    host = synth.gauss_plane(N, T, C)
    d = torch.from_numpy(host).cuda()
    out_a = xe.correlate(d, N, T, C)
    jobs = [(d[c], xe.empty_vis(N, 1), N, T, 1) for c in range(C)]
    xe.correlate_batch(jobs, use_graph=True)
    torch.cuda.synchronize()
    xe.device_status()
    a = out_a.cpu().numpy()
    for c in range(C):
        np.testing.assert_array_equal(a[c], oracle.correlate_dense(host[c], N, T, 1)[0])
        np.testing.assert_array_equal(jobs[c][1].cpu().numpy()[0], a[c])
    for c in (0, 7, 15):
        solo = xe.correlate(d[c].contiguous(), N, T, 1)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(a[c], solo.cpu().numpy()[0])


def test_config4_uneven_64_instances_batched(xe):
    # 64 instances, N in {256..2048}, T in {4096..65536} (seeded), one persistent launch:
    # every instance's full output equals the oracle and its own plain launch.
    shapes = synth.uneven_shapes(64)
    host = [synth.uniform(N, T, 1, seed=synth.BASE_SEED + 1 + q) for q, (N, T) in enumerate(shapes)]
    dev = [torch.from_numpy(h).cuda() for h in host]
    outs = [xe.empty_vis(N, 1) for (N, T) in shapes]
    xe.correlate_batch([(d, o, N, T, 1) for d, o, (N, T) in zip(dev, outs, shapes)])
    torch.cuda.synchronize()
    xe.device_status()
    for q, ((N, T), h, d, o) in enumerate(zip(shapes, host, dev, outs)):
        solo = xe.correlate(d, N, T, 1)
        torch.cuda.synchronize()
        g = o.cpu().numpy()
        np.testing.assert_array_equal(g, solo.cpu().numpy())
        np.testing.assert_array_equal(g, oracle.correlate_dense(h, N, T, 1))


def test_accumulate_adds_into_outputs(xe):
    shapes = [(300, 1000, 2), (520, 640, 1)]
    host_a, dev_a = make_batch(shapes, seed=8)
    host_b, dev_b = make_batch(shapes, seed=9)
    outs = [xe.empty_vis(N, C) for (N, T, C) in shapes]
    xe.correlate_batch([(d, o, N, T, C) for d, o, (N, T, C) in zip(dev_a, outs, shapes)])
    xe.correlate_accumulate([(d, o, N, T, C) for d, o, (N, T, C) in zip(dev_b, outs, shapes)])
    torch.cuda.synchronize()
    for (N, T, C), ha, hb, o in zip(shapes, host_a, host_b, outs):
        both = np.concatenate([ha, hb], axis=1)
        np.testing.assert_array_equal(o.cpu().numpy(), oracle.correlate_dense(both, N, 2 * T, C))


def test_later_launch_group_needing_more_scratch(xe):
    # More jobs than one launch holds: 208 small jobs, then 2 large ones.  The second launch
    # group needs more staging and workspace than the first; the scratch is sized for the
    # largest group before any launch record is bound to it.
    shapes = [(64, 64)] * 208 + [(1024, 4096), (2048, 2048)]
    ins = [synth.uniform(n, t, 1, seed=500 + q) for q, (n, t) in enumerate(shapes)]
    devs = [torch.from_numpy(p).cuda() for p in ins]
    outs = [xe.empty_vis(n, 1) for (n, t) in shapes]
    xe.correlate_batch([(d, o, n, t, 1) for d, o, (n, t) in zip(devs, outs, shapes)])
    torch.cuda.synchronize()
    xe.device_status()
    for q in (0, 207, 208, 209):
        n, t = shapes[q]
        want = oracle.correlate_dense(ins[q], n, t, 1) if n > 256 else oracle.correlate(ins[q], n, t, 1)
        np.testing.assert_array_equal(outs[q].cpu().numpy(), want)


def test_release_stream_frees_scratch_and_reallocates(xe):
    # Scratch is kept per stream; releasing it waits for the stream's work, and the next call
    # on the same stream allocates afresh and stays exact.
    N, T = 256, 4096
    p = synth.uniform(N, T, 1, seed=91)
    want = oracle.correlate_dense(p, N, T, 1)
    d = torch.from_numpy(p).cuda()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    for _ in range(2):
        with torch.cuda.stream(s):
            out = xe.empty_vis(N, 1)
            xe.correlate(d, N, T, 1, out=out, stream=s)
        xe.device_status(s)
        xe.release_stream(s)
        assert np.array_equal(out.cpu().numpy(), want)
    xe.release_stream(s)                    # nothing left to free: still XE_OK
