"""Streaming server: integrations equal one-shot correlations of the concatenated frames
(exactly), in every mix of channels; lost frames, admission by HBM budget, backpressure."""
import time

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


def frames_for(N, frame_T, n_frames, seed):
    return synth.gauss_plane(N, frame_T * n_frames, 1, seed=seed)[0].reshape(n_frames, frame_T, N)


def drain(st, want, timeout_s=20.0):
    out = []
    t0 = time.time()
    while len(out) < want and time.time() - t0 < timeout_s:
        r = st.poll(timeout_ms=100)
        if r is not None:
            out.append(r)
    assert len(out) == want, f"got {len(out)} of {want} integrations"
    return out


@pytest.mark.parametrize("device_source", [False, True])
def test_integrations_equal_oracle(xe, device_source):
    N, fT, F, C, n_int = 200, 1024, 4, 3, 2
    budget = 1 << 30
    with xe.Stream(N, fT, F * fT, max_chan=8, hbm_budget=budget, ring_frames=3,
                   device_source=device_source) as st:
        data = {}
        for c in range(C):
            assert st.admit(c) == 0
            data[c] = frames_for(N, fT, F * n_int, seed=100 + c)
        for k in range(F * n_int):
            for c in range(C):
                fr = torch.from_numpy(data[c][k])
                fr = fr.cuda() if device_source else fr
                while st.push(c, fr, k) == xe.XE_EAGAIN:
                    time.sleep(0.001)
        res = drain(st, C * n_int)
        # Every frame counts once, also when consecutive frames were merged into one job.
        assert st.stats()["frames"] == C * F * n_int
    for meta, vis in res:
        c, q = meta["chan"], meta["integ_index"]
        assert meta["complete"] == 1 and meta["n_samples"] == F * fT
        block = data[c][q * F:(q + 1) * F].reshape(1, F * fT, N)
        np.testing.assert_array_equal(vis, oracle.correlate_dense(block, N, F * fT, 1)[0])
        assert meta["t_ready_ns"] >= meta["t_last_arrival_ns"] >= meta["t_first_arrival_ns"]


def test_same_result_alone_and_in_the_mix(xe):
    # Channel 0's integrations are bit-identical whether it streams alone or among 12
    # channels whose frames are batched into the same persistent launches.
    N, fT, F = 256, 2048, 2
    mine = frames_for(N, fT, 2 * F, seed=7)

    def run(n_other):
        with xe.Stream(N, fT, F * fT, max_chan=16, hbm_budget=8 << 30, ring_frames=2) as st:
            for c in range(1 + n_other):
                assert st.admit(c) == 0
            others = {c: frames_for(N, fT, 2 * F, seed=200 + c) for c in range(1, 1 + n_other)}
            for k in range(2 * F):
                for c in range(1 + n_other):
                    fr = torch.from_numpy(mine[k] if c == 0 else others[c][k])
                    while st.push(c, fr, k) == xe.XE_EAGAIN:
                        time.sleep(0.0005)
            res = drain(st, 2 * (1 + n_other))
            return {m["integ_index"]: v for m, v in res if m["chan"] == 0}

    alone, mixed = run(0), run(11)
    assert alone.keys() == mixed.keys() == {0, 1}
    for q in (0, 1):
        np.testing.assert_array_equal(alone[q], mixed[q])


def test_lost_frame_marks_integration_incomplete(xe):
    N, fT, F = 130, 512, 4
    fr = frames_for(N, fT, 2 * F, seed=3)
    with xe.Stream(N, fT, F * fT, max_chan=2, hbm_budget=1 << 30, ring_frames=2) as st:
        assert st.admit(0) == 0
        for k in range(2 * F):
            if k == 2:
                continue                       # frame 2 never arrives
            while st.push(0, torch.from_numpy(fr[k]), k) == xe.XE_EAGAIN:
                time.sleep(0.001)
        res = sorted(drain(st, 2), key=lambda r: r[0]["integ_index"])
        assert st.stats()["dropped"] == 1
    (m0, v0), (m1, v1) = res
    assert m0["complete"] == 0 and m0["n_samples"] == 3 * fT
    got0 = np.concatenate([fr[0], fr[1], fr[3]])[None]
    np.testing.assert_array_equal(v0, oracle.correlate_dense(got0, N, 3 * fT, 1)[0])
    assert m1["complete"] == 1
    np.testing.assert_array_equal(v1, oracle.correlate_dense(fr[F:].reshape(1, F * fT, N), N, F * fT, 1)[0])


def test_admission_by_hbm_budget(xe):
    N, fT, F = 512, 4096, 2
    # 2 accumulators + ring + staging share (min(4, ring_frames) merged frames' operands)
    per_chan = 2 * N * (N + 1) * 4 + 2 * fT * N + 2 * (2 * 512 * fT)
    with xe.Stream(N, fT, F * fT, max_chan=8, hbm_budget=2 * per_chan + 1000, ring_frames=2) as st:
        assert st.admit(0) == 0 and st.admit(1) == 0
        assert st.admit(2) == xe.XE_EBUDGET
        st.evict(1)
        assert st.admit(2) == 0
        assert st.stats()["admitted"] == 2
    with pytest.raises(xe.XeError):
        xe.Stream(N, fT, F * fT, max_chan=8, hbm_budget=1000)


def test_push_errors_and_backpressure(xe):
    N, fT = 64, 256
    fr = torch.from_numpy(frames_for(N, fT, 1, seed=1)[0])
    with xe.Stream(N, fT, 4 * fT, max_chan=2, hbm_budget=1 << 28, ring_frames=2) as st:
        with pytest.raises(xe.XeError):
            st.push(1, fr, 0)                  # channel not admitted
        assert st.admit(0) == 0
        assert st.push(0, fr, 0) == 0
        with pytest.raises(xe.XeError):
            st.push(0, fr, 0)                  # duplicate sequence number
        st.flush()


def test_push_frames_batch_matches_single_pushes(xe):
    N, fT, F, C = 160, 512, 2, 5
    data = {c: frames_for(N, fT, 2 * F, seed=300 + c) for c in range(C)}
    with xe.Stream(N, fT, F * fT, max_chan=C, hbm_budget=1 << 30, ring_frames=3,
                   device_source=True) as st:
        for c in range(C):
            assert st.admit(c) == 0
        dev = {c: [torch.from_numpy(data[c][k]).cuda() for k in range(2 * F)] for c in range(C)}
        for k in range(2 * F):
            todo = list(range(C))
            while todo:
                rc = st.push_frames(todo, [dev[c][k] for c in todo], [k] * len(todo))
                todo = [c for c, r in zip(todo, rc) if r == xe.XE_EAGAIN]
                if todo:
                    time.sleep(0.001)
        res = drain(st, C * 2)
    for meta, vis in res:
        c, q = meta["chan"], meta["integ_index"]
        block = data[c][q * F:(q + 1) * F].reshape(1, F * fT, N)
        np.testing.assert_array_equal(vis, oracle.correlate_dense(block, N, F * fT, 1)[0])


def test_backlog_frames_merge_into_jobs_and_stay_exact(xe):
    # Eight frames of one channel pushed at once into a ring of eight: consecutive slots are
    # correlated as merged jobs (up to four frames each), across two integrations.
    N, fT, F = 320, 1024, 4
    fr = frames_for(N, fT, 2 * F, seed=77)
    dev = torch.from_numpy(fr).cuda()
    torch.cuda.synchronize()
    with xe.Stream(N, fT, F * fT, max_chan=1, hbm_budget=1 << 30, ring_frames=8, device_source=True) as st:
        assert st.admit(0) == 0
        for q in range(2 * F):
            assert st.push(0, dev[q], q) == 0
        st.flush()
        res = [st.poll(timeout_ms=20000) for _ in range(2)]
    for k, (meta, vis) in enumerate(res):
        assert meta["complete"] == 1 and meta["integ_index"] == k
        want = oracle.correlate_dense(fr[k * F:(k + 1) * F].reshape(1, F * fT, N), N, F * fT, 1)[0]
        np.testing.assert_array_equal(vis, want)


def test_ten_second_cadence_integration(xe):
    # The paper's export cadence: 10 s integrations (Table tab:data-flow), here 477 frames of
    # 8192 samples = 3,907,584 samples at 390625 samples/s.  Frames cycle through a few
    # distinct ones; by linearity in time the exact result is sum_d n_d V(frame_d).
    N, fT, F, D = 64, 8192, 477, 5
    fr = frames_for(N, fT, D, seed=99)
    dev = torch.from_numpy(fr).cuda()
    torch.cuda.synchronize()
    with xe.Stream(N, fT, F * fT, max_chan=1, hbm_budget=1 << 30, ring_frames=8, device_source=True) as st:
        assert st.admit(0) == 0
        q = 0
        t0 = time.time()
        while q < F and time.time() - t0 < 60:
            rc = st.push(0, dev[q % D], q)
            if rc == 0:
                q += 1
            else:
                assert rc == xe.XE_EAGAIN
                time.sleep(0.0005)
        assert q == F
        st.flush()
        meta, vis = st.poll(timeout_ms=30000)
    assert meta["complete"] == 1 and meta["n_samples"] == F * fT
    want = np.zeros((N * (N + 1) // 2, 2), np.int64)
    for d in range(D):
        n_d = len(range(d, F, D))
        want += n_d * oracle.correlate64(fr[d], N, fT, 1)[0]
    np.testing.assert_array_equal(vis, want)


def test_ten_second_cadence_extreme_values_fit_int32(xe):
    # All samples -8-8i for 10 s: Re V_ii = 128 * 3,907,584 = 500,170,752 < 2^31.
    N, fT, F = 32, 8192, 477
    frame = torch.from_numpy(synth.constant(N, fT, -8, -8)[0]).cuda()
    with xe.Stream(N, fT, F * fT, max_chan=1, hbm_budget=1 << 30, ring_frames=8, device_source=True) as st:
        assert st.admit(0) == 0
        q = 0
        while q < F:
            if st.push(0, frame, q) == 0:
                q += 1
            else:
                time.sleep(0.0005)
        st.flush()
        meta, vis = st.poll(timeout_ms=30000)
    diag = [i * N - i * (i - 1) // 2 for i in range(N)]
    assert np.all(vis[diag, 0] == 128 * F * fT) and np.all(vis[:, 1] == 0)
    assert np.all(vis[:, 0] == 128 * F * fT)


@pytest.mark.parametrize("implicit", [1, 0])
def test_implicit_plans_cover_every_tile_shape(xe, implicit):
    # The server's batches run whole tiles decoded in the kernel from the job table (option
    # implicit_plans 1) instead of host-built plans (0).  Inputs at the edges of the 128-row
    # blocks and 256-wide column tiles (half tiles, empty rows of full tiles, one input):
    # every integration equals the oracle either way, with channels of one shape batched.
    xe.set_option("implicit_plans", implicit)
    try:
        for N in (1, 17, 127, 128, 129, 255, 256, 257, 383, 385, 512, 640, 2048):
            fT, F, C = 128, 2, 3
            data = {c: frames_for(N, fT, F, seed=N * 10 + c) for c in range(C)}
            with xe.Stream(N, fT, F * fT, max_chan=C, hbm_budget=1 << 31, ring_frames=2,
                           device_source=True) as st:
                for c in range(C):
                    assert st.admit(c) == 0
                dev = {c: torch.from_numpy(data[c]).cuda() for c in range(C)}
                torch.cuda.synchronize()
                for k in range(F):
                    rc = st.push_frames(list(range(C)), [dev[c][k] for c in range(C)], [k] * C)
                    assert (rc == 0).all()
                st.flush()
                res = drain(st, C)
            for meta, vis in res:
                c = meta["chan"]
                want = oracle.correlate_dense(data[c].reshape(1, F * fT, N), N, F * fT, 1)[0]
                np.testing.assert_array_equal(vis, want, err_msg=f"N={N} chan {c}")
    finally:
        xe.set_option("implicit_plans", 1)


def wait_frames(st, n, timeout_s=20.0):
    t0 = time.time()
    while st.stats()["frames"] < n and time.time() - t0 < timeout_s:
        time.sleep(0.002)
    assert st.stats()["frames"] >= n


@pytest.mark.parametrize("device_source", [False, True])
def test_snapshot_restore_continues_an_integration(xe, device_source):
    # A checkpoint taken after 3 of 5 frames holds exactly those frames' sums; the stream it
    # came from goes on undisturbed, and a second stream restored from it completes the same
    # integration from frame 3 on: both equal the oracle of all 5 frames.
    N, fT, F = 136, 1024, 5
    data = frames_for(N, fT, F, seed=31)

    def push(st, k):
        fr = torch.from_numpy(data[k])
        fr = fr.cuda() if device_source else fr
        while st.push(2, fr, k) == xe.XE_EAGAIN:
            time.sleep(0.001)

    want_all = oracle.correlate_dense(data.reshape(1, F * fT, N), N, F * fT, 1)[0]
    with xe.Stream(N, fT, F * fT, max_chan=4, hbm_budget=1 << 30, ring_frames=3,
                   device_source=device_source) as st:
        assert st.admit(2) == 0
        info0, vis0 = st.snapshot(2)
        assert info0["frames"] == 0 and info0["next_seq"] == 0 and not vis0.any()
        for k in range(3):
            push(st, k)
        st.flush()
        wait_frames(st, 3)
        info, vis = st.snapshot(2)
        assert (info["integ_index"], info["next_seq"], info["frames"], info["n_samples"], info["lost"]) == \
            (0, 3, 3, 3 * fT, 0)
        np.testing.assert_array_equal(vis, oracle.correlate_dense(data[:3].reshape(1, 3 * fT, N), N, 3 * fT, 1)[0])
        for k in range(3, F):
            push(st, k)
        (meta, got), = drain(st, 1)
        assert meta["complete"] == 1
        np.testing.assert_array_equal(got, want_all)
        # After the close the channel's next integration is empty.
        info1, vis1 = st.snapshot(2)
        assert (info1["integ_index"], info1["frames"], info1["next_seq"]) == (1, 0, F) and not vis1.any()

    with xe.Stream(N, fT, F * fT, max_chan=4, hbm_budget=1 << 30, ring_frames=3,
                   device_source=device_source) as st2:
        assert st2.admit(2) == 0
        bad = dict(info, next_seq=info["next_seq"] + 1)
        with pytest.raises(xe.XeError) as e:
            st2.restore(2, bad, vis)
        assert e.value.code == xe.XE_EINVAL
        st2.restore(2, info, vis)
        with pytest.raises(xe.XeError) as e:            # a frame older than the checkpoint
            st2.push(2, torch.from_numpy(data[2]).cuda() if device_source else torch.from_numpy(data[2]), 2)
        assert e.value.code == xe.XE_EINVAL
        for k in range(3, F):
            push(st2, k)
        (meta, got), = drain(st2, 1)
        assert meta["integ_index"] == 0 and meta["complete"] == 1 and meta["n_samples"] == F * fT
        np.testing.assert_array_equal(got, want_all)
        with pytest.raises(xe.XeError) as e:            # the channel is no longer fresh
            st2.restore(2, info, vis)
        assert e.value.code == xe.XE_EINVAL


def test_snapshot_with_lost_frames_and_a_later_integration(xe):
    # A checkpoint inside the second integration, after a lost frame, restores onto a stream
    # whose channel then finishes that integration as incomplete with the right sums.
    N, fT, F = 64, 512, 4
    data = frames_for(N, fT, 2 * F, seed=47)
    with xe.Stream(N, fT, F * fT, max_chan=2, hbm_budget=1 << 30, ring_frames=2) as st:
        assert st.admit(0) == 0
        for k in (0, 1, 2, 3, 4, 6):                    # frame 5 never arrives
            while st.push(0, torch.from_numpy(data[k]), k) == xe.XE_EAGAIN:
                time.sleep(0.001)
        st.flush()
        (meta0, _), = drain(st, 1)
        wait_frames(st, 6)
        info, vis = st.snapshot(0)
    assert (info["integ_index"], info["frames"], info["n_samples"], info["lost"], info["next_seq"]) == \
        (1, 3, 2 * fT, 1, 7)
    with xe.Stream(N, fT, F * fT, max_chan=2, hbm_budget=1 << 30, ring_frames=2) as st2:
        assert st2.admit(1) == 0
        st2.restore(1, info, vis)
        while st2.push(1, torch.from_numpy(data[7]), 7) == xe.XE_EAGAIN:
            time.sleep(0.001)
        (meta, got), = drain(st2, 1)
    assert meta["integ_index"] == 1 and meta["complete"] == 0 and meta["n_samples"] == 3 * fT
    kept = np.concatenate([data[4], data[6], data[7]]).reshape(1, 3 * fT, N)
    np.testing.assert_array_equal(got, oracle.correlate_dense(kept, N, 3 * fT, 1)[0])


def test_rejected_admissions_are_counted(xe):
    from paper_2005_09481_gb300 import serve
    N, fT = 128, 1024
    per = serve.per_channel_bytes(N, fT, 2)
    with xe.Stream(N, fT, 2 * fT, max_chan=4, hbm_budget=2 * per, ring_frames=2) as st:
        assert st.admit(0) == 0 and st.admit(1) == 0
        assert st.admit(2) == xe.XE_EBUDGET and st.admit(3) == xe.XE_EBUDGET
        c = st.counters()
        assert c["admitted"] == 2 and c["rejected"] == 2
