"""A seeded sweep over shapes and forced planner options, full outputs against the CPU
oracle (tolerance 0).  Each case draws input counts and lengths at and around the tile and
k-block edges (128- and 256-input blocks, 64-sample blocks), a channel or job count, and a
schedule, tile width and CTA count, so that the combinations of whole tiles, k-splits,
exchanged parts, last-arriver sums, several segments per CTA and ragged edges are all met
together; some cases also take f16 operands or short exact windows (integrations split
into windows that add into the output).  Batches also add into their outputs
(correlate_accumulate).  Flag-masked calls (with and without counts, both encodings),
phased-array beams, streaming runs (ragged frames, lost frames), the corner turn with
bundle views, and the allocation-free and host-buffer entry points get their own sweeps.  Every call goes through the C ABI."""
import random

import numpy as np
import pytest

import oracle
from paper_2005_09481_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_EDGES = [1, 2, 31, 63, 64, 65, 127, 128, 129, 191, 255, 256, 257, 300, 383, 384, 385, 511, 512, 513, 640,
           767, 768, 769, 1023, 1025]
T_EDGES = [1, 7, 63, 64, 65, 127, 128, 129, 1000, 4095, 4096, 4097, 8191, 8192, 8193, 12000]
SCHEDS = [-1, 0, 1, 2, 3, 4]
TILES = [0, 128, 256]
CTAS = [0, 5, 37, 152, 300]
OPERAND_BYTES = [1, 1, 1, 2]
CHUNKS = [131072, 131072, 131072, 4096, 1024]


def _cases(seed, n, batch):
    rng = random.Random(seed)
    out = []
    for k in range(n):
        n_jobs = rng.randint(2, 4) if batch else 1
        jobs = []
        for _ in range(n_jobs):
            N, T = rng.choice(N_EDGES), rng.choice(T_EDGES)
            # keep the oracle's dense products small: at most 2.5e9 N^2 T per job
            while N * N * T > 2.5e9:
                T = max(1, T // 2)
            jobs.append((N, T, rng.randint(1, 3 if not batch else 2)))
        opts = (rng.choice(SCHEDS), rng.choice(TILES), rng.choice(CTAS), rng.choice(OPERAND_BYTES),
                rng.choice(CHUNKS))
        out.append(pytest.param(jobs, opts, k, id=f"{'b' if batch else 's'}{k}-" +
                                "+".join(f"{N}x{T}x{C}" for N, T, C in jobs) +
                                f"-sched{opts[0]}-tile{opts[1]}-cta{opts[2]}-eb{opts[3]}-win{opts[4]}"))
    return out


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
    xe.set_option("sched", -1)
    xe.set_option("tile_n", 0)
    xe.set_option("n_cta", 0)
    xe.set_option("operand_bytes", 1)
    xe.set_option("exact_chunk_t", 131072)
    xe.set_option("count_launch", 1)


def _set(xe, opts):
    sched, tile, cta, eb, chunk = opts
    xe.set_option("sched", sched)
    xe.set_option("tile_n", tile)
    xe.set_option("n_cta", cta)
    xe.set_option("operand_bytes", eb)
    xe.set_option("exact_chunk_t", chunk)


def _assert_exact(got, want, what):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        k = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {k}: got {got[k]} want {want[k]}")


@pytest.mark.parametrize("jobs,opts,k", _cases(20050948, 64, batch=False))
def test_single_calls(xe, jobs, opts, k):
    (N, T, C), = jobs
    p = synth.uniform(N, T, C, seed=1000 + k)
    _set(xe, opts)
    got = xe.correlate(torch.from_numpy(p).cuda(), N, T, C)
    torch.cuda.synchronize()
    xe.device_status()
    _assert_exact(got.cpu().numpy(), oracle.correlate_dense(p, N, T, C), f"{N}x{T}x{C} {opts}")


@pytest.mark.parametrize("jobs,opts,k", _cases(94810502, 24, batch=True))
def test_batches_and_accumulation(xe, jobs, opts, k):
    ps = [synth.uniform(N, T, C, seed=2000 + 10 * k + j) for j, (N, T, C) in enumerate(jobs)]
    ins = [torch.from_numpy(p).cuda() for p in ps]
    outs = [xe.empty_vis(N, C) for (N, T, C) in jobs]
    _set(xe, opts)
    xe.correlate_batch([(x, o, N, T, C) for x, o, (N, T, C) in zip(ins, outs, jobs)], use_graph=bool(k & 1))
    # then add the same visibilities once more: every output must read 2 V
    xe.correlate_accumulate([(x, o, N, T, C) for x, o, (N, T, C) in zip(ins, outs, jobs)])
    torch.cuda.synchronize()
    xe.device_status()
    for j, ((N, T, C), p, o) in enumerate(zip(jobs, ps, outs)):
        want = oracle.correlate_dense(p, N, T, C).astype(np.int64) * 2
        _assert_exact(o.cpu().numpy().astype(np.int64), want, f"job {j} {N}x{T}x{C} {opts}")


def _masked_cases(seed, n):
    rng = random.Random(seed)
    out = []
    for k in range(n):
        N, T = rng.choice(N_EDGES), rng.choice(T_EDGES)
        while N * N * T > 1.5e9:
            T = max(1, T // 2)
        C = rng.randint(1, 2)
        flags = rng.choice(["none", "sparse", "bursts", "half"])
        enc = rng.choice(["twos", "offset"])
        counts = rng.random() < 0.8
        opts = (rng.choice(SCHEDS), rng.choice(CTAS), rng.choice([0, 1]), rng.choice([131072, 131072, 4096]))
        out.append(pytest.param(N, T, C, flags, enc, counts, opts, k,
                                id=f"m{k}-{N}x{T}x{C}-{flags}-{enc}-{'counts' if counts else 'vis'}-"
                                   f"sched{opts[0]}-cta{opts[1]}-cl{opts[2]}-win{opts[3]}"))
    return out


@pytest.mark.parametrize("N,T,C,flags,enc,with_counts,opts,k", _masked_cases(27182818, 20))
def test_masked_calls(xe, N, T, C, flags, enc, with_counts, opts, k):
    # Every byte value (both encodings' extremes), four flag patterns, with and without
    # counts, under forced schedules, CTA counts, count-launch modes and exact windows.
    rs = np.random.default_rng(3000 + k)
    p = rs.integers(0, 256, size=(C, T, N), dtype=np.uint8)
    if flags == "none":
        f = None
    elif flags == "half":
        f = synth.flags(N, T, C, p_bad=0.5, seed=3000 + k)
    else:
        f = synth.flags(N, T, C, p_bad=0.02, seed=3000 + k, burst=256 if flags == "bursts" else 0)
    sched, cta, count_launch, chunk = opts
    xe.set_option("sched", sched)
    xe.set_option("n_cta", cta)
    xe.set_option("count_launch", count_launch)
    xe.set_option("exact_chunk_t", chunk)
    try:
        vis, cnt = xe.correlate_masked(torch.from_numpy(p).cuda(), None if f is None else torch.from_numpy(f).cuda(),
                                       N, T, C, encoding=enc, with_counts=with_counts)
        torch.cuda.synchronize()
        xe.device_status()
    finally:
        xe.set_option("count_launch", 1)
    e = 1 if enc == "offset" else 0
    _assert_exact(vis.cpu().numpy(), oracle.correlate_masked_dense(p, f, N, T, C, encoding=e), f"vis {N}x{T}x{C}")
    if with_counts:
        if f is None:
            want = np.full((C, oracle.n_baselines(N)), T, np.int64)
        else:
            want = oracle.flag_counts_dense(f, N, T, C)
        _assert_exact(cnt.cpu().numpy().astype(np.int64), want, f"counts {N}x{T}x{C}")


def _beam_cases(seed, n):
    rng = random.Random(seed)
    out = []
    for k in range(n):
        N, T = rng.choice(N_EDGES), rng.choice(T_EDGES)
        B = rng.choice([1, 3, 10, 16, 17, 33, 64, 65, 100, 128])
        while N * T * B > 4e8:
            T = max(1, T // 2)
        C = rng.randint(1, 2)
        out.append(pytest.param(N, T, C, B, k, id=f"y{k}-{N}x{T}x{C}-B{B}"))
    return out


@pytest.mark.parametrize("N,T,C,B,k", _beam_cases(16180339, 16))
def test_beam_calls(xe, N, T, C, B, k):
    # Every byte value and every int8 weight, -128 included; ragged and unaligned input
    # counts (byte-load path), ragged sample tiles, beams in one or several launches.
    rs = np.random.default_rng(4000 + k)
    p = rs.integers(0, 256, size=(C, T, N), dtype=np.uint8)
    w = rs.integers(-128, 128, size=(B, N, 2), dtype=np.int8)
    got = xe.beamform(torch.from_numpy(p).cuda(), torch.from_numpy(w).cuda(), N, T, C)
    torch.cuda.synchronize()
    xe.device_status()
    _assert_exact(got.cpu().numpy().astype(np.int64), oracle.beamform_dense(p, w, N, T, C, B),
                  f"beams {N}x{T}x{C} B={B}")


def _stream_cases(seed, n):
    rng = random.Random(seed)
    out = []
    for k in range(n):
        N = rng.choice([1, 63, 130, 257, 384, 513])
        fT = rng.choice([37, 64, 100, 512, 777, 1024, 2048])
        F = rng.choice([1, 2, 3, 4, 5, 8])
        while N * N * F * fT > 1e9:
            fT = max(1, fT // 2)
        n_int = rng.randint(1, 3)
        C = rng.randint(1, max(1, min(10, 12 // n_int)))
        ring = rng.randint(2, 6)
        dev = rng.random() < 0.5
        out.append(pytest.param(N, fT, F, n_int, C, ring, dev, k,
                                id=f"st{k}-N{N}-frame{fT}x{F}-int{n_int}-ch{C}-ring{ring}-{'dev' if dev else 'host'}"))
    return out


@pytest.mark.parametrize("N,fT,F,n_int,C,ring,dev,k", _stream_cases(31415926, 10))
def test_stream_runs(xe, N, fT, F, n_int, C, ring, dev, k):
    # Ragged frame lengths, 1 to 8 frames per integration, several channels pushed in a
    # shuffled order every tick, and about 8 % of the frames lost (never a channel's last,
    # whose loss only a later frame would reveal): every integration equals the oracle over
    # the frames it received, with its sample count and completeness.
    import time
    rng = random.Random(k)
    n_frames = F * n_int
    data = {c: synth.uniform(N, fT * n_frames, 1, seed=5000 + 10 * k + c)[0].reshape(n_frames, fT, N)
            for c in range(C)}
    lost = {(c, q) for c in range(C) for q in range(n_frames - 1) if rng.random() < 0.08}
    with xe.Stream(N, fT, F * fT, max_chan=16, hbm_budget=8 << 30, ring_frames=ring, device_source=dev) as st:
        for c in range(C):
            assert st.admit(c) == 0
        for q in range(n_frames):
            order = list(range(C))
            rng.shuffle(order)
            for c in order:
                if (c, q) in lost:
                    continue
                fr = torch.from_numpy(np.ascontiguousarray(data[c][q]))
                fr = fr.cuda() if dev else fr
                t0 = time.time()
                while st.push(c, fr, q) == xe.XE_EAGAIN:
                    assert time.time() - t0 < 20, "push kept returning XE_EAGAIN"
                    time.sleep(0.0005)
        res = []
        t0 = time.time()
        while len(res) < C * n_int and time.time() - t0 < 30:
            r = st.poll(timeout_ms=100)
            if r is not None:
                res.append(r)
        assert len(res) == C * n_int, f"got {len(res)} of {C * n_int} integrations"
        assert st.stats()["dropped"] == len(lost)
    for meta, vis in res:
        c, g = meta["chan"], meta["integ_index"]
        got_frames = [q for q in range(g * F, (g + 1) * F) if (c, q) not in lost]
        assert meta["n_samples"] == len(got_frames) * fT
        assert meta["complete"] == (1 if len(got_frames) == F else 0)
        if got_frames:
            block = np.concatenate([data[c][q] for q in got_frames])[None]
            want = oracle.correlate_dense(block, N, len(got_frames) * fT, 1)[0]
        else:
            want = np.zeros((oracle.n_baselines(N), 2), np.int32)
        _assert_exact(vis, want, f"chan {c} integration {g}")


def _corner_cases(seed, n):
    rng = random.Random(seed)
    out = []
    for k in range(n):
        n_cyl, n_freq = rng.randint(1, 4), rng.randint(1, 4)
        n_in = rng.choice([1, 5, 16, 20, 64, 100, 128, 256])
        T = rng.choice(T_EDGES)
        while (n_cyl * n_in) ** 2 * T * n_freq > 1.5e9:
            T = max(1, T // 2)
        win = rng.choice([131072, 131072, 1024])
        out.append(pytest.param(n_cyl, n_freq, n_in, T, win, k,
                                id=f"ct{k}-cyl{n_cyl}-freq{n_freq}-in{n_in}-T{T}-win{win}"))
    return out


@pytest.mark.parametrize("n_cyl,n_freq,n_in,T,win,k", _corner_cases(14142135, 12))
def test_corner_turn_and_bundle_views(xe, n_cyl, n_freq, n_in, T, win, k):
    # The corner turn with pre-sums, and the correlation read straight from the bundles
    # through an input view (with exact windows, so views with a time offset), both against
    # the oracle's corner turn.
    rs = np.random.default_rng(6000 + k)
    b = rs.integers(0, 256, size=(n_cyl, T, n_freq, n_in), dtype=np.uint8)
    bd = torch.from_numpy(b).cuda()
    N = n_cyl * n_in
    frames, ps = xe.corner_turn(bd, n_cyl, n_freq, n_in, T)
    xe.set_option("exact_chunk_t", win)
    vis = xe.correlate_bundles(bd, n_cyl, n_freq, n_in, T)
    torch.cuda.synchronize()
    xe.device_status()
    want = oracle.corner_turn(b, n_cyl, n_freq, n_in, T)
    _assert_exact(frames.cpu().numpy(), want, "frames")
    _assert_exact(ps.cpu().numpy(), oracle.presum(want, N, T, n_freq), "pre-sums")
    _assert_exact(vis.cpu().numpy(), oracle.correlate_dense(want, N, T, n_freq), "bundle-view visibilities")


def _entry_cases(seed, n):
    rng = random.Random(seed)
    out = []
    for k in range(n):
        N, T = rng.choice(N_EDGES), rng.choice(T_EDGES)
        while N * N * T > 1.5e9:
            T = max(1, T // 2)
        C = rng.randint(1, 3)
        out.append(pytest.param(N, T, C, k, id=f"e{k}-{N}x{T}x{C}"))
    return out


@pytest.mark.parametrize("N,T,C,k", _entry_cases(17320508, 12))
def test_noalloc_and_host_entry_points(xe, N, T, C, k):
    # The allocation-free entry point, the synchronous host-buffer call and the slotted
    # asynchronous host-buffer call on the same input: each equals the oracle.
    p = synth.uniform(N, T, C, seed=7000 + k)
    want = oracle.correlate_dense(p, N, T, C)
    got = xe.correlate_noalloc(torch.from_numpy(p).cuda(), N, T, C)
    torch.cuda.synchronize()
    xe.noalloc_status()
    _assert_exact(got.cpu().numpy(), want, "noalloc")
    host = torch.from_numpy(p).pin_memory()
    _assert_exact(xe.correlate_host(host, N, T, C).numpy(), want, "host")
    out, slot = xe.correlate_host_async(host, N, T, C, slot=k % xe.HOST_SLOTS)
    xe.host_wait(slot)
    _assert_exact(out.numpy(), want, "host async")
