"""Parity of the CUDA path with the CPU oracle, element by element (tolerance 0: the
visibilities are exact integers).  Every call goes through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2005_09481_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALGOS = ("tc", "imma")


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
    xe.set_option("operand_bytes", 1)
    xe.set_option("exact_chunk_t", 131072)
    xe.set_option("n_cta", 0)


def run(xe, packed, N, T, C, algo="tc"):
    dev = torch.from_numpy(np.ascontiguousarray(packed)).cuda()
    out = xe.correlate(dev, N, T, C, algo=algo)
    torch.cuda.synchronize()
    xe.device_status()
    return out.cpu().numpy()


def assert_exact(got, want, what=""):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        k = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} mismatches, first at {k}: got {got[k]} want {want[k]}")


@pytest.mark.parametrize("algo", ALGOS)
def test_config1_plain_single_channel(xe, algo):
    # N=64, T=1024, one channel, uniform [-7, 7]: 2080 baselines.
    N, T = 64, 1024
    p = synth.uniform(N, T, 1)
    assert_exact(run(xe, p, N, T, 1, algo), oracle.correlate(p, N, T, 1), algo)


def test_maximum_input_count(xe):
    # N = XE_MAX_N = 65536 inputs: 2.1e9 baselines, a 17.2 GB output, 65,536 triangle tiles;
    # T = 96 samples (one full and one ragged k-block).  Checked against the oracle on
    # sampled baselines computed one by one: every pair of a set of rows and columns at the
    # tile edges and the array's ends, and 4096 random pairs.  The packed index passes 2^31.
    N, T = xe.XE_MAX_N, 96
    p = synth.uniform(N, T, 1, seed=4242)
    dev = torch.from_numpy(p).cuda()
    out = xe.correlate(dev, N, T, 1)
    torch.cuda.synchronize()
    xe.device_status()
    edges = [0, 1, 127, 128, 129, 255, 256, 257, N // 2 - 1, N // 2, N - 257, N - 256, N - 129,
             N - 128, N - 2, N - 1]
    pairs = [(a, b) for a in edges for b in edges if a <= b]
    rng = np.random.default_rng(99)
    u, v = rng.integers(0, N, 4096), rng.integers(0, N, 4096)
    pairs += [(int(min(a, b)), int(max(a, b))) for a, b in zip(u, v)]
    i = np.array([a for a, _ in pairs], np.int64)
    j = np.array([b for _, b in pairs], np.int64)
    k = i * N - i * (i - 1) // 2 + (j - i)
    assert k.max() > 2**31
    got = out[0][torch.from_numpy(k).cuda()].cpu().numpy().astype(np.int64)
    want = oracle.pairs(p, N, T, 1, np.zeros_like(i), i, j)
    assert_exact(got, want, "N=XE_MAX_N sampled baselines")
    del out, dev
    torch.cuda.empty_cache()


@pytest.mark.parametrize("N,T,C,parts", [(128, 65536, 1, 8), (512, 8192, 1, 4), (300, 8192, 2, 4),
                                         (1024, 32768, 1, 4), (2048, 4096, 1, 2)])
def test_exchanged_parts_are_exact(xe, N, T, C, parts):
    # Tiles split into 4 or 8 parts that exchange column slices (each part finalises its
    # slice from the others' published sums), including 128-wide tiles cut into 32-column
    # slices and a ragged input count; the default plan is checked to be that split.
    d = xe.plan_dump([(N, T, C)], 152)
    per_tile = {}
    for (cta, t, lo, hi, slot) in d["segs"]:
        per_tile[int(t)] = per_tile.get(int(t), 0) + 1
    assert set(per_tile.values()) == {parts}
    p = synth.uniform(N, T, C, seed=N + T + parts)
    assert_exact(run(xe, p, N, T, C, "tc"), oracle.correlate_dense(p, N, T, C), f"{N}x{T}x{C} in {parts} parts")


SHAPES = [(1, 1, 1), (2, 1, 1), (3, 5, 2), (17, 63, 1), (64, 64, 1), (100, 65, 3),
          (129, 127, 1), (255, 200, 1), (256, 1000, 1), (257, 129, 2), (300, 77, 1),
          (513, 300, 1), (640, 4096, 1)]


@pytest.mark.parametrize("N,T,C", SHAPES)
@pytest.mark.parametrize("algo", ALGOS)
def test_ragged_shapes(xe, N, T, C, algo):
    p = synth.uniform(N, T, C, seed=N * 1000 + T)
    assert_exact(run(xe, p, N, T, C, algo), oracle.correlate_dense(p, N, T, C), f"{algo} {N}x{T}x{C}")


def test_full_range_bytes_including_minus_eight(xe):
    rng = np.random.default_rng(9)
    N, T = 200, 500
    p = rng.integers(0, 256, size=(1, T, N), dtype=np.uint8)
    want = oracle.correlate_dense(p, N, T, 1)
    for algo in ALGOS:
        assert_exact(run(xe, p, N, T, 1, algo), want, algo)


def test_config2_full_array_full_output(xe):
    # N=2048, T=32768, quantised Gaussian + plane wave; oracle on the FULL output.
    N, T = 2048, 32768
    p = synth.gauss_plane(N, T, 1)
    want = oracle.correlate_dense(p, N, T, 1)
    assert np.abs(want[0, :, 1]).max() > 0          # the sky term makes Im nonzero
    assert_exact(run(xe, p, N, T, 1, "tc"), want, "tc config2")


def test_f16_operands_match(xe):
    N, T = 300, 1000
    p = synth.gauss_plane(N, T, 2, seed=3)
    want = oracle.correlate_dense(p, N, T, 2)
    xe.set_option("operand_bytes", 2)
    assert_exact(run(xe, p, N, T, 2, "tc"), want, "f16")


@pytest.mark.parametrize("n_cta", [1, 3, 7, 150, 152, 500])
def test_stream_k_splits_are_exact(xe, n_cta):
    # Different CTA counts split tiles at different k positions; sums must be identical.
    N, T = 520, 2000
    p = synth.uniform(N, T, 2, seed=5)
    want = oracle.correlate_dense(p, N, T, 2)
    xe.set_option("n_cta", n_cta)
    assert_exact(run(xe, p, N, T, 2, "tc"), want, f"n_cta={n_cta}")


@pytest.mark.parametrize("chunk", [64, 4096])
def test_exact_chunk_windows_accumulate(xe, chunk):
    # Long integrations are split into windows that accumulate into the int32 output.
    N, T = 130, 10000 + 37
    p = synth.uniform(N, T, 1, seed=6)
    xe.set_option("exact_chunk_t", chunk)
    assert_exact(run(xe, p, N, T, 1, "tc"), oracle.correlate_dense(p, N, T, 1), f"chunk={chunk}")


def test_extreme_magnitudes_across_windows(xe):
    # All samples -8-8i: Re V = 128 T, Im V = 0, with T past one 131072-sample window.
    N, T = 64, 131072 + 64 + 5
    p = synth.constant(N, T, -8, -8)
    got = run(xe, p, N, T, 1, "tc")
    assert (got[0, :, 0] == 128 * T).all() and (got[0, :, 1] == 0).all()
    p = synth.constant(N, 65536, 7, 7)
    got = run(xe, p, N, 65536, 1, "tc")
    assert (got[0, :, 0] == 98 * 65536).all() and (got[0, :, 1] == 0).all()


@pytest.mark.parametrize("algo", ALGOS)
def test_maximum_integration_length(xe, algo):
    # T = XE_MAX_T = 2^24 - 1 samples (128 windows of the f32 accumulator) of the extreme
    # values: even inputs hold -8-8i and odd inputs -8+7i, so Re V reaches 128 T = 2^31 - 128
    # and Im V reaches +120 T (even i < odd j) and -120 T (odd i < even j).  The samples do not change with t, so by linearity
    # in time V = T * V(one sample), the one-sample visibilities from the oracle.
    N, T = 17, xe.XE_MAX_T
    row = np.where(np.arange(N) % 2 == 0, synth.pack(-8, -8), synth.pack(-8, 7)).astype(np.uint8)
    one = oracle.correlate(row[None, None, :], N, 1, 1).astype(np.int64)
    want = one * T
    assert want.max() == 128 * T and want[..., 1].max() == 120 * T and want[..., 1].min() == -120 * T
    assert want.max() < 2**31 and want.min() >= -2**31
    dev = torch.from_numpy(row).cuda().expand(T, N).contiguous()[None]
    got = xe.correlate(dev, N, T, 1, algo=algo)
    torch.cuda.synchronize()
    xe.device_status()
    assert_exact(got.cpu().numpy().astype(np.int64), want, f"T=XE_MAX_T {algo}")
    del dev
    dev = torch.zeros((1, T + 1, N), dtype=torch.uint8, device="cuda")
    with pytest.raises(xe.XeError) as e:
        xe.correlate(dev, N, T + 1, 1, algo=algo)
    assert e.value.code == xe.XE_EOVERFLOW


def test_fp8_accumulation_adversaries(xe):
    # Patterns aimed at any precision loss of the f32 tensor-memory accumulator:
    # a large partial sum followed by +-1 terms, alternating +-7 cancellations, and
    # per-block magnitudes near powers of two.
    N = 256
    T1 = 60000
    big = synth.constant(N, T1, 7, -7)[0]
    rng = np.random.default_rng(1)
    small = synth.pack(rng.choice([-1, 1], size=(4096, N)), rng.choice([-1, 0, 1], size=(4096, N)))
    alt = np.where((np.arange(2048)[:, None] + np.arange(N)[None, :]) % 2 == 0,
                   synth.pack(7, 7), synth.pack(-7, -7)).astype(np.uint8)
    ramps = []
    for e in range(1, 8):
        v = min(7, 1 << (e % 3))
        ramps.append(np.full((512, N), synth.pack(v, -v), np.uint8))
    p = np.concatenate([big, small, alt, *ramps, small], axis=0)[None]
    T = p.shape[1]
    want = oracle.correlate_dense(p, N, T, 1)
    assert_exact(run(xe, p, N, T, 1, "tc"), want, "adversary")


def test_unaligned_input_pointer(xe):
    N, T = 96, 300
    p = synth.uniform(N, T, 1, seed=8)
    raw = torch.zeros(N * T + 1, dtype=torch.uint8, device="cuda")
    raw[1:] = torch.from_numpy(p.reshape(-1)).cuda()
    out = xe.correlate(raw[1:], N, T, 1)
    torch.cuda.synchronize()
    assert_exact(out.cpu().numpy(), oracle.correlate(p, N, T, 1), "unaligned")


def test_deterministic_repeats(xe):
    N, T = 700, 3000
    p = synth.gauss_plane(N, T, 1, seed=4)
    a = run(xe, p, N, T, 1, "tc")
    for _ in range(3):
        assert np.array_equal(run(xe, p, N, T, 1, "tc"), a)


def test_host_buffers_entry_point(xe):
    N, T = 333, 1111
    p = synth.uniform(N, T, 2, seed=12)
    got = xe.correlate_host(torch.from_numpy(p).pin_memory(), N, T, 2)
    assert_exact(got.numpy(), oracle.correlate_dense(p, N, T, 2), "host")


@pytest.mark.parametrize("chunk", [0, 64, 320, 8192])
def test_host_buffers_pipelined_chunks(xe, chunk):
    # The host entry point copies chunk k + 1 while chunk k is correlated (accumulating):
    # ragged last chunks, several channels (the chunk view's channel stride), one-shot mode.
    N, T, C = 272, 1000, 3
    p = synth.uniform(N, T, C, seed=chunk + 1)
    xe.set_option("host_chunk_t", chunk)
    try:
        got = xe.correlate_host(torch.from_numpy(p).pin_memory(), N, T, C)
    finally:
        xe.set_option("host_chunk_t", 8192)
    assert_exact(got.numpy(), oracle.correlate(p, N, T, C), f"host chunk {chunk}")


def test_host_async_slots_overlap_and_stay_exact(xe):
    N, T, C = 512, 4000, 2
    ins = [synth.uniform(N, T, C, seed=40 + k) for k in range(3)]
    pinned = [torch.from_numpy(p).pin_memory() for p in ins]
    outs = [xe.correlate_host_async(pinned[k], N, T, C, slot=k)[0] for k in range(3)]
    with pytest.raises(xe.XeError) as ei:          # slot 1 is still in flight
        xe.correlate_host_async(pinned[0], N, T, C, slot=1)
    assert ei.value.code == xe.XE_EAGAIN
    for k in (2, 0, 1):
        xe.host_wait(k)
    for k in range(3):
        assert_exact(outs[k].numpy(), oracle.correlate(ins[k], N, T, C), f"slot {k}")
    out, _ = xe.correlate_host_async(pinned[2], N, T, C, slot=1)   # reuse after the wait
    xe.host_wait(1)
    assert_exact(out.numpy(), oracle.correlate(ins[2], N, T, C), "slot reuse")


def test_bounded_wait_times_out_and_context_survives(xe):
    # Test hook: the producer warp issues no copies, so the MMA warp's bounded wait on the
    # pipeline barrier runs out (about a second); the kernel sets the status word, every
    # role exits, and the next call on the same context is exact again.
    N, T = 256, 1024
    p = synth.uniform(N, T, 1, seed=31)
    dev = torch.from_numpy(p).cuda()
    xe.set_option("inject_stall", 1)
    xe.correlate(dev, N, T, 1)
    with pytest.raises(xe.XeError) as ei:
        xe.device_status()
    assert ei.value.code == xe.XE_ETIMEOUT
    out = xe.correlate(dev, N, T, 1)
    torch.cuda.synchronize()
    xe.device_status()
    assert_exact(out.cpu().numpy(), oracle.correlate(p, N, T, 1), "after timeout")
