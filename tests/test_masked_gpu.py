"""Flag-masked correlation and offset-binary input on the GPU, against the CPU oracle,
element by element (tolerance 0: visibilities and counts are exact integers).  Every call
goes through the C ABI (xe_correlate_masked / xe_correlate_masked_batch)."""
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
    xe.set_option("n_cta", 0)
    xe.set_option("sched", -1)
    xe.set_option("tile_n", 0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_masked(xe, packed, flags, N, T, C, enc=0, counts=True):
    vis, cnt = xe.correlate_masked(dev(packed), None if flags is None else dev(flags), N, T, C,
                                   encoding="offset" if enc else "twos", with_counts=counts)
    torch.cuda.synchronize()
    xe.device_status()
    return vis.cpu().numpy(), (cnt.cpu().numpy() if cnt is not None else None)


def check(xe, packed, flags, N, T, C, enc=0, dense=False):
    vis, cnt = run_masked(xe, packed, flags, N, T, C, enc)
    if dense:
        want = oracle.correlate_masked_dense(packed, flags, N, T, C, enc)
    else:
        want = oracle.correlate_masked(packed, flags, N, T, C, enc)
    bad = np.argwhere(vis != want)
    assert bad.size == 0, f"{len(bad)} visibility mismatches, first {bad[:3].tolist()}"
    f = flags if flags is not None else np.full((C, T, (N + 7) // 8), 0xFF, np.uint8)
    wc = oracle.flag_counts_dense(f, N, T, C) if dense else oracle.flag_counts(f, N, T, C)
    badc = np.argwhere(cnt != wc)
    assert badc.size == 0, f"{len(badc)} count mismatches, first {badc[:3].tolist()}"


def test_small_config_random_flags(xe):
    N, T = 64, 1024
    p = synth.uniform(N, T, 1)
    f = synth.flags(N, T, 1, p_bad=0.1, burst=16)
    check(xe, p, f, N, T, 1)


@pytest.mark.parametrize("enc", [0, 1])
@pytest.mark.parametrize("with_flags", [False, True])
def test_encodings(xe, enc, with_flags):
    N, T, C = 256, 2048, 2
    p = synth.gauss_plane(N, T, C, seed=41)
    if enc:
        p = synth.to_offset_binary(p)
    f = synth.flags(N, T, C, p_bad=0.2, seed=42) if with_flags else None
    check(xe, p, f, N, T, C, enc)


def test_offset_binary_equals_twos_on_same_values(xe):
    N, T = 512, 4096
    p = synth.uniform(N, T, 1, seed=3)
    f = synth.flags(N, T, 1, p_bad=0.05, seed=4, burst=64)
    a, ca = run_masked(xe, p, f, N, T, 1, 0)
    b, cb = run_masked(xe, synth.to_offset_binary(p), f, N, T, 1, 1)
    assert np.array_equal(a, b) and np.array_equal(ca, cb)


@pytest.mark.parametrize("N,T", [(1, 1), (3, 2), (7, 65), (100, 63), (130, 1000), (257, 129),
                                 (300, 77), (520, 300)])
def test_ragged_shapes(xe, N, T):
    # N % 16 != 0 or ceil(N/8) % 16 != 0 take the byte-load staging paths; ragged T ends
    # inside a 64-sample stage and inside a 256-sample count step.
    p = synth.uniform(N, T, 1, seed=N + T)
    f = synth.flags(N, T, 1, p_bad=0.3, seed=N * T + 1)
    check(xe, p, f, N, T, 1, enc=(N + T) % 2)


def test_flag_padding_bits_ignored(xe):
    N, T = 13, 50
    p = synth.uniform(N, T, 1, seed=8)
    f = synth.flags(N, T, 1, p_bad=0.3, seed=9)
    g = f.copy()
    g[..., -1] |= np.uint8(0xE0)            # bits of inputs 13..15 (do not exist)
    assert np.array_equal(run_masked(xe, p, f, N, T, 1)[0], run_masked(xe, p, g, N, T, 1)[0])
    assert np.array_equal(run_masked(xe, p, f, N, T, 1)[1], run_masked(xe, p, g, N, T, 1)[1])


def test_all_flagged_and_all_valid(xe):
    N, T = 384, 640
    p = synth.uniform(N, T, 1, seed=5)
    zero = np.zeros((1, T, N // 8), np.uint8)
    vis, cnt = run_masked(xe, p, zero, N, T, 1)
    assert not vis.any() and not cnt.any()
    ones = np.full((1, T, N // 8), 0xFF, np.uint8)
    vis, cnt = run_masked(xe, p, ones, N, T, 1)
    assert np.array_equal(vis, oracle.correlate(p, N, T)) and np.all(cnt == T)


def test_windows_offset_flags(xe):
    # Several exact accumulation windows: flag rows and count words start at t0 > 0.
    xe.set_option("exact_chunk_t", 192)
    N, T = 256, 1000
    p = synth.uniform(N, T, 1, seed=6)
    f = synth.flags(N, T, 1, p_bad=0.15, seed=7, burst=40)
    check(xe, p, f, N, T, 1, enc=0)


def test_unaligned_flags_pointer(xe):
    N, T = 2048, 512
    p = synth.uniform(N, T, 1, seed=10)
    f = synth.flags(N, T, 1, p_bad=0.1, seed=11)
    buf = torch.zeros(f.size + 16, dtype=torch.uint8, device="cuda")
    view = buf[3:3 + f.size]                 # 16-byte rows, but misaligned base
    view.copy_(dev(f.reshape(-1)))
    vis, cnt = xe.correlate_masked(dev(p), view, N, T, 1)
    torch.cuda.synchronize()
    xe.device_status()
    assert np.array_equal(vis.cpu().numpy(), oracle.correlate_masked_dense(p, f, N, T, 1))
    assert np.array_equal(cnt.cpu().numpy(), oracle.flag_counts_dense(f, N, T, 1))


def test_accumulate(xe):
    N, T = 256, 1536
    p1, p2 = synth.uniform(N, T, 1, seed=12), synth.uniform(N, T, 1, seed=13)
    f1, f2 = synth.flags(N, T, 1, 0.1, seed=14), synth.flags(N, T, 1, 0.3, seed=15)
    vis, cnt = xe.correlate_masked(dev(p1), dev(f1), N, T, 1)
    xe.correlate_masked(dev(p2), dev(f2), N, T, 1, out=vis, counts=cnt, accumulate=True)
    torch.cuda.synchronize()
    want = oracle.correlate_masked(p1, f1, N, T) + oracle.correlate_masked(p2, f2, N, T)
    wc = oracle.flag_counts(f1, N, T) + oracle.flag_counts(f2, N, T)
    assert np.array_equal(vis.cpu().numpy(), want)
    assert np.array_equal(cnt.cpu().numpy(), wc)


def test_masked_batch_mixed(xe):
    shapes = [(256, 2048, 1, 0, True, True), (512, 1024, 2, 1, True, False),
              (100, 333, 1, 1, False, True), (2048, 256, 1, 0, True, True)]
    jobs, want = [], []
    for q, (N, T, C, enc, has_f, has_c) in enumerate(shapes):
        p = synth.uniform(N, T, C, seed=100 + q)
        f = synth.flags(N, T, C, 0.2, seed=200 + q) if has_f else None
        pin = synth.to_offset_binary(p) if enc else p
        jobs.append({"in": dev(pin), "flags": dev(f) if has_f else None,
                     "vis": xe.empty_vis(N, C), "counts": xe.empty_counts(N, C) if has_c else None,
                     "N": N, "T": T, "C": C, "encoding": "offset" if enc else "twos"})
        fc = f if has_f else np.full((C, T, (N + 7) // 8), 0xFF, np.uint8)
        want.append((oracle.correlate_masked_dense(p, f, N, T, C),
                     oracle.flag_counts_dense(fc, N, T, C) if has_c else None))
    xe.correlate_masked_batch(jobs)
    torch.cuda.synchronize()
    xe.device_status()
    for j, (wv, wc) in zip(jobs, want):
        assert np.array_equal(j["vis"].cpu().numpy(), wv)
        if wc is not None:
            assert np.array_equal(j["counts"].cpu().numpy(), wc)


def test_full_size_masked(xe):
    # The masked workload at full size: N = 2048, T = 32768, RFI-like flags, offset binary.
    N, T = 2048, 32768
    p = synth.gauss_plane(N, T, 1)
    f = synth.flags(N, T, 1, p_bad=0.02, burst=256)
    check(xe, synth.to_offset_binary(p), f, N, T, 1, enc=1, dense=True)


def test_maximum_integration_length(xe):
    # T = XE_MAX_T = 2^24 - 1 samples of extreme offset-binary values (even inputs -8-8i,
    # odd inputs -8+7i), inputs 3 and 12 flagged throughout: Re V reaches 128 T = 2^31 - 128,
    # Im V +-120 T, and the valid-sample counts T.  The samples and flags do not change with t,
    # so by linearity in time V = T * V(one sample) and n = T * n(one sample), both from the
    # oracle.
    N, T = 17, xe.XE_MAX_T
    row = np.where(np.arange(N) % 2 == 0, synth.pack(-8, -8), synth.pack(-8, 7)).astype(np.uint8)
    row = synth.to_offset_binary(row[None, None, :])
    valid = np.ones(N, bool)
    valid[[3, 12]] = False
    frow = np.packbits(np.concatenate([valid, np.zeros(7, bool)])[:24].reshape(3, 8)[:, ::-1], axis=1)
    frow = frow.reshape(1, 1, 3)
    assert [(frow[0, 0, n // 8] >> (n % 8)) & 1 for n in range(N)] == valid.astype(int).tolist()
    want = oracle.correlate_masked(row, frow, N, 1, 1, encoding=1).astype(np.int64) * T
    want_n = oracle.flag_counts(frow, N, 1, 1) * T
    assert want.max() == 128 * T and want[..., 1].min() == -120 * T and want_n.max() == T
    x = dev(row[0, 0]).expand(T, N).contiguous()[None]
    f = dev(frow[0, 0]).expand(T, 3).contiguous()[None]
    vis, cnt = xe.correlate_masked(x, f, N, T, 1, encoding="offset")
    torch.cuda.synchronize()
    xe.device_status()
    assert np.array_equal(vis.cpu().numpy().astype(np.int64), want)
    assert np.array_equal(cnt.cpu().numpy().astype(np.int64), want_n)


def test_plain_path_unchanged_after_masked(xe):
    N, T = 1024, 4096
    p = synth.uniform(N, T, 1, seed=77)
    run_masked(xe, p, synth.flags(N, T, 1, 0.5, seed=78), N, T, 1)
    out = xe.correlate(dev(p), N, T, 1)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.correlate_dense(p, N, T))
