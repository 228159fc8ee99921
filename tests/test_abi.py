"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and exports every
function include/xe.h declares; host-only entry points behave (no GPU needed)."""
import ctypes
import os
import re
import struct

import numpy as np
import pytest

from paper_2005_09481_gb300 import xe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(xe_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("xe_correlate", "xe_correlate_async", "xe_correlate_batch",
                     "xe_stream_open", "xe_stream_push", "xe_stream_poll", "xe_stream_close",
                     "xe_strerror"):
        assert required in names


def test_binding_constants_match_the_header():
    src = open(os.path.join(ROOT, "include", "xe.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define\s+(XE_\w+)\s+(-?\d+)(?:LL)?\b", src)}
    for name in ("XE_OK", "XE_EINVAL", "XE_EOVERFLOW", "XE_ENOMEM", "XE_EBUDGET", "XE_EAGAIN",
                 "XE_ETIMEOUT", "XE_ECUDA", "XE_ENODEV", "XE_ECLOSED", "XE_ECHECK", "XE_MAX_T", "XE_MAX_N"):
        assert getattr(xe, name) == defs[name], name
    assert 128 * xe.XE_MAX_T < 2**31 <= 128 * (xe.XE_MAX_T + 1)


def test_every_entry_point_has_its_own_comment():
    # Each declaration in include/*.h follows a comment block (at most a #define between).
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        lines = open(os.path.join(ROOT, "include", h)).read().split("\n")
        depth = 0
        for i, line in enumerate(lines):
            s = line.strip()
            if s.startswith("/*") or depth:
                depth = 0 if s.endswith("*/") else 1
                continue
            if re.match(r"^[A-Za-z_][\w\s\*]*?\b(xe_\w+)\s*\(", s) and not s.startswith("#"):
                j = i - 1
                while j >= 0 and (not lines[j].strip() or lines[j].strip().startswith("#define")):
                    j -= 1
                assert lines[j].strip().endswith("*/"), f"{h}:{i + 1} {s[:50]}"


def test_every_declared_symbol_is_exported():
    L = xe.load()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, f"declared in include/*.h but not exported: {missing}"


def test_strerror_and_version():
    L = xe.load()
    assert L.xe_strerror(0) == b"ok"
    for code in range(-9, 0):
        assert L.xe_strerror(code) and L.xe_strerror(code) != b"unknown error"
    assert L.xe_version() >= 100


def test_cmac_count():
    assert xe.cmac(2048, 32768, 1) == 2_098_176 * 32768
    assert xe.cmac(64, 1024, 3) == 3 * 1024 * 2080


def test_argument_validation_before_any_device_call():
    L = xe.load()
    buf = (ctypes.c_uint8 * 64)()
    out = (ctypes.c_int32 * 64)()
    cases = [
        (None, 4, 4, 1, out, xe.XE_EINVAL),
        (buf, 4, 4, 1, None, xe.XE_EINVAL),
        (buf, 0, 4, 1, out, xe.XE_EINVAL),
        (buf, 4, 0, 1, out, xe.XE_EINVAL),
        (buf, 4, 4, 0, out, xe.XE_EINVAL),
        (buf, 4, 16777216, 1, out, xe.XE_EOVERFLOW),
        (buf, 70000, 4, 1, out, xe.XE_EINVAL),
    ]
    for inp, N, T, C, o, want in cases:
        rc = L.xe_correlate_async(inp, N, T, C, o, 1, None)
        assert rc == want, (N, T, C, rc)
    misaligned = ctypes.c_void_p(ctypes.addressof(out) + 4)
    assert L.xe_correlate_async(buf, 4, 4, 1, misaligned, 1, None) == xe.XE_EINVAL
    assert L.xe_correlate_async(buf, 4, 4, 1, out, 9, None) == xe.XE_EINVAL
    assert L.xe_last_error()


def test_masked_argument_validation_before_any_device_call():
    L = xe.load()
    buf = (ctypes.c_uint8 * 64)()
    flags = (ctypes.c_uint8 * 64)()
    out = (ctypes.c_int32 * 64)()
    cnt = (ctypes.c_int32 * 64)()
    # bad encoding, bad sizes, misaligned outputs: rejected before any device work
    assert L.xe_correlate_masked(buf, flags, 4, 4, 1, 2, out, cnt, 0, None) == xe.XE_EINVAL
    assert L.xe_correlate_masked(buf, flags, 4, 4, 1, -1, out, cnt, 0, None) == xe.XE_EINVAL
    assert L.xe_correlate_masked(buf, flags, 0, 4, 1, 0, out, cnt, 0, None) == xe.XE_EINVAL
    assert L.xe_correlate_masked(None, flags, 4, 4, 1, 0, out, cnt, 0, None) == xe.XE_EINVAL
    assert L.xe_correlate_masked(buf, flags, 4, 16777216, 1, 0, out, cnt, 0, None) == xe.XE_EOVERFLOW
    bad_cnt = ctypes.c_void_p(ctypes.addressof(cnt) + 2)
    assert L.xe_correlate_masked(buf, flags, 4, 4, 1, 0, out, bad_cnt, 0, None) == xe.XE_EINVAL
    bad_vis = ctypes.c_void_p(ctypes.addressof(out) + 4)
    assert L.xe_correlate_masked(buf, flags, 4, 4, 1, 1, bad_vis, cnt, 0, None) == xe.XE_EINVAL
    assert L.xe_correlate_masked_batch(None, 1, None) == xe.XE_EINVAL
    assert L.xe_correlate_masked(buf, flags, 4, 4, 1, 5, out, cnt, 0, None) == xe.XE_EINVAL
    assert b"encoding" in L.xe_last_error()


def test_beamform_argument_validation_before_any_device_call():
    L = xe.load()
    buf = (ctypes.c_uint8 * 64)()
    w = (ctypes.c_int8 * 64)()
    y = (ctypes.c_int32 * 64)()
    assert L.xe_beamform(None, 4, 4, 1, w, 1, y, None) == xe.XE_EINVAL
    assert L.xe_beamform(buf, 4, 4, 1, None, 1, y, None) == xe.XE_EINVAL
    assert L.xe_beamform(buf, 4, 4, 1, w, 0, y, None) == xe.XE_EINVAL
    assert L.xe_beamform(buf, 4, 4, 1, w, 129, y, None) == xe.XE_EINVAL
    assert L.xe_beamform(buf, 0, 4, 1, w, 1, y, None) == xe.XE_EINVAL
    assert L.xe_beamform(buf, 4, 0, 1, w, 1, y, None) == xe.XE_EINVAL
    bad = ctypes.c_void_p(ctypes.addressof(y) + 2)
    assert L.xe_beamform(buf, 4, 4, 1, w, 1, bad, None) == xe.XE_EINVAL
    assert L.xe_beamform(buf, 4, 4, 1, w, 200, y, None) == xe.XE_EINVAL
    assert b"n_beams" in L.xe_last_error()


def test_host_async_validation_before_any_device_call():
    L = xe.load()
    buf = (ctypes.c_uint8 * 64)()
    out = (ctypes.c_int32 * 64)()
    assert L.xe_correlate_host_async(buf, 4, 4, 1, out, -1) == xe.XE_EINVAL
    assert L.xe_correlate_host_async(buf, 4, 4, 1, out, 4) == xe.XE_EINVAL
    assert L.xe_correlate_host_async(None, 4, 4, 1, out, 0) == xe.XE_EINVAL
    assert L.xe_host_wait(7) == xe.XE_EINVAL


def test_options_validation():
    with pytest.raises(xe.XeError):
        xe.set_option("operand_bytes", 3)
    with pytest.raises(xe.XeError):
        xe.set_option("exact_chunk_t", 1 << 30)
    with pytest.raises(xe.XeError):
        xe.set_option("no_such_option", 1)
    with pytest.raises(xe.XeError):
        xe.set_option("host_chunk_t", 100)
    xe.set_option("operand_bytes", 1)


def _e4m3_value(code):
    s = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    m = code & 7
    if e == 0:
        return s * (m / 8.0) * 2.0 ** -6
    return s * (1 + m / 8.0) * 2.0 ** (e - 7)


def test_operand_encoder_is_exact():
    # e4m3 (sign, 4-bit exponent bias 7, 3-bit mantissa) and IEEE half represent every
    # integer in [-16, 16] exactly; the encoder must produce those bit patterns.
    for v in range(-16, 17):
        c8 = xe.operand_code(v, 1)
        assert c8 < 256 and _e4m3_value(c8) == v
        c16 = xe.operand_code(v, 2)
        assert struct.unpack("<e", struct.pack("<H", c16))[0] == v


def _tiles_py(N):
    """Independent enumeration of the tile cover: every (i, j >= i) exactly once."""
    cover = np.zeros((N, N), np.int32)
    tiles = 0
    for i0 in range(0, N, 128):
        j0 = i0
        spans = []
        if j0 % 256:
            spans.append((j0, 128))
            j0 += 128
        while j0 < N:
            spans.append((j0, 256))
            j0 += 256
        for (a, w) in spans:
            tiles += 1
            for i in range(i0, min(i0 + 128, N)):
                lo = max(a, i)
                if lo < min(a + w, N):
                    cover[i, lo:min(a + w, N)] += 1
    return tiles, cover


@pytest.mark.parametrize("N", [1, 100, 128, 129, 255, 256, 257, 384, 600, 2048])
def test_plan_covers_triangle_once(N):
    tiles, cover = _tiles_py(N)
    iu = np.triu_indices(N)
    assert (cover[iu] == 1).all() and cover.sum() == N * (N + 1) // 2
    # 4096 samples (64 k-blocks): long enough that the default keeps 256-wide tiles (short
    # calls of up to 256 inputs take 128-wide ones; a one-block N <= 128 is one tile either way).
    n_tiles, n_iters, _ = xe.plan_stats([(N, 4096, 1)], 152)
    assert n_tiles == tiles
    assert n_iters == tiles * 64


def test_plan_stats_batch_and_split():
    n_tiles, n_iters, n_split = xe.plan_stats([(2048, 32768, 1)], 152)
    assert n_tiles == 72 and n_iters == 72 * 512
    assert 0 < n_split <= 72
    # one CTA: nothing is split
    assert xe.plan_stats([(2048, 32768, 1)], 1)[2] == 0
    t2, i2, _ = xe.plan_stats([(256, 4096, 2), (512, 8192, 1)], 152)
    assert t2 == 2 * 2 + 6 and i2 == 4 * 64 + 6 * 128


def _check_plan(shapes, n_cta, sched, tile_n):
    d = xe.plan_dump(shapes, n_cta, sched, tile_n)
    tiles, segs = d["tiles"], d["segs"]
    # tiles: cover every (i, j >= i) of every job/channel exactly once
    for q, (N, T, C) in enumerate(shapes):
        for c in range(C):
            cover = np.zeros((N, N), np.int32)
            for (job, ch, i0, j0, nj, kb) in tiles:
                if job != q or ch != c:
                    continue
                assert kb == (T + 63) // 64
                for i in range(i0, min(i0 + 128, N)):
                    lo = max(j0, i)
                    if lo < min(j0 + nj, N):
                        cover[i, lo:min(j0 + nj, N)] += 1
            iu = np.triu_indices(N)
            assert (cover[iu] == 1).all() and cover.sum() == N * (N + 1) // 2
    # segments: every k of every tile exactly once; partial segments own distinct slots
    seen = {t: np.zeros(int(tiles[t][5]), np.int32) for t in range(len(tiles))}
    slots = []
    per_tile = {}
    for (cta, t, lo, hi, slot) in segs:
        assert 0 <= cta < d["n_cta"] <= n_cta and lo < hi and 0 <= t < len(tiles)
        seen[int(t)][lo:hi] += 1
        per_tile.setdefault(int(t), []).append(int(slot))
    for t, v in seen.items():
        assert (v == 1).all(), f"tile {t} k-cover {v.min()}..{v.max()}"
        sl = per_tile[t]
        if len(sl) == 1:
            assert sl == [-1]
        else:
            assert min(sl) >= 0
            slots += sl
    assert len(slots) == len(set(slots)) == d["n_partial"]
    return d


@pytest.mark.parametrize("sched", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("tile_n", [128, 256])
def test_schedules_cover_every_tile_and_k_once(sched, tile_n):
    for shapes, n_cta in [([(2048, 32768, 1)], 152), ([(300, 1000, 3)], 7), ([(100, 64, 1)], 152),
                          ([(256, 4096, 2), (512, 8192, 1), (130, 700, 1)], 19),
                          ([(1024, 8192, 1)] * 4, 152)]:
        _check_plan(shapes, n_cta, sched, tile_n)


@pytest.mark.parametrize("seed", range(12))
def test_plan_sweep_covers_every_tile_and_k_once(seed):
    # Seeded batches at the tile and k-block edges under every schedule (and the automatic
    # choice), tile width and CTA count from 1 to beyond one per SM: each plan covers every
    # baseline of every job and channel once, every k-block of every tile once, and gives
    # the parts of each split tile distinct workspace slots.
    rng = np.random.default_rng(100 + seed)
    Ns = [1, 2, 63, 64, 65, 127, 128, 129, 255, 256, 257, 511, 513, 1023, 1025, 2048]
    Ts = [1, 63, 64, 65, 1000, 4096, 8193, 32768, 65536]
    for _ in range(10):
        shapes = [(int(rng.choice(Ns)), int(rng.choice(Ts)), int(rng.integers(1, 3)))
                  for _ in range(int(rng.integers(1, 5)))]
        n_cta = int(rng.choice([1, 2, 5, 37, 144, 152, 300]))
        _check_plan(shapes, n_cta, int(rng.choice([-1, 0, 1, 2, 3, 4])), int(rng.choice([0, 128, 256])))


@pytest.mark.parametrize("seed", range(6))
def test_lpt_schedule_is_the_greedy_longest_first(seed):
    # The uneven-batch schedule against a plain heap greedy: tiles longest first (ties in tile
    # order), each to the CTA with the least load (lowest index among equals); every CTA then
    # walks its tiles in tile order, each whole.
    import heapq
    rng = np.random.default_rng(seed)
    shapes = [(int(rng.choice([64, 130, 256, 700, 2048])), int(rng.choice([64, 1000, 8192, 16384, 32768])), 1)
              for _ in range(int(rng.integers(2, 30)))]
    if rng.integers(2):
        shapes.sort(key=lambda s: -s[1])
    n_cta = int(rng.choice([7, 148, 152, 304]))
    d = xe.plan_dump(shapes, n_cta, xe.SCHEDULES["lpt"], 256)
    kb = d["tiles"][:, 5]
    order = sorted(range(len(kb)), key=lambda t: -kb[t])          # stable: ties keep tile order
    heap = [(0, b) for b in range(n_cta)]
    per = [[] for _ in range(n_cta)]
    for t in order:
        load, b = heapq.heappop(heap)
        per[b].append(t)
        heapq.heappush(heap, (load + int(kb[t]), b))
    want = [(b, t, 0, int(kb[t])) for b in range(n_cta) for t in sorted(per[b])]
    got = [tuple(int(v) for v in s[:4]) for s in d["segs"]]
    assert got == want


def test_split_schedule_aligns_parts_for_the_headline():
    d = _check_plan([(2048, 32768, 1)], 152, 1, 256)
    assert d["n_cta"] == 144                       # 72 tiles x 2 equal k-parts
    assert set(map(tuple, d["segs"][:, 2:4].tolist())) == {(0, 256), (256, 512)}


def test_hybrid_schedule_full_waves_whole():
    d = _check_plan([(2048, 16384, 16)], 152, 2, 256)
    whole = (d["segs"][:, 4] == -1).sum()
    assert whole >= (1152 // 152) * 152            # full waves are whole tiles


def _parts_per_tile(d):
    counts = {}
    for (cta, t, lo, hi, slot) in d["segs"]:
        counts[int(t)] = counts.get(int(t), 0) + 1
    return sorted(set(counts.values()))


def test_split_parts_follow_the_fix_up_cost_model():
    # Parts per tile minimise (longest tile's k-blocks / parts) + fix-up: 8 k-blocks for two
    # parts and 30 or 56 for four or eight parts that exchange column slices (at least 32
    # columns each, every part alone on its CTA), else 20 per part beyond the first (the
    # last arriver's sum); up to the CTAs per tile.  The default schedule for fewer tiles
    # than CTAs is the split, also for jobs of different lengths.
    def model(kb, s_max, min_nj):
        cost = {1: kb}
        for c in range(2, s_max + 1):
            fix = 8 if c == 2 else 20 * (c - 1)
            if c in (4, 8) and min_nj // c >= 32:
                fix = 30 if c == 4 else 56
            cost[c] = kb / c + fix
        return min(cost, key=lambda c: (cost[c], c))
    for (N, T, C) in [(64, 1024, 1), (256, 4096, 1), (512, 8192, 1), (128, 65536, 1), (2048, 4096, 1),
                      (2048, 32768, 1), (256, 32768, 1), (1024, 32768, 1)]:
        d = _check_plan([(N, T, C)], 152, -1, 0)
        n_tiles, min_nj = len(d["tiles"]), int(d["tiles"][:, 4].min())
        kb = (T + 63) // 64
        want = model(kb, min(152 // n_tiles, kb), min_nj)
        assert _parts_per_tile(d) == [want], (N, T, _parts_per_tile(d), want)
    # Worked values: a 16-k-block tile whole, a 128-k-block tile in four exchanging parts, a
    # 1024-k-block tile in eight, 512-k-block tiles in four when 7 CTAs are free per tile,
    # the headline's two.
    assert [model(16, 152, 256), model(128, 25, 128), model(1024, 152, 256), model(512, 7, 256),
            model(512, 2, 256)] == [1, 4, 8, 4, 2]
    # Four or eight parts exchange slices (the plan's exchange flag is visible in the eight
    # parts of a single 128-input tile and the two of the headline).
    for sh in [(128, 65536, 1), (2048, 32768, 1)]:
        d = xe.plan_dump([sh], 152)
        assert d["n_partial"] == len(d["segs"])
    # Jobs of different lengths with fewer tiles than CTAs are split, not dealt whole.
    d = _check_plan([(1024, 32768, 1), (256, 4096, 1), (512, 2048, 1)], 152, -1, 0)
    assert max(_parts_per_tile(d)) > 1


def test_default_tile_width_follows_the_problem_size():
    # 128-wide tiles for one-block problems (N <= 128) of up to 256 k-blocks and for short
    # calls of up to 256 inputs (at most 32 k-blocks); 256-wide tiles otherwise.
    for (N, T), nj in [((64, 1024), 128), ((128, 16384), 128), ((128, 65536), 256), ((256, 1024), 128),
                       ((200, 2048), 128),
                       ((256, 4096), 256), ((257, 1024), 256), ((2048, 1024), 256), ((2048, 32768), 256)]:
        d = _check_plan([(N, T, 1)], 152, -1, 0)
        assert set(d["tiles"][:, 4].tolist()) <= {nj, 128} and int(d["tiles"][:, 4].max()) == nj, (N, T)


def test_hybrid_tail_is_split_by_the_cost_model():
    # 178 tiles on 152 CTAs: one whole wave, then the 26 tail tiles split over the CTAs
    # (up to 5 per tile; two segments on a CTA, so no exchange) by the same model, not cut
    # into a stream-K share of every CTA.
    d = _check_plan([(2176, 8192, 2)], 152, 2, 256)
    kb = 128
    parts = _parts_per_tile(d)
    assert 1 in parts and max(parts) == 3            # 128/3 + 40 < 128/2 + 20 < 128
    assert kb / 3 + 40 < kb / 2 + 20 < kb


def test_schedule_options_are_the_five_single_cta_schedules():
    # Schedules 0..4 exist; there is no clustered (multi-CTA) variant any more.
    for sched in range(5):
        xe.set_option("sched", sched)
    xe.set_option("sched", -1)
    with pytest.raises(xe.XeError):
        xe.set_option("sched", 5)
    with pytest.raises(xe.XeError):
        xe.plan_dump([(256, 1024, 1)], 8, 5, 256)


def test_plain_c_program_links_and_calls_the_library(tmp_path):
    # The boundary is a C ABI: a C11 program includes xe.h, links libxe.so and calls the
    # host-only entry points (no GPU needed).
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lib = xe.lib_path()
    src = tmp_path / "use_xe.c"
    src.write_text(r"""
#include <stdio.h>
#include "xe.h"
int main(void) {
    const int N[1] = {2048};
    const int64_t T[1] = {32768};
    const int C[1] = {1};
    int64_t tiles = 0, iters = 0, split = 0;
    int rc = xe_plan_stats(N, T, C, 1, 152, &tiles, &iters, &split);
    printf("%d %.0f %d %d %d %lld %lld %s\n", xe_version() >= 100, xe_cmac(2048, 32768, 1),
           xe_correlate(NULL, 4, 4, 1, NULL), xe_correlate(NULL, 4, 16777216, 1, NULL), rc,
           (long long)tiles, (long long)split, xe_strerror(XE_OK));
    return 0;
}
""")
    exe = tmp_path / "use_xe"
    libdir = os.path.dirname(lib)
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-pedantic", f"-I{os.path.join(ROOT, 'include')}",
                    str(src), f"-L{libdir}", "-lxe", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert out == ["1", str(2_098_176 * 32768), str(xe.XE_EINVAL), str(xe.XE_EINVAL), "0", "72", "72", "ok"]


def test_error_detail_is_per_thread():
    # xe_last_error reports the last failure of the calling thread only.
    import threading
    L = xe.load()
    buf = (ctypes.c_uint8 * 64)()
    out = (ctypes.c_int32 * 64)()
    barrier = threading.Barrier(2)
    seen = {}

    def worker(name, args, code):
        assert L.xe_correlate(*args) == code
        barrier.wait()                      # both threads have failed before either reads
        seen[name] = L.xe_last_error().decode()

    a = threading.Thread(target=worker, args=("overflow", (buf, 4, 16777216, 1, out), xe.XE_EOVERFLOW))
    b = threading.Thread(target=worker, args=("n", (buf, 0, 4, 1, out), xe.XE_EINVAL))
    a.start(), b.start()
    a.join(), b.join()
    assert "16777216" in seen["overflow"] and "N=0" in seen["n"]


def test_compute_calls_without_a_device_fail_with_enodev():
    # No CPU fallback: on a machine without a usable CUDA device every compute entry point
    # returns XE_ENODEV (and the binding raises), for valid arguments.
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    L = xe.load()
    N, T = 64, 128
    inp = (ctypes.c_uint8 * (N * T))()
    vis = (ctypes.c_int32 * (N * (N + 1)))()
    w = (ctypes.c_int8 * (2 * N))()
    y = (ctypes.c_int32 * (2 * T))()
    frames = (ctypes.c_uint8 * (N * T))()
    d = ctypes.c_double()
    calls = {
        "xe_correlate": lambda: L.xe_correlate(inp, N, T, 1, vis),
        "xe_correlate_host": lambda: L.xe_correlate_host(inp, N, T, 1, vis, 0),
        "xe_correlate_noalloc": lambda: L.xe_correlate_noalloc(inp, N, T, 1, vis, None),
        "xe_noalloc_status": lambda: L.xe_noalloc_status(None),
        "xe_beamform": lambda: L.xe_beamform(inp, N, T, 1, w, 1, y, None),
        "xe_corner_turn": lambda: L.xe_corner_turn(inp, 2, 1, N // 2, T, frames, None, None),
        "xe_peak_probe": lambda: L.xe_peak_probe(0, ctypes.byref(d), ctypes.byref(d)),
        "xe_release_stream": lambda: L.xe_release_stream(None),
    }
    for name, call in calls.items():
        assert call() == xe.XE_ENODEV, (name, L.xe_last_error())
    with pytest.raises(xe.XeError) as e:
        xe.correlate_host(torch.zeros((1, T, N), dtype=torch.uint8), N, T, 1)
    assert e.value.code == xe.XE_ENODEV
    with pytest.raises(xe.XeError) as e:
        xe.Stream(N, 8192, 32768, max_chan=1, hbm_budget=1 << 30)
    assert e.value.code == xe.XE_ENODEV


def test_stream_slot_bytes_match_the_serving_loop():
    # The serving loop sizes HBM budgets with serve.per_channel_bytes; the library admits a
    # channel only if its slot fits.  Both count the same bytes: one byte less than a slot
    # is refused before any device work (XE_EBUDGET), a whole slot passes that check.
    from paper_2005_09481_gb300 import serve
    L = xe.load()
    for N, frame_T, ring in ((2048, 8192, 8), (64, 1000, 2), (300, 4096, 3), (17, 64, 5)):
        per = serve.per_channel_bytes(N, frame_T, ring)
        h = ctypes.c_void_p()
        cfg = xe.StreamCfg(N, frame_T, 4 * frame_T, 4, per - 1, ring, 390625.0, 0)
        assert L.xe_stream_open(ctypes.byref(cfg), ctypes.byref(h)) == xe.XE_EBUDGET
        cfg.hbm_budget = per
        rc = L.xe_stream_open(ctypes.byref(cfg), ctypes.byref(h))
        assert rc != xe.XE_EBUDGET, (N, frame_T, ring)
        if rc == xe.XE_OK:
            L.xe_stream_close(h)


def test_noalloc_limits_refused_before_any_device_call():
    # The allocation-free entry point refuses requests beyond its fixed scratch on the host:
    # the integration length, the staged planes of one 64-sample block, the tile table.
    L = xe.load()
    buf = (ctypes.c_uint8 * 64)()
    out = (ctypes.c_int32 * 64)()
    for (N, T, C, code, what) in [(64, xe.XE_MAX_T + 1, 1, xe.XE_EOVERFLOW, b"XE_MAX_T"),
                                  (2048, 64, 200, xe.XE_EINVAL, b"staged operands"),
                                  (65536, 64, 4, xe.XE_EINVAL, b"staged operands"),
                                  (16384, 64, 1, xe.XE_EINVAL, b"tiles")]:
        assert L.xe_correlate_noalloc(buf, N, T, C, out, None) == code
        assert what in L.xe_last_error(), (N, T, C, L.xe_last_error())


@pytest.mark.parametrize("n_cyl,n_freq,n_in,T", [(4, 4, 512, 7), (3, 2, 5, 9), (1, 1, 16, 3), (4, 2, 128, 2)])
def test_bundle_view_addresses_every_sample_of_the_bundles(n_cyl, n_freq, n_in, T):
    # The view's address of sample (c, t, n), c*s_c + t*s_t + (n // seg)*s_seg + n % seg, is
    # where the cylinder bundles [n_cyl][T][n_freq][n_in] hold that sample of channel c.
    from paper_2005_09481_gb300 import synth
    N = n_cyl * n_in
    v = xe.bundle_view(n_cyl, n_freq, n_in, T)
    assert v.seg_inputs == n_in
    frames = synth.uniform(N, T, n_freq, seed=5)                    # [n_freq][T][N]
    flat = synth.bundles_of(frames, n_cyl).reshape(-1)
    c, t, n = np.meshgrid(np.arange(n_freq), np.arange(T), np.arange(N), indexing="ij")
    addr = c * v.chan_stride + t * v.time_stride + (n // v.seg_inputs) * v.seg_stride + n % v.seg_inputs
    assert addr.min() >= 0 and addr.max() < flat.size
    assert np.array_equal(flat[addr], frames)
    assert len(np.unique(addr)) == addr.size                         # one byte per sample


def test_bundle_view_rejects_bad_shapes():
    L = xe.load()
    v = xe.View()
    for args in [(0, 4, 512, 10), (4, 0, 512, 10), (4, 4, 0, 10), (4, 4, 512, 0), (200, 1, 512, 10)]:
        assert L.xe_bundle_view(*args, ctypes.byref(v)) == xe.XE_EINVAL, args


def test_binding_checks_tensors_before_calling_the_library():
    # The binding refuses wrong dtypes, layouts, sizes and devices itself (no library call).
    torch = pytest.importorskip("torch")
    N, T = 8, 16
    x = torch.zeros((1, T, N), dtype=torch.uint8)
    with pytest.raises(TypeError):
        xe.correlate(x.to(torch.int8), N, T, 1)
    with pytest.raises(ValueError):
        xe.correlate(torch.zeros((1, T, 2 * N), dtype=torch.uint8)[:, :, ::2], N, T, 1)   # not contiguous
    with pytest.raises(ValueError):
        xe.correlate(x, N, T + 1, 1)                                                       # wrong size
    with pytest.raises(ValueError):
        xe.correlate(x, N, T, 1)                                                           # host tensor
    with pytest.raises(ValueError):
        xe.correlate_host(x.cuda() if torch.cuda.is_available() else x[:, :1], N, T, 1)
    with pytest.raises(ValueError):
        xe.beamform(x, torch.zeros((1, N, 2), dtype=torch.int8), N, T, 1)                # host weights
    with pytest.raises(ValueError):
        xe.correlate_masked(x, torch.zeros((1, T, 1), dtype=torch.uint8), N, T, 1)       # host flags
    B = N * (N + 1) // 2
    for bad in (torch.zeros(2 * B - 1, dtype=torch.int32), torch.zeros(2 * B, dtype=torch.int64),
                torch.zeros((2, B), dtype=torch.int32).t()):
        with pytest.raises(ValueError):
            xe.correlate_host(x, N, T, 1, out=bad)                                         # bad outputs
    with pytest.raises(ValueError):
        xe.correlate_batch([(x, torch.zeros((1, B, 2), dtype=torch.int32), N, T, 1)])      # host input


def test_check_corruption_hook_needs_the_checks():
    # The corruption test hook is refused unless the descriptor checks are on, so that no
    # corrupted descriptor can reach a kernel unchecked.
    L = xe.load()
    assert L.xe_set_option(b"checks", 0) == xe.XE_OK
    assert L.xe_set_option(b"check_corrupt", 1) == xe.XE_EINVAL
    assert L.xe_set_option(b"checks", 1) == xe.XE_OK
    assert L.xe_set_option(b"check_corrupt", 3) == xe.XE_EINVAL
    assert L.xe_set_option(b"check_corrupt", 2) == xe.XE_OK
    assert L.xe_set_option(b"checks", 0) == xe.XE_OK      # also clears the hook
    assert L.xe_set_option(b"check_corrupt", 0) == xe.XE_OK
    assert L.xe_strerror(xe.XE_ECHECK).startswith(b"a device-side check")


def test_stream_config_validation_before_any_device_call():
    # Every field of the stream configuration is checked before the library touches a
    # device: bad shapes are XE_EINVAL, an integration too long for int32 sums XE_EOVERFLOW.
    L = xe.load()
    good = dict(N=64, frame_T=1024, integ_T=4096, max_chan=4, hbm_budget=1 << 30, ring_frames=3)

    def opened(**kw):
        c = dict(good, **kw)
        cfg = xe.StreamCfg(c["N"], c["frame_T"], c["integ_T"], c["max_chan"], c["hbm_budget"],
                           c["ring_frames"], 390625.0, 0)
        h = ctypes.c_void_p()
        rc = L.xe_stream_open(ctypes.byref(cfg), ctypes.byref(h))
        if rc == xe.XE_OK:
            L.xe_stream_close(h)
        return rc

    for kw in (dict(N=0), dict(N=xe.XE_MAX_N + 1), dict(frame_T=0), dict(frame_T=131073, integ_T=131073),
               dict(integ_T=1000), dict(integ_T=4097), dict(max_chan=0), dict(max_chan=65537),
               dict(ring_frames=1), dict(ring_frames=65)):
        assert opened(**kw) == xe.XE_EINVAL, kw
    assert opened(frame_T=8192, integ_T=8192 * 2049) == xe.XE_EOVERFLOW
    assert opened() in (xe.XE_OK, xe.XE_ENODEV)
    assert L.xe_stream_open(None, None) == xe.XE_EINVAL
