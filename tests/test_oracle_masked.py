"""Pins of the flag-masked / offset-binary oracle (CPU only).

What fixes the masked oracle, independently of itself:
* hand-computed cases (tests/golden/masked_hand.txt);
* relations to the plain oracle, which is pinned on its own (test_oracle_pins.py):
  flags=None is the plain correlation, a flagged sample equals a zero byte (0 + 0i in two's
  complement), and offset-binary bytes are the two's-complement bytes XOR 0x88;
* brute force in pure Python on tiny inputs (complex arithmetic, explicit loops);
* closed forms of the counts: per-time flags give the same count on every baseline, the
  diagonal count is the number of valid samples of that input, all-valid gives T;
* planted mistakes: each mutant of the masked C code fails one of the pins above.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2005_09481_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden", "masked_hand.txt")
SRC = os.path.join(ROOT, "oracle", "xe_oracle.c")


def golden_cases():
    with open(GOLDEN) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    out = []
    for row in rows:
        bar = [k for k, tok in enumerate(row) if tok == "|"]
        name, enc, N, T = row[0], int(row[1]), int(row[2]), int(row[3])
        b = np.array([int(x, 16) for x in row[bar[0] + 1:bar[1]]], np.uint8)
        ftok = row[bar[1] + 1:bar[2]]
        flags = None if ftok == ["-"] else np.array([int(x, 16) for x in ftok], np.uint8)
        vis = np.array([[int(v) for v in p.split(",")] for p in row[bar[2] + 1:bar[3]]], np.int64)
        cnt = np.array([int(v) for v in row[bar[3] + 1:]], np.int64)
        out.append((name, enc, N, T, b, flags, vis, cnt))
    return out


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c[0])
def test_golden_hand_cases(case):
    name, enc, N, T, b, flags, vis, cnt = case
    assert np.array_equal(oracle.correlate_masked(b, flags, N, T, 1, enc)[0], vis)
    assert np.array_equal(oracle.correlate_masked_dense(b, flags, N, T, 1, enc)[0], vis)
    f = flags if flags is not None else np.full(T * ((N + 7) // 8), 0xFF, np.uint8)
    assert np.array_equal(oracle.flag_counts(f, N, T)[0], cnt)
    assert np.array_equal(oracle.flag_counts_dense(f, N, T)[0], cnt)


def _zero_flagged(packed, flags, N, T, C):
    valid = oracle.valid_bits(flags, N, T, C)
    z = np.asarray(packed, np.uint8).reshape(C, T, N).copy()
    z[~valid] = 0
    return z


@pytest.mark.parametrize("N,T,C", [(1, 5, 1), (9, 40, 2), (33, 17, 1), (64, 128, 1)])
def test_flagged_sample_equals_zero_byte(N, T, C):
    p = synth.uniform(N, T, C, seed=11)
    f = synth.flags(N, T, C, p_bad=0.3, seed=12, burst=3)
    got = oracle.correlate_masked(p, f, N, T, C)
    assert np.array_equal(got, oracle.correlate(_zero_flagged(p, f, N, T, C), N, T, C))


@pytest.mark.parametrize("N,T,C", [(3, 7, 1), (40, 64, 2)])
def test_no_flags_is_plain_correlation(N, T, C):
    p = synth.gauss_plane(N, T, C, seed=5)
    assert np.array_equal(oracle.correlate_masked(p, None, N, T, C), oracle.correlate(p, N, T, C))
    ones = np.full((C, T, (N + 7) // 8), 0xFF, np.uint8)
    assert np.array_equal(oracle.correlate_masked(p, ones, N, T, C), oracle.correlate(p, N, T, C))
    assert np.all(oracle.flag_counts(ones, N, T, C) == T)


@pytest.mark.parametrize("N,T", [(5, 9), (48, 100)])
def test_offset_binary_is_xor_0x88(N, T):
    p = synth.uniform(N, T, 1, seed=21)
    f = synth.flags(N, T, 1, p_bad=0.2, seed=22)
    ob = synth.to_offset_binary(p)
    assert np.array_equal(oracle.correlate_masked(ob, None, N, T, 1, 1), oracle.correlate(p, N, T))
    assert np.array_equal(oracle.correlate_masked(ob, f, N, T, 1, 1),
                          oracle.correlate_masked(p, f, N, T, 1, 0))


def test_offset_binary_full_decode_table():
    # Every byte: offset-binary value (u - 8, w - 8) for nibbles (u, w); the autocorrelation
    # of one sample is |x|^2 and the cross term with the unit sample 1 + 0i is x itself.
    one = 0x98   # offset binary of 1 + 0i
    for byte in range(256):
        u, w = byte >> 4, byte & 0xF
        b = np.array([byte, one], np.uint8)
        v = oracle.correlate_masked(b, None, 2, 1, 1, 1)[0]
        assert v[0, 0] == (u - 8) ** 2 + (w - 8) ** 2 and v[0, 1] == 0
        assert v[1, 0] == u - 8 and v[1, 1] == w - 8


def test_brute_force_python_loops():
    rng = np.random.default_rng(7)
    for _ in range(6):
        N, T = int(rng.integers(1, 6)), int(rng.integers(1, 9))
        enc = int(rng.integers(0, 2))
        b = rng.integers(0, 256, size=(T, N)).astype(np.uint8)
        f = rng.integers(0, 256, size=(T, (N + 7) // 8)).astype(np.uint8)

        def val(byte):
            hi, lo = byte >> 4, byte & 0xF
            if enc == 1:
                return complex(hi - 8, lo - 8)
            return complex(hi - 16 if hi >= 8 else hi, lo - 16 if lo >= 8 else lo)

        def ok(t, n):
            return (int(f[t, n // 8]) >> (n % 8)) & 1

        want, cnt = [], []
        for i in range(N):
            for j in range(i, N):
                s, n = 0j, 0
                for t in range(T):
                    if ok(t, i) and ok(t, j):
                        s += val(int(b[t, i])) * val(int(b[t, j])).conjugate()
                        n += 1
                want.append((int(s.real), int(s.imag)))
                cnt.append(n)
        assert np.array_equal(oracle.correlate_masked(b, f, N, T, 1, enc)[0], np.array(want))
        assert np.array_equal(oracle.flag_counts(f, N, T)[0], np.array(cnt))


def test_counts_closed_forms():
    N, T = 37, 300
    # Per-time flags (a sample flagged on every input): every baseline counts the same.
    rng = np.random.default_rng(3)
    good_t = rng.random(T) > 0.35
    f = np.zeros((1, T, (N + 7) // 8), np.uint8)
    f[0, good_t, :] = 0xFF
    assert np.all(oracle.flag_counts(f, N, T) == good_t.sum())
    # Diagonal count = valid samples of that input; off-diagonal <= both diagonals.
    g = synth.flags(N, T, 1, p_bad=0.4, seed=9)
    cnt = oracle.flag_counts(g, N, T)[0]
    valid = oracle.valid_bits(g, N, T)[0]
    for i in range(N):
        assert cnt[oracle.tri_index(N, i, i)] == valid[:, i].sum()
    iu = np.triu_indices(N)
    diag = cnt[[oracle.tri_index(N, i, i) for i in range(N)]]
    assert np.all(cnt <= np.minimum(diag[iu[0]], diag[iu[1]]))


@pytest.mark.parametrize("N,T,C,enc", [(50, 333, 2, 0), (130, 77, 1, 1)])
def test_dense_forms_match_loops(N, T, C, enc):
    p = synth.uniform(N, T, C, seed=31)
    f = synth.flags(N, T, C, p_bad=0.25, seed=32, burst=5)
    assert np.array_equal(oracle.correlate_masked_dense(p, f, N, T, C, enc, t_chunk=64),
                          oracle.correlate_masked(p, f, N, T, C, enc))
    assert np.array_equal(oracle.flag_counts_dense(f, N, T, C, t_chunk=50),
                          oracle.flag_counts(f, N, T, C))


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        oracle.correlate_masked(np.zeros(8, np.uint8), np.zeros(3, np.uint8), 4, 2)
    with pytest.raises(ValueError):
        oracle.correlate_masked(np.zeros(8, np.uint8), None, 4, 2, 1, encoding=2)


# ---- planted mistakes ----------------------------------------------------------------------

MUTANTS = {
    "flag_of_first_input_only": ("if (!flag_valid(cf, N, t, i) || !flag_valid(cf, N, t, j)) continue;",
                                 "if (!flag_valid(cf, N, t, i)) continue;"),
    "flag_bit_order_reversed": ("return (chan_flags[t * row + n / 8] >> (n % 8)) & 1;",
                                "return (chan_flags[t * row + n / 8] >> (7 - n % 8)) & 1;"),
    "flag_polarity_inverted": ("return (chan_flags[t * row + n / 8] >> (n % 8)) & 1;",
                               "return !((chan_flags[t * row + n / 8] >> (n % 8)) & 1);"),
    "offset_as_sign_magnitude": ("*re = (int64_t)((byte >> 4) & 0xF) - 8;",
                                 "*re = ((byte >> 4) & 8) ? -(int64_t)((byte >> 4) & 7) : (int64_t)((byte >> 4) & 7);"),
    "offset_off_by_one": ("*im = (int64_t)(byte & 0xF) - 8;", "*im = (int64_t)(byte & 0xF) - 7;"),
    "counts_or_not_and": ("n += flag_valid(cf, N, t, i) & flag_valid(cf, N, t, j);",
                          "n += flag_valid(cf, N, t, i) | flag_valid(cf, N, t, j);"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, f"mutation anchor for {name} not found"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(path)])
    lib = ctypes.CDLL(str(so))
    i64, p = ctypes.c_int64, ctypes.c_void_p
    lib.xe_oracle_correlate_masked.argtypes = [p, p, i64, i64, i64, ctypes.c_int, p]
    lib.xe_oracle_flag_counts.argtypes = [p, i64, i64, i64, p]
    return lib


def _mutant_passes_pins(lib) -> bool:
    for name, enc, N, T, b, flags, vis, cnt in golden_cases():
        B = N * (N + 1) // 2
        out = np.zeros((B, 2), np.int64)
        lib.xe_oracle_correlate_masked(b.ctypes.data, None if flags is None else flags.ctypes.data,
                                       N, T, 1, enc, out.ctypes.data)
        if not np.array_equal(out, vis):
            return False
        f = flags if flags is not None else np.full(T * ((N + 7) // 8), 0xFF, np.uint8)
        c = np.zeros(B, np.int64)
        lib.xe_oracle_flag_counts(f.ctypes.data, N, T, 1, c.ctypes.data)
        if not np.array_equal(c, cnt):
            return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(tmp_path, name):
    old, new = MUTANTS[name]
    assert not _mutant_passes_pins(_build_mutant(tmp_path, name, old, new))


def test_unmutated_source_passes_pins(tmp_path):
    assert _mutant_passes_pins(_build_mutant(tmp_path, "none", "int xe_oracle_correlate_masked",
                                             "int xe_oracle_correlate_masked"))
