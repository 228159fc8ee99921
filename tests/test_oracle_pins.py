"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: values worked by hand
(tests/golden), numbers printed in the paper (Table tab:corrs), brute force with Python
complex arithmetic, closed forms (identical inputs, quarter-turn plane waves, rank one),
and algebraic invariants (Hermitian symmetry, linearity in time).  A dropped term, a
wrong sign, a transposed operand or a wrong triangle index fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2005_09481_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# --- decode -----------------------------------------------------------------------

def test_decode_golden_examples():
    rows = _lines("decode_examples.txt")
    b = np.array([int(r[0], 16) for r in rows], np.uint8)
    re, im = oracle.decode(b)
    assert re.tolist() == [int(r[1]) for r in rows]
    assert im.tolist() == [int(r[2]) for r in rows]


def test_decode_all_bytes_by_arithmetic_shift():
    # Independent mechanism: an arithmetic right shift of the byte viewed as int8
    # sign-extends the high nibble; shifting the low nibble up first does the same for it.
    b = np.arange(256, dtype=np.uint8)
    re, im = oracle.decode(b)
    hi = (b.view(np.int8) >> 4).astype(np.int64)
    lo = ((b << 4).astype(np.uint8).view(np.int8) >> 4).astype(np.int64)
    np.testing.assert_array_equal(re, hi)
    np.testing.assert_array_equal(im, lo)
    assert re.min() == -8 and re.max() == 7


def test_synth_pack_roundtrip():
    v = np.arange(-8, 8)
    re, im = np.meshgrid(v, v, indexing="ij")
    r2, i2 = oracle.decode(synth.pack(re, im))
    np.testing.assert_array_equal(r2, re)
    np.testing.assert_array_equal(i2, im)


# --- triangle layout and cMAC count ---------------------------------------------------

def test_triangle_index_is_row_major_upper_triangle():
    for N in (1, 2, 3, 7, 64):
        k = 0
        for i in range(N):
            for j in range(i, N):
                assert oracle.tri_index(N, i, j) == k
                k += 1
        assert oracle.n_baselines(N) == k


def test_eta_matches_paper_table():
    # eta = delta-nu * N(N+1)/2 (section 2.2) reproduces every consistent row of
    # Table tab:corrs to the printed precision; N^2 and N(N-1)/2 do not.
    ok = [r for r in _lines("eta_table.txt") if r[4] == "ok"]
    assert len(ok) == 10
    for name, n, dnu, printed, _ in ok:
        n, dnu = int(n), float(dnu) * 1e6
        half_ulp = 0.5 * 10 ** -(len(printed.split(".")[1]) if "." in printed else 0)
        eta = dnu * oracle.n_baselines(n) / 1e12
        assert abs(eta - float(printed)) <= half_ulp + 1e-9, name
        assert oracle.cmac(n, 1, 1) == n * (n + 1) / 2
    # the CHIME row separates N(N+1)/2 from the alternatives
    assert round(400e6 * 2048 * 2047 / 2 / 1e12) != 839
    assert round(400e6 * 2048 * 2048 / 1e12) != 839


def test_cmac_of_configs_and_paper_rates():
    # 2048 inputs: 2,098,176 baselines; one 390625 Hz channel needs 8.196e11 cMAC/s and
    # four channels per node 3.3e12 (Table tab:node-stats); 400 MHz needs 8.39e14 (section 2.2).
    assert oracle.n_baselines(2048) == 2_098_176
    assert oracle.cmac(2048, 390625, 1) == pytest.approx(8.196e11, rel=1e-3)
    assert round(oracle.cmac(2048, 390625, 4) / 1e12, 1) == 3.3
    assert round(oracle.cmac(2048, 400_000_000, 1) / 1e14, 2) == 8.39
    assert oracle.cmac(2048, 32768, 1) == 2_098_176 * 32768
    # input rate N * dnu * d with d = 8 bits: 6553 Gb/s (Table tab:data-flow), "6.6 Tb/s"
    assert abs(2048 * 400e6 * 8 / 1e9 - 6553) < 1
    # 8 bytes per visibility (int32 Re + int32 Im) at 10 s over 1024 channels is within
    # 1 % of the 13.6 Gb/s printed in Table tab:data-flow
    rate = 1024 * oracle.n_baselines(2048) * 8 * 8 / 10.0
    assert abs(rate / 13.6e9 - 1) < 0.015


# --- hand-worked visibilities -----------------------------------------------------------

@pytest.mark.parametrize("row", _lines("hand_visibilities.txt"), ids=lambda r: r[0])
def test_hand_worked_visibilities(row):
    bar = [k for k, tok in enumerate(row) if tok == "|"]
    N, T = int(row[1]), int(row[2])
    b = np.array([int(x, 16) for x in row[bar[0] + 1:bar[1]]], np.uint8)
    want = np.array([[int(v) for v in p.split(",")] for p in row[bar[1] + 1:]], np.int64)
    got = oracle.correlate64(b, N, T, 1)[0]
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(oracle.correlate_dense(b, N, T, 1)[0], want)


# --- brute force -----------------------------------------------------------------------

def _brute(packed, N, T):
    """Pure-Python complex arithmetic on values decoded by the int8-shift mechanism."""
    b = packed.reshape(T, N)
    hi = (b.view(np.int8) >> 4).astype(int)
    lo = ((b << 4).astype(np.uint8).view(np.int8) >> 4).astype(int)
    out = []
    for i in range(N):
        for j in range(i, N):
            s = 0j
            for t in range(T):
                s += complex(hi[t, i], lo[t, i]) * complex(hi[t, j], lo[t, j]).conjugate()
            out.append((int(s.real), int(s.imag)))
    return np.array(out, np.int64)


def test_brute_force_all_byte_pairs_rank_one():
    # N = 2, T = 1: every pair of bytes (65,536 cases) through V_01 = x0 conj(x1).
    a, b = np.meshgrid(np.arange(256, dtype=np.uint8), np.arange(256, dtype=np.uint8),
                       indexing="ij")
    C = a.size
    packed = np.stack([a.ravel(), b.ravel()], axis=1).reshape(C, 1, 2)
    got = oracle.correlate64(packed, 2, 1, C)
    hi = (packed.view(np.int8) >> 4).astype(np.int64).reshape(C, 2)
    lo = ((packed << 4).astype(np.uint8).view(np.int8) >> 4).astype(np.int64).reshape(C, 2)
    x = hi + 1j * lo
    v01 = x[:, 0] * np.conj(x[:, 1])
    np.testing.assert_array_equal(got[:, 1, 0], v01.real.astype(np.int64))
    np.testing.assert_array_equal(got[:, 1, 1], v01.imag.astype(np.int64))
    np.testing.assert_array_equal(got[:, 0, 0], hi[:, 0] ** 2 + lo[:, 0] ** 2)
    np.testing.assert_array_equal(got[:, 0, 1], 0)


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_random_small(seed):
    rng = np.random.default_rng(seed)
    N, T = int(rng.integers(1, 9)), int(rng.integers(1, 17))
    packed = rng.integers(0, 256, size=(T, N), dtype=np.uint8)   # full [-8, 7] range
    np.testing.assert_array_equal(oracle.correlate64(packed, N, T, 1)[0], _brute(packed, N, T))


def test_c_loop_and_dense_form_agree():
    for (N, T, C, seed) in [(17, 33, 2, 1), (64, 1024, 1, 2), (96, 300, 3, 3)]:
        packed = synth.uniform(N, T, C, seed)
        np.testing.assert_array_equal(oracle.correlate(packed, N, T, C),
                                      oracle.correlate_dense(packed, N, T, C, t_chunk=100))


def test_pairs_match_full():
    N, T, C = 40, 77, 3
    packed = synth.gauss_plane(N, T, C, 5)
    full = oracle.correlate64(packed, N, T, C)
    rng = np.random.default_rng(0)
    c = rng.integers(0, C, 50)
    i = rng.integers(0, N, 50)
    j = np.array([rng.integers(a, N) for a in i])
    got = oracle.pairs(packed, N, T, C, c, i, j)
    idx = [oracle.tri_index(N, a, b) for a, b in zip(i, j)]
    np.testing.assert_array_equal(got, full[c, idx])


# --- closed forms and invariants ----------------------------------------------------------

def test_hermitian_and_diagonal():
    N, T = 23, 41
    packed = synth.uniform(N, T, 1, 7)
    V = oracle.unpack_triangle(oracle.correlate64(packed, N, T, 1)[0], N)
    X = oracle.voltages(packed[0], N, T)
    # the lower triangle is the conjugate of the upper one; compare against X X^H
    np.testing.assert_array_equal(V, X @ X.conj().T)
    np.testing.assert_array_equal(np.diag(V).imag, 0)
    np.testing.assert_array_equal(np.diag(V).real, (X.real ** 2 + X.imag ** 2).sum(axis=1))


def test_identical_inputs():
    # x_i(t) = s(t) for all i  =>  V_ij = sum_t |s(t)|^2, Im = 0.
    N, T = 9, 50
    rng = np.random.default_rng(3)
    s = rng.integers(-7, 8, size=(T, 2))
    packed = np.repeat(synth.pack(s[:, 0], s[:, 1])[:, None], N, axis=1)
    v = oracle.correlate64(packed, N, T, 1)[0]
    assert (v[:, 0] == int((s ** 2).sum())).all()
    assert (v[:, 1] == 0).all()


def test_quarter_turn_plane_wave():
    # x_i(t) = s(t) * i^{k_i}, k_i = (m*i) mod 4: an exact integer phase ramp across the
    # inputs.  Closed form: V_ij = sum_t |s(t)|^2 * i^{k_i - k_j}.
    N, T, m = 11, 64, 3
    rng = np.random.default_rng(4)
    s = rng.integers(-7, 8, size=T) + 1j * rng.integers(-7, 8, size=T)
    k = (m * np.arange(N)) % 4
    x = s[:, None] * (1j ** k)[None, :]
    packed = synth.pack(np.rint(x.real).astype(int), np.rint(x.imag).astype(int))
    v = oracle.correlate64(packed, N, T, 1)[0]
    S = int((s.real ** 2 + s.imag ** 2).sum())
    for i in range(N):
        for j in range(i, N):
            want = S * (1j ** ((k[i] - k[j]) % 4))
            got = v[oracle.tri_index(N, i, j)]
            assert (got[0], got[1]) == (int(want.real), int(want.imag))


def test_linearity_in_time():
    N, T1, T2 = 13, 30, 45
    a = synth.uniform(N, T1, 1, 11)
    b = synth.uniform(N, T2, 1, 12)
    both = np.concatenate([a, b], axis=1)
    np.testing.assert_array_equal(oracle.correlate64(both, N, T1 + T2, 1),
                                  oracle.correlate64(a, N, T1, 1) + oracle.correlate64(b, N, T2, 1))


def test_channels_independent():
    N, T = 10, 20
    p = synth.uniform(N, T, 3, 21)
    full = oracle.correlate64(p, N, T, 3)
    for c in range(3):
        np.testing.assert_array_equal(full[c], oracle.correlate64(p[c], N, T, 1)[0])


def test_extremes_and_int32_bound():
    # all 7+7i: Re V = 98 T; all -8-8i: Re V = 128 T; Im = 0 for both.
    for (re, im, per) in [(7, 7, 98), (-8, -8, 128)]:
        T = 65536
        v = oracle.correlate64(synth.constant(3, T, re, im), 3, T, 1)[0]
        assert (v[:, 0] == per * T).all() and (v[:, 1] == 0).all()
    # max |Im| per sample: (a+ib)(p-iq) with a=-8,b=7,p=-8,q=-8 -> Im = b p - a q = -56-64
    v = oracle.correlate64(np.array([[synth.pack(-8, 7), synth.pack(-8, -8)]], np.uint8), 2, 1, 1)[0]
    assert tuple(v[1]) == (64 - 56, -56 - 64)
    big = np.array([[[2 ** 31]]], np.int64)
    with pytest.raises(OverflowError):
        oracle.to_int32(big)


def test_empty_time_axis():
    v = oracle.correlate64(np.zeros((0, 4), np.uint8), 4, 0, 1)
    assert v.shape == (1, 10, 2) and not v.any()
