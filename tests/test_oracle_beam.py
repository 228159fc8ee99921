"""Pins of the phased-array beamforming oracle (CPU only).

The paper names the product (section 2.1: 10 phased-array beams for pulsar timing; Table
tab:computing: "Pulsar Beamforming") but prints no formula; the reading is the weighted
coherent sum y_b(t) = sum_i w_{b,i} x_i(t) with int8 complex weights.  What fixes the oracle:
* hand-computed sums (tests/golden/beam_hand.txt);
* pure-Python brute force on tiny inputs over the full byte and weight ranges;
* closed forms: a one-hot weight selects an input; a phased array whose weights undo an
  exact quarter-turn phase ramp adds N inputs coherently (gain N), and a ramp it does not
  match cancels to zero;
* a relation to the correlation oracle (pinned on its own): the beam power
  sum_t |y_b(t)|^2 equals w^T V conj(w) with V the visibility matrix;
* planted mistakes, each caught by one of the pins above.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2005_09481_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden", "beam_hand.txt")
SRC = os.path.join(ROOT, "oracle", "xe_oracle.c")


def golden_cases():
    out = []
    with open(GOLDEN) as f:
        for ln in f:
            if not ln.strip() or ln.startswith("#"):
                continue
            parts = [p.split() for p in ln.split("|")]
            N, T, B = map(int, parts[0])
            b = np.array([int(x, 16) for x in parts[1]], np.uint8)
            w = np.array([[int(v) for v in p.split(",")] for p in parts[2]], np.int8).reshape(B, N, 2)
            y = np.array([[int(v) for v in p.split(",")] for p in parts[3]], np.int64).reshape(T, B, 2)
            out.append((N, T, B, b, w, y))
    return out


@pytest.mark.parametrize("case", golden_cases())
def test_golden_hand_sums(case):
    N, T, B, b, w, y = case
    assert np.array_equal(oracle.beamform(b, w, N, T, 1, B)[0], y)
    assert np.array_equal(oracle.beamform_dense(b, w, N, T, 1, B)[0], y)


def _val(byte):
    hi, lo = byte >> 4, byte & 0xF
    return complex(hi - 16 if hi >= 8 else hi, lo - 16 if lo >= 8 else lo)


def test_brute_force_python():
    rng = np.random.default_rng(17)
    for _ in range(8):
        N, T, B = int(rng.integers(1, 6)), int(rng.integers(1, 5)), int(rng.integers(1, 4))
        b = rng.integers(0, 256, size=(T, N)).astype(np.uint8)
        w = rng.integers(-127, 128, size=(B, N, 2)).astype(np.int8)
        want = np.zeros((T, B, 2), np.int64)
        for t in range(T):
            for k in range(B):
                s = 0j
                for i in range(N):
                    s += complex(int(w[k, i, 0]), int(w[k, i, 1])) * _val(int(b[t, i]))
                want[t, k] = (int(s.real), int(s.imag))
        assert np.array_equal(oracle.beamform(b, w, N, T, 1, B)[0], want)


def test_one_hot_weight_selects_an_input():
    N, T = 13, 40
    p = synth.uniform(N, T, 1, seed=3)
    sel = [0, 5, 12]
    w = np.zeros((len(sel), N, 2), np.int8)
    for k, s in enumerate(sel):
        w[k, s, 0] = 1
    y = oracle.beamform(p, w, N, T, 1, len(sel))[0]
    re, im = oracle.decode(p[0])
    for k, s in enumerate(sel):
        assert np.array_equal(y[:, k, 0], re[:, s]) and np.array_equal(y[:, k, 1], im[:, s])


def test_phased_array_coherent_gain_and_null():
    # x_i(t) = s(t) * i^(m i): an exact quarter-turn phase ramp across the array.  Weights
    # i^(-m i) undo it, so y(t) = N s(t); weights of another ramp m' != m (mod 4) sum a full
    # set of quarter turns per 4 inputs and cancel exactly when N is a multiple of 4.
    N, T, m = 32, 50, 1
    rng = np.random.default_rng(5)
    s = rng.integers(-3, 4, size=(T, 2))
    unit = [1, 1j, -1, -1j]
    x = np.empty((T, N), np.complex128)
    for i in range(N):
        x[:, i] = (s[:, 0] + 1j * s[:, 1]) * unit[(m * i) % 4]
    p = synth.pack(np.rint(x.real).astype(int), np.rint(x.imag).astype(int)).reshape(1, T, N)

    def ramp_weights(mm):
        w = np.zeros((1, N, 2), np.int8)
        for i in range(N):
            u = unit[(-mm * i) % 4]
            w[0, i] = (int(u.real), int(u.imag))
        return w

    y = oracle.beamform(p, ramp_weights(m), N, T, 1, 1)[0, :, 0]
    assert np.array_equal(y[:, 0], N * s[:, 0]) and np.array_equal(y[:, 1], N * s[:, 1])
    null = oracle.beamform(p, ramp_weights(m + 1), N, T, 1, 1)[0, :, 0]
    assert not null.any()


def test_beam_power_equals_quadratic_form_of_visibilities():
    N, T, B = 24, 300, 3
    p = synth.gauss_plane(N, T, 1, seed=8)
    w = synth.beam_weights(B, N, seed=9, amp=20)
    y = oracle.beamform(p, w, N, T, 1, B)[0]
    V = oracle.unpack_triangle(oracle.correlate(p, N, T)[0], N)        # V_ij, Hermitian
    for k in range(B):
        wc = w[k, :, 0].astype(np.int64) + 1j * w[k, :, 1].astype(np.int64)
        power = int((y[:, k, 0] ** 2 + y[:, k, 1] ** 2).sum())
        quad = wc @ V @ np.conj(wc)
        assert abs(quad.imag) < 1e-6 and int(round(quad.real)) == power


def test_linearity_in_weights():
    N, T = 40, 64
    p = synth.uniform(N, T, 1, seed=2)
    w1 = synth.beam_weights(2, N, seed=1, amp=60)
    w2 = synth.beam_weights(2, N, seed=2, amp=60)
    ws = (w1.astype(np.int16) + w2.astype(np.int16)).astype(np.int8)
    assert np.array_equal(oracle.beamform(p, ws, N, T, 1, 2),
                          oracle.beamform(p, w1, N, T, 1, 2) + oracle.beamform(p, w2, N, T, 1, 2))


@pytest.mark.parametrize("N,T,C,B", [(70, 33, 2, 3), (256, 500, 1, 10)])
def test_dense_matches_loop(N, T, C, B):
    p = synth.gauss_plane(N, T, C, seed=4)
    w = synth.beam_weights(B, N, seed=6)
    assert np.array_equal(oracle.beamform_dense(p, w, N, T, C, B, t_chunk=100),
                          oracle.beamform(p, w, N, T, C, B))


def test_weights_generator_range():
    w = synth.beam_weights(10, 2048)
    assert w.dtype == np.int8 and w.min() >= -127 and w.max() <= 127
    mag = np.hypot(w[..., 0].astype(float), w[..., 1].astype(float))
    assert 120 < mag.mean() < 132


MUTANTS = {
    "conjugated_weight": ("acc_re += wr * a - wi * bb;", "acc_re += wr * a + wi * bb;"),
    "imag_cross_sign": ("acc_im += wr * bb + wi * a;", "acc_im += wr * bb - wi * a;"),
    "dropped_imag_term": ("acc_im += wr * bb + wi * a;", "acc_im += wr * bb;"),
    "beam_input_transposed": ("const int64_t wr = w[(b * N + i) * 2 + 0], wi = w[(b * N + i) * 2 + 1];",
                              "const int64_t wr = w[(i * B + b) * 2 + 0], wi = w[(i * B + b) * 2 + 1];"),
    "output_time_beam_swapped": ("y[((c * T + t) * B + b) * 2 + 0] = acc_re;",
                                 "y[((c * B + b) * T + t) * 2 + 0] = acc_re;"),
}


def _mutant_passes(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(path)])
    lib = ctypes.CDLL(str(so))
    i64, p = ctypes.c_int64, ctypes.c_void_p
    lib.xe_oracle_beamform.argtypes = [p, p, i64, i64, i64, i64, p]
    for N, T, B, b, w, y in golden_cases():
        out = np.full((T, B, 2), -99, np.int64)
        lib.xe_oracle_beamform(b.ctypes.data, w.ctypes.data, N, T, 1, B, out.ctypes.data)
        if not np.array_equal(out, y):
            return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(tmp_path, name):
    assert not _mutant_passes(tmp_path, name, *MUTANTS[name])


def test_unmutated_passes(tmp_path):
    assert _mutant_passes(tmp_path, "none", "int xe_oracle_beamform", "int xe_oracle_beamform")
