"""Pins of the corner-turn and pre-sum oracle (CPU only).

Section 2.1 of the paper: the F-engine delivers bundles of four frequency channels, each with
one cylinder's inputs, and every GPU node combines four bundles into full-array data;
Table tab:computing lists the GPU task "Re-Order and Pre-Sum".  The byte layout of a bundle
and the meaning of the pre-sum are readings (a bundle is [T][n_freq][n_in] of one cylinder;
the pre-sum is the per-input time sum of re and im).  What fixes the oracle:
* a hand-worked case (tests/golden/corner_hand.txt);
* the inverse written independently (numpy reshape/transpose in synth.bundles_of);
* the visibilities of a cylinder's own inputs: the corner-turned frame's cylinder-diagonal
  block of V equals the correlation of that cylinder's bundle alone (correlation oracle
  pinned separately);
* the pre-sum: constant input gives T x; an all-ones beam sums to the sum of the pre-sums
  (beam oracle pinned separately); pure-Python brute force;
* planted mistakes caught by the above.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2005_09481_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden", "corner_hand.txt")
SRC = os.path.join(ROOT, "oracle", "xe_oracle.c")


def golden():
    d = {}
    with open(GOLDEN) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                k, *v = ln.split()
                d[k] = v
    b = np.array([int(x, 16) for x in d["bundles"]], np.uint8)
    fr = np.array([int(x, 16) for x in d["frames"]], np.uint8).reshape(2, 2, 4)
    ps = np.array([[int(v) for v in p.split(",")] for p in d["presum"]], np.int64).reshape(2, 4, 2)
    return b, fr, ps


def test_golden_hand_case():
    b, fr, ps = golden()
    assert np.array_equal(oracle.corner_turn(b, 2, 2, 2, 2), fr)
    assert np.array_equal(oracle.presum(fr, 4, 2, 2), ps)


@pytest.mark.parametrize("n_cyl,n_freq,n_in,T", [(4, 4, 512, 8), (3, 2, 5, 7), (1, 1, 1, 1), (4, 1, 16, 33)])
def test_inverse_round_trip(n_cyl, n_freq, n_in, T):
    frames = synth.uniform(n_cyl * n_in, T, n_freq, seed=n_cyl + T)
    b = synth.bundles_of(frames, n_cyl)
    assert b.shape == (n_cyl, T, n_freq, n_in)
    assert np.array_equal(oracle.corner_turn(b, n_cyl, n_freq, n_in, T), frames)


def test_cylinder_block_of_visibilities():
    n_cyl, n_freq, n_in, T = 3, 2, 16, 64
    rng = np.random.default_rng(4)
    b = rng.integers(0, 256, size=(n_cyl, T, n_freq, n_in)).astype(np.uint8)
    frames = oracle.corner_turn(b, n_cyl, n_freq, n_in, T)
    N = n_cyl * n_in
    for f in range(n_freq):
        V = oracle.unpack_triangle(oracle.correlate(frames[f], N, T)[0], N)
        for cyl in range(n_cyl):
            own = np.ascontiguousarray(b[cyl, :, f, :])
            W = oracle.unpack_triangle(oracle.correlate(own, n_in, T)[0], n_in)
            blk = slice(cyl * n_in, (cyl + 1) * n_in)
            assert np.array_equal(V[blk, blk], W)


def test_presum_closed_forms_and_beam_relation():
    N, T = 40, 300
    assert np.array_equal(oracle.presum(synth.constant(N, T, -8, 7), N, T)[0],
                          np.tile([-8 * T, 7 * T], (N, 1)))
    p = synth.gauss_plane(N, T, 1, seed=5)
    s = oracle.presum(p, N, T)[0]
    w = np.zeros((1, N, 2), np.int8)
    w[..., 0] = 1
    y = oracle.beamform(p, w, N, T, 1, 1)[0, :, 0]           # y(t) = sum_n x_n(t)
    assert y[:, 0].sum() == s[:, 0].sum() and y[:, 1].sum() == s[:, 1].sum()
    half = T // 2
    a = oracle.presum(np.ascontiguousarray(p[0, :half]), N, half)[0]
    b = oracle.presum(np.ascontiguousarray(p[0, half:]), N, T - half)[0]
    assert np.array_equal(a + b, s)


def test_presum_brute_force():
    rng = np.random.default_rng(2)
    N, T, C = 5, 9, 2
    fr = rng.integers(0, 256, size=(C, T, N)).astype(np.uint8)

    def val(x):
        hi, lo = x >> 4, x & 15
        return (hi - 16 if hi >= 8 else hi), (lo - 16 if lo >= 8 else lo)

    want = np.zeros((C, N, 2), np.int64)
    for c in range(C):
        for t in range(T):
            for n in range(N):
                r, i = val(int(fr[c, t, n]))
                want[c, n] += (r, i)
    assert np.array_equal(oracle.presum(fr, N, T, C), want)


MUTANTS = {
    "freq_cyl_swapped": ("bundles[((cyl * T + t) * n_freq + f) * n_in + i];",
                         "bundles[((f * T + t) * n_cyl + cyl) * n_in + i];"),
    "input_order_reversed": ("frames[(f * T + t) * N + cyl * n_in + i] =",
                             "frames[(f * T + t) * N + (n_cyl - 1 - cyl) * n_in + i] ="),
    "presum_re_im_swapped": ("sums[(c * N + n) * 2 + 0] = sr;", "sums[(c * N + n) * 2 + 0] = si;"),
    "presum_drops_last_sample": ("for (int64_t t = 0; t < T; ++t) {\n                int64_t a, b;",
                                 "for (int64_t t = 0; t + 1 < T; ++t) {\n                int64_t a, b;"),
}


def _passes(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(path)])
    lib = ctypes.CDLL(str(so))
    i64, p = ctypes.c_int64, ctypes.c_void_p
    lib.xe_oracle_corner_turn.argtypes = [p, i64, i64, i64, i64, p]
    lib.xe_oracle_presum.argtypes = [p, i64, i64, i64, p]
    b, fr, ps = golden()
    out = np.zeros(16, np.uint8)
    lib.xe_oracle_corner_turn(b.ctypes.data, 2, 2, 2, 2, out.ctypes.data)
    sums = np.zeros((2, 4, 2), np.int64)
    frc = np.ascontiguousarray(fr)
    lib.xe_oracle_presum(frc.ctypes.data, 4, 2, 2, sums.ctypes.data)
    return np.array_equal(out.reshape(2, 2, 4), fr) and np.array_equal(sums, ps)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(tmp_path, name):
    assert not _passes(tmp_path, name, *MUTANTS[name])


def test_unmutated_passes(tmp_path):
    assert _passes(tmp_path, "none", "int xe_oracle_presum", "int xe_oracle_presum")
