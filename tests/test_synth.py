"""The seeded input generators against the recipe they state: value ranges, distributions,
the plane wave's phase ramp across inputs, flag rates and bursts, steering weights, uneven
shapes and the bundle layout.  (Host only; no correlation arithmetic is involved.)"""
import numpy as np
import pytest

from paper_2005_09481_gb300 import synth


def unpack(b):
    b = np.asarray(b, np.uint8).astype(np.int16)
    return ((b >> 4) ^ 8) - 8, ((b & 15) ^ 8) - 8


def test_pack_is_twos_complement_high_nibble_real():
    assert synth.pack(np.array(1), np.array(-1)) == 0x1F
    assert synth.pack(np.array(-8), np.array(7)) == 0x87
    with pytest.raises(ValueError):
        synth.pack(np.array(8), np.array(0))


def test_uniform_range_frequencies_and_seeds():
    p = synth.uniform(64, 4096, 2)
    re, im = unpack(p)
    assert re.min() == -7 and re.max() == 7 and im.min() == -7 and im.max() == 7
    freq = np.bincount((re + 7).ravel(), minlength=15) / re.size
    assert np.abs(freq - 1 / 15).max() < 0.01
    assert np.array_equal(p, synth.uniform(64, 4096, 2))                # reproducible
    assert np.array_equal(p[1], synth.uniform(64, 4096, 1, seed=synth.BASE_SEED + 1)[0])
    assert not np.array_equal(p[0], p[1])                                # channel c: seed + c


def test_gauss_plane_statistics_and_phase_ramp():
    N, T, k = 64, 8192, 3
    p = synth.gauss_plane(N, T, 1)
    re, im = unpack(p[0])
    assert re.min() >= -7 and re.max() <= 7 and im.min() >= -7 and im.max() <= 7
    # Per component: noise sigma 2.5 plus half the sky power A^2 / 2 = 4.5 (clipping at +-7
    # trims a little).
    for comp in (re, im):
        assert abs(comp.mean()) < 0.05
        assert 2.9 < comp.std() < 3.4
    # The common sky term gives <x_i conj x_j> ~ A^2 exp(i 2 pi k (i - j) / N).
    x = re + 1j * im
    for j in (1, 5, 11, 21):
        m = np.mean(x[:, 0] * np.conj(x[:, j]))
        want = 2 * np.pi * k * (0 - j) / N
        assert abs(np.angle(m * np.exp(-1j * want))) < 0.1
        assert 6.0 < abs(m) < 9.5
    # Independent noise: the autocorrelation exceeds the cross-correlation by sigma^2-ish.
    auto = np.mean(np.abs(x[:, 0]) ** 2)
    assert auto - abs(np.mean(x[:, 0] * np.conj(x[:, 1]))) > 8.0


def test_flags_rate_bursts_and_padding():
    N, T = 20, 20000
    f = synth.flags(N, T, 1, p_bad=0.1)
    valid = np.unpackbits(f, axis=2, bitorder="little")[..., :N].astype(bool)
    assert abs(valid.mean() - 0.9) < 0.01
    pad = np.unpackbits(f, axis=2, bitorder="little")[..., N:]
    assert not pad.any()                                     # bits past N are zero
    fb = synth.flags(N, T, 1, p_bad=0.0, burst=64)
    vb = np.unpackbits(fb, axis=2, bitorder="little")[0, :, :N].astype(bool)
    rows = vb.all(axis=1)
    assert (vb.any(axis=1) == rows).all()                    # a burst flags every input
    assert 0 < (~rows).sum() <= (T // (64 * 20)) * 64        # at most T / 1280 bursts
    # Every maximal run of flagged samples is at least one burst long (bursts may overlap),
    # unless the data ends inside it.
    edges = np.flatnonzero(np.diff(np.concatenate([[0], (~rows).astype(np.int8), [0]])))
    for start, stop in zip(edges[0::2], edges[1::2]):
        assert stop - start >= 64 or stop == T


def test_offset_binary_is_an_involution_on_values():
    p = synth.uniform(32, 100, 1)
    ob = synth.to_offset_binary(p)
    assert np.array_equal(synth.to_offset_binary(ob), p)
    u = ob.astype(np.int16)
    re, im = unpack(p)
    assert np.array_equal((u >> 4) - 8, re) and np.array_equal((u & 15) - 8, im)


def test_beam_weights_magnitude_and_linear_phase():
    B, N = 10, 256
    w = synth.beam_weights(B, N)
    c = w[..., 0].astype(float) + 1j * w[..., 1]
    assert np.abs(w).max() <= 127
    assert np.abs(np.abs(c) - 127).max() < 1.0
    d = np.angle(c[:, 1:] * np.conj(c[:, :-1]))               # constant step per input
    assert (np.abs(d - d[:, :1]) < 0.02).all()
    assert np.array_equal(w, synth.beam_weights(B, N))


def test_uneven_shapes_choices_and_seed():
    s = synth.uneven_shapes(64)
    assert len(s) == 64 and s == synth.uneven_shapes(64)
    assert {n for n, _ in s} <= set(synth.UNEVEN_N) and {t for _, t in s} <= set(synth.UNEVEN_T)
    assert len({n for n, _ in s}) > 1 and len({t for _, t in s}) > 1


def test_bundles_hold_one_cylinder_each():
    n_cyl, n_freq, n_in, T = 4, 2, 8, 5
    frames = synth.uniform(n_cyl * n_in, T, n_freq)
    b = synth.bundles_of(frames, n_cyl)
    assert b.shape == (n_cyl, T, n_freq, n_in)
    for cyl in range(n_cyl):
        for f in range(n_freq):
            assert np.array_equal(b[cyl, :, f, :], frames[f, :, cyl * n_in:(cyl + 1) * n_in])
