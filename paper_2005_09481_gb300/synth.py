"""Seeded synthetic channelised voltages (input generators only).

This module holds no correlation arithmetic: it draws integer sample values and packs
them into the 4+4-bit byte format (Denman et al. 2020, section 2.2: 4 bits real and
4 bits imaginary, d = 8 bits).  Both the CUDA path and the CPU oracle consume the bytes
it produces, so its rounding choices never affect parity; they are fixed only for
reproducibility.

Byte layout: high nibble = real part, low nibble = imaginary part, two's complement.
Layout of a batch: uint8 [C][T][N] (per channel, per time sample, all N inputs
contiguous: the corner-turned order in which the X-engine receives data, section 2.3).

Workload recipes (the CHIME shapes: N = 2048 inputs, 390625 samples/s per channel):
* ``uniform``: re, im i.i.d. uniform integers in [-7, 7].
* ``gauss_plane``: per component a Gaussian of sigma = 2.5 levels, plus a common sky
  term A * s(t) * exp(i (2 pi k n / N + phi0)) with s(t) a unit complex Gaussian,
  A = 3, k = 3, phi0 drawn from the seed; round half to even, clip to [-7, 7].  The
  linear phase ramp across inputs makes off-diagonal visibilities nonzero (it mirrors
  the linear phase evolution of a transiting source, section 3, first light).
* ``uneven_batch``: instance shapes drawn from N in {256, 512, 1024, 2048} and
  T in {4096, 8192, 32768, 65536}, uniform values.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20050948


def pack(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Integer arrays with values in [-8, 7] -> packed uint8 bytes."""
    r = np.asarray(re).astype(np.int16)
    i = np.asarray(im).astype(np.int16)
    if r.size and (r.min() < -8 or r.max() > 7 or i.min() < -8 or i.max() > 7):
        raise ValueError("4-bit values must lie in [-8, 7]")
    return (((r & 0xF) << 4) | (i & 0xF)).astype(np.uint8)


def uniform(N: int, T: int, C: int = 1, seed: int = BASE_SEED) -> np.ndarray:
    """uint8 [C][T][N], re and im uniform in [-7, 7]; channel c uses seed + c."""
    out = np.empty((C, T, N), np.uint8)
    for c in range(C):
        rng = np.random.default_rng(seed + c)
        v = rng.integers(-7, 8, size=(T, N, 2), dtype=np.int8)
        out[c] = pack(v[..., 0], v[..., 1])
    return out


def gauss_plane(N: int, T: int, C: int = 1, seed: int = BASE_SEED,
                sigma: float = 2.5, amp: float = 3.0, k: int = 3) -> np.ndarray:
    """uint8 [C][T][N]: quantised Gaussian noise plus a plane wave; channel c uses seed + c."""
    out = np.empty((C, T, N), np.uint8)
    n = np.arange(N, dtype=np.float32)
    for c in range(C):
        rng = np.random.default_rng(seed + c)
        phi0 = np.float32(rng.uniform(0.0, 2.0 * np.pi))
        s = (rng.standard_normal(T, dtype=np.float32)
             + 1j * rng.standard_normal(T, dtype=np.float32)).astype(np.complex64)
        s *= np.float32(amp / np.sqrt(2.0))
        ramp = np.exp(1j * (2.0 * np.pi * k * n / N + phi0)).astype(np.complex64)
        noise = rng.standard_normal((T, N, 2), dtype=np.float32)
        noise *= np.float32(sigma)
        sky = s[:, None] * ramp[None, :]
        re = np.clip(np.rint(noise[..., 0] + sky.real), -7, 7).astype(np.int8)
        im = np.clip(np.rint(noise[..., 1] + sky.imag), -7, 7).astype(np.int8)
        out[c] = pack(re, im)
    return out


UNEVEN_N = (256, 512, 1024, 2048)
UNEVEN_T = (4096, 8192, 32768, 65536)


def uneven_shapes(n_inst: int = 64, seed: int = BASE_SEED,
                  n_choices=UNEVEN_N, t_choices=UNEVEN_T) -> list[tuple[int, int]]:
    """Seeded (N, T) draws for the uneven sub-array batch."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(n_choices), size=n_inst)
    ts = rng.choice(np.asarray(t_choices), size=n_inst)
    return [(int(a), int(b)) for a, b in zip(ns, ts)]


def uneven_batch(n_inst: int = 64, seed: int = BASE_SEED, shapes=None) -> list[np.ndarray]:
    """List of uint8 [1][T][N] arrays, instance q drawn with seed + 1 + q."""
    shapes = shapes if shapes is not None else uneven_shapes(n_inst, seed)
    return [uniform(N, T, 1, seed + 1 + q) for q, (N, T) in enumerate(shapes)]


def constant(N: int, T: int, re: int, im: int, C: int = 1) -> np.ndarray:
    """Every sample equal to re + i im (extreme-magnitude cases)."""
    return np.full((C, T, N), pack(np.array(re), np.array(im)), np.uint8)


def flags(N: int, T: int, C: int = 1, p_bad: float = 0.1, seed: int = BASE_SEED,
          burst: int = 0) -> np.ndarray:
    """Validity bits uint8 [C][T][ceil(N/8)] (bit n%8 of byte n/8; 1 = valid): each
    (sample, input) is flagged independently with probability p_bad; with burst > 0, whole
    time samples are also flagged in runs of `burst` (RFI-like)."""
    rng = np.random.default_rng(seed + 7919)
    valid = rng.random((C, T, N)) >= p_bad
    if burst > 0 and T > 0:
        starts = rng.integers(0, T, size=max(1, T // (burst * 20)))
        for c in range(C):
            for s in starts:
                valid[c, s:s + burst, :] = False
    pad = (-N) % 8
    if pad:
        valid = np.concatenate([valid, np.zeros((C, T, pad), bool)], axis=2)
    return np.packbits(valid, axis=2, bitorder="little")


def to_offset_binary(packed: np.ndarray) -> np.ndarray:
    """The same sample values written with offset-binary nibbles (value = nibble - 8)."""
    return (np.asarray(packed, np.uint8) ^ np.uint8(0x88)).astype(np.uint8)


def beam_weights(B: int, N: int, seed: int = BASE_SEED, amp: int = 127) -> np.ndarray:
    """Phased-array steering weights int8 [B][N][2] {re, im}: beam b steers to a seeded
    phase gradient, w_{b,i} = amp * exp(-i (2 pi k_b i / N + phi_b)), rounded half to even
    and clipped to [-127, 127]."""
    rng = np.random.default_rng(seed + 104729)
    k = rng.uniform(-N / 8, N / 8, size=B)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=B)
    i = np.arange(N)
    ph = 2.0 * np.pi * k[:, None] * i[None, :] / N + phi[:, None]
    w = np.empty((B, N, 2), np.int8)
    w[..., 0] = np.clip(np.rint(amp * np.cos(ph)), -127, 127).astype(np.int8)
    w[..., 1] = np.clip(np.rint(-amp * np.sin(ph)), -127, 127).astype(np.int8)
    return w


def bundles_of(frames: np.ndarray, n_cyl: int) -> np.ndarray:
    """Split full-array frames uint8 [n_freq][T][N] into per-cylinder bundles uint8
    [n_cyl][T][n_freq][N / n_cyl] (the F-engine's delivery format read as R13): cylinder
    `cyl` holds inputs cyl * (N / n_cyl) .. +N / n_cyl - 1 of every frequency."""
    f = np.asarray(frames, np.uint8)
    n_freq, T, N = f.shape
    n_in = N // n_cyl
    if n_in * n_cyl != N:
        raise ValueError("N must be a multiple of n_cyl")
    return np.ascontiguousarray(f.reshape(n_freq, T, n_cyl, n_in).transpose(2, 1, 0, 3))
