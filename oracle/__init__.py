"""CPU oracle for the CHIME X-engine correlation.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(``cpu_baseline`` and ``--impl reference``) may import this package.  The product
path (``paper_2005_09481_gb300``) never imports it and shares no code with it.

Two forms of the same definition, V_ij = sum_t x_i(t) conj(x_j(t)) for i <= j
(Denman et al. 2020, section 1 and section 2.2; 4-bit real + 4-bit imaginary samples,
section 2.2; channels independent, section 2.3):

* ``correlate`` / ``pairs``: the plain C triple loop in ``xe_oracle.c`` (int64).
* ``correlate_dense``: the definition written as the matrix product V = X X^H with a
  library complex128 matmul.  It is exact, not approximate: every product and every
  partial sum is an integer of magnitude below 2 * 64 * T, far below 2**53, so no
  floating-point rounding can occur in any summation order.  It exists so that full
  outputs at N=2048 can be checked in seconds; tests pin it to the C loop.

Readings where the paper is silent: high nibble = real, low nibble = imaginary, two's
complement, conjugate on the second index, row-major packed upper triangle with {Re, Im}
interleaved.

Phased-array beams (section 2.1; "Pulsar Beamforming" in Table tab:computing):
``beamform`` (C loop) and ``beamform_dense`` (library matmul), y_b(t) = sum_i w_{b,i} x_i(t)
with int8 complex weights (reading: the paper gives no formula or weight format).

Corner turn and pre-sum (section 2.1 bundles of four frequencies per cylinder, section 2.3
transpose, "Re-Order and Pre-Sum" in Table tab:computing): ``corner_turn`` and ``presum``
(C loops).  Readings: bundle = [T][n_freq][n_in] of one cylinder, full-array input
n = cyl * n_in + i; pre-sum = per-input time sums of re and im.

Flag-masked correlation (flags travel with the data, section 2.2 and Table
tab:data-flow; RFI excision precedes correlation, Table tab:computing):
``correlate_masked`` / ``flag_counts`` (C loops) and ``correlate_masked_dense`` /
``flag_counts_dense`` (library matmuls of the masked voltages and of the 0/1 validity
matrix).  Readings: one validity bit per (sample, input), bit n%8 of byte n/8, 1 = valid;
a sample counts only where both inputs are valid; offset-binary nibbles encode u - 8.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xe_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libxe_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc -O2 -fopenmp, plain C; no target-specific flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-std=c11", "-fPIC", "-shared",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, p = ctypes.c_int64, ctypes.c_void_p
            lib.xe_oracle_decode.argtypes = [p, i64, p, p]
            lib.xe_oracle_tri_index.argtypes = [i64, i64, i64]
            lib.xe_oracle_tri_index.restype = i64
            lib.xe_oracle_n_baselines.argtypes = [i64]
            lib.xe_oracle_n_baselines.restype = i64
            lib.xe_oracle_correlate.argtypes = [p, i64, i64, i64, p]
            lib.xe_oracle_correlate.restype = ctypes.c_int
            lib.xe_oracle_pairs.argtypes = [p, i64, i64, i64, p, p, p, p]
            lib.xe_oracle_pairs.restype = ctypes.c_int
            lib.xe_oracle_cmac.argtypes = [i64, i64, i64]
            lib.xe_oracle_cmac.restype = ctypes.c_double
            lib.xe_oracle_threads.restype = ctypes.c_int
            lib.xe_oracle_set_threads.argtypes = [ctypes.c_int]
            lib.xe_oracle_set_threads.restype = ctypes.c_int
            lib.xe_oracle_correlate_masked.argtypes = [p, p, i64, i64, i64, ctypes.c_int, p]
            lib.xe_oracle_correlate_masked.restype = ctypes.c_int
            lib.xe_oracle_flag_counts.argtypes = [p, i64, i64, i64, p]
            lib.xe_oracle_flag_counts.restype = ctypes.c_int
            lib.xe_oracle_beamform.argtypes = [p, p, i64, i64, i64, i64, p]
            lib.xe_oracle_beamform.restype = ctypes.c_int
            lib.xe_oracle_corner_turn.argtypes = [p, i64, i64, i64, i64, p]
            lib.xe_oracle_corner_turn.restype = ctypes.c_int
            lib.xe_oracle_presum.argtypes = [p, i64, i64, i64, p]
            lib.xe_oracle_presum.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def decode(packed: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Packed bytes -> (re, im) int64 arrays of the same shape."""
    b = np.ascontiguousarray(packed, dtype=np.uint8)
    re = np.empty(b.shape, np.int64)
    im = np.empty(b.shape, np.int64)
    _load().xe_oracle_decode(_ptr(b), b.size, _ptr(re), _ptr(im))
    return re, im


def tri_index(N: int, i: int, j: int) -> int:
    return int(_load().xe_oracle_tri_index(N, i, j))


def n_baselines(N: int) -> int:
    return int(_load().xe_oracle_n_baselines(N))


def cmac(N: int, T: int, C: int = 1) -> float:
    """Complex MACs of one correlation, C * T * N(N+1)/2 (section 2.2, eta / delta-nu)."""
    return float(_load().xe_oracle_cmac(N, T, C))


def threads() -> int:
    return int(_load().xe_oracle_threads())


def set_threads(n: int) -> int:
    """Threads of the OpenMP loops (timing harnesses only); returns the count in force."""
    return int(_load().xe_oracle_set_threads(int(n)))


def _check_in(packed: np.ndarray, N: int, T: int, C: int) -> np.ndarray:
    b = np.ascontiguousarray(packed, dtype=np.uint8).reshape(-1)
    if b.size != C * T * N:
        raise ValueError(f"packed has {b.size} bytes, expected C*T*N = {C * T * N}")
    return b


def correlate64(packed: np.ndarray, N: int, T: int, C: int = 1) -> np.ndarray:
    """Plain C triple loop.  Returns int64 [C, N(N+1)/2, 2]."""
    b = _check_in(packed, N, T, C)
    out = np.empty((C, n_baselines(N), 2), np.int64)
    rc = _load().xe_oracle_correlate(_ptr(b), N, T, C, _ptr(out))
    if rc != 0:
        raise ValueError("xe_oracle_correlate rejected its arguments")
    return out


def to_int32(v64: np.ndarray) -> np.ndarray:
    """int64 visibilities -> int32, refusing values that do not fit (overflow reading)."""
    if v64.size and (v64.max() > np.iinfo(np.int32).max or v64.min() < np.iinfo(np.int32).min):
        raise OverflowError("visibility does not fit int32")
    return v64.astype(np.int32)


def correlate(packed: np.ndarray, N: int, T: int, C: int = 1) -> np.ndarray:
    """Plain C triple loop, int32 result [C, N(N+1)/2, 2]."""
    return to_int32(correlate64(packed, N, T, C))


def pairs(packed: np.ndarray, N: int, T: int, C: int, c, i, j) -> np.ndarray:
    """Selected baselines (c[k], i[k], j[k]) one by one; int64 [n, 2]."""
    b = _check_in(packed, N, T, C)
    c = np.ascontiguousarray(c, np.int64)
    i = np.ascontiguousarray(i, np.int64)
    j = np.ascontiguousarray(j, np.int64)
    if not (c.shape == i.shape == j.shape) or (c.size and c.max() >= C):
        raise ValueError("bad pair arrays")
    out = np.empty((c.size, 2), np.int64)
    rc = _load().xe_oracle_pairs(_ptr(b), N, T, c.size, _ptr(c), _ptr(i), _ptr(j), _ptr(out))
    if rc != 0:
        raise ValueError("xe_oracle_pairs rejected a pair")
    return out


def voltages(packed_chan: np.ndarray, N: int, T: int) -> np.ndarray:
    """One channel's packed [T][N] bytes -> complex128 X with X[i, t] = x_i(t)."""
    re, im = decode(np.asarray(packed_chan, np.uint8).reshape(T, N))
    return (re + 1j * im).T.astype(np.complex128)


def correlate_dense(packed: np.ndarray, N: int, T: int, C: int = 1,
                    t_chunk: int = 4096) -> np.ndarray:
    """V = X X^H with a complex128 library matmul; int32 [C, N(N+1)/2, 2].

    The time sum is taken in chunks of ``t_chunk`` samples (the sum over t is an exact
    integer sum, so splitting it changes nothing).  Exact while 2*64*T < 2**53.
    """
    b = _check_in(packed, N, T, C).reshape(C, T, N)
    iu = np.triu_indices(N)               # row-major (i, j >= i): the packed order
    out = np.empty((C, n_baselines(N), 2), np.int64)
    for c in range(C):
        V = np.zeros((N, N), np.complex128)
        for t0 in range(0, T, t_chunk):
            X = voltages(b[c, t0:t0 + t_chunk], N, min(t_chunk, T - t0))
            V += X @ X.conj().T
        tri = V[iu]
        out[c, :, 0] = np.rint(tri.real).astype(np.int64)
        out[c, :, 1] = np.rint(tri.imag).astype(np.int64)
    return to_int32(out)


def unpack_triangle(vis: np.ndarray, N: int) -> np.ndarray:
    """Packed [N(N+1)/2, 2] -> full Hermitian complex matrix (test helper)."""
    iu = np.triu_indices(N)
    V = np.zeros((N, N), np.complex128)
    V[iu] = vis[:, 0] + 1j * vis[:, 1]
    V[(iu[1], iu[0])] = vis[:, 0] - 1j * vis[:, 1]
    return V


def correlate_masked(packed: np.ndarray, flags, N: int, T: int, C: int = 1,
                     encoding: int = 0) -> np.ndarray:
    """Flag-masked correlation (plain C loop).  flags: uint8 [C][T][ceil(N/8)] validity
    bits (bit n%8 of byte n/8, 1 = valid) or None; encoding 0 = two's complement nibbles,
    1 = offset binary.  Returns int32 [C, N(N+1)/2, 2]."""
    b = _check_in(packed, N, T, C)
    f = None
    if flags is not None:
        f = np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
        if f.size != C * T * ((N + 7) // 8):
            raise ValueError("flags must hold C*T*ceil(N/8) bytes")
    out = np.empty((C, n_baselines(N), 2), np.int64)
    rc = _load().xe_oracle_correlate_masked(_ptr(b), None if f is None else _ptr(f), N, T, C,
                                            encoding, _ptr(out))
    if rc != 0:
        raise ValueError("xe_oracle_correlate_masked rejected its arguments")
    return to_int32(out)


def flag_counts(flags, N: int, T: int, C: int = 1) -> np.ndarray:
    """Valid-sample count of every baseline, n_ij = sum_t f_i(t) f_j(t); int64 [C, B]."""
    f = np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
    if f.size != C * T * ((N + 7) // 8):
        raise ValueError("flags must hold C*T*ceil(N/8) bytes")
    out = np.empty((C, n_baselines(N)), np.int64)
    rc = _load().xe_oracle_flag_counts(_ptr(f), N, T, C, _ptr(out))
    if rc != 0:
        raise ValueError("xe_oracle_flag_counts rejected its arguments")
    return out


def valid_bits(flags, N: int, T: int, C: int = 1) -> np.ndarray:
    """Validity bits uint8 [C][T][ceil(N/8)] -> bool [C, T, N] (bit n%8 of byte n/8)."""
    f = np.ascontiguousarray(flags, dtype=np.uint8).reshape(C, T, (N + 7) // 8)
    return np.unpackbits(f, axis=2, bitorder="little")[:, :, :N].astype(bool)


def correlate_masked_dense(packed: np.ndarray, flags, N: int, T: int, C: int = 1,
                           encoding: int = 0, t_chunk: int = 4096) -> np.ndarray:
    """The masked definition as a matrix product: with f in {0, 1},
    f_i f_j x_i conj(x_j) = (f_i x_i) conj(f_j x_j), so V = Y Y^H with Y = F * X
    (complex128 library matmul; exact for the same reason as correlate_dense).
    Offset-binary samples (encoding 1) decode as nibble - 8.  int32 [C, B, 2]."""
    b = _check_in(packed, N, T, C).reshape(C, T, N)
    valid = None if flags is None else valid_bits(flags, N, T, C)
    iu = np.triu_indices(N)
    out = np.empty((C, n_baselines(N), 2), np.int64)
    for c in range(C):
        V = np.zeros((N, N), np.complex128)
        for t0 in range(0, T, t_chunk):
            blk = b[c, t0:t0 + t_chunk]
            if encoding == 1:
                re = (blk >> 4).astype(np.int64) - 8
                im = (blk & 0xF).astype(np.int64) - 8
            else:
                re, im = decode(blk)
            Y = (re + 1j * im).astype(np.complex128)
            if valid is not None:
                Y = Y * valid[c, t0:t0 + t_chunk]
            Y = Y.T
            V += Y @ Y.conj().T
        tri = V[iu]
        out[c, :, 0] = np.rint(tri.real).astype(np.int64)
        out[c, :, 1] = np.rint(tri.imag).astype(np.int64)
    return to_int32(out)


def flag_counts_dense(flags, N: int, T: int, C: int = 1, t_chunk: int = 8192) -> np.ndarray:
    """Valid-sample counts as the matrix product F^T F of the 0/1 validity matrix (float64
    library matmul; exact, every partial sum is an integer <= T < 2**53).  int64 [C, B]."""
    valid = valid_bits(flags, N, T, C)
    iu = np.triu_indices(N)
    out = np.empty((C, n_baselines(N)), np.int64)
    for c in range(C):
        M = np.zeros((N, N), np.float64)
        for t0 in range(0, T, t_chunk):
            F = valid[c, t0:t0 + t_chunk].astype(np.float64)
            M += F.T @ F
        out[c] = np.rint(M[iu]).astype(np.int64)
    return out


def _check_w(w, N: int, B: int) -> np.ndarray:
    a = np.ascontiguousarray(w, dtype=np.int8)
    if a.size != B * N * 2:
        raise ValueError(f"weights must hold B*N*2 = {B * N * 2} int8 values")
    return a.reshape(B, N, 2)


def beamform(packed: np.ndarray, w, N: int, T: int, C: int = 1, B: int = 1) -> np.ndarray:
    """Plain C loop: y_b(t) = sum_i w_{b,i} x_i(t).  w: int8 [B][N][2]; int64 [C, T, B, 2]."""
    b = _check_in(packed, N, T, C)
    wa = _check_w(w, N, B)
    out = np.empty((C, T, B, 2), np.int64)
    rc = _load().xe_oracle_beamform(_ptr(b), _ptr(wa), N, T, C, B, _ptr(out))
    if rc != 0:
        raise ValueError("xe_oracle_beamform rejected its arguments")
    return out


def beamform_dense(packed: np.ndarray, w, N: int, T: int, C: int = 1, B: int = 1,
                   t_chunk: int = 8192) -> np.ndarray:
    """The beams as a matrix product Y = X W^T (complex128 library matmul, exact: every
    partial sum is an integer of magnitude below 2 * 8 * 128 * N < 2**53).
    int64 [C, T, B, 2]."""
    b = _check_in(packed, N, T, C).reshape(C, T, N)
    wa = _check_w(w, N, B).astype(np.int64)
    W = (wa[..., 0] + 1j * wa[..., 1]).astype(np.complex128)          # [B, N]
    out = np.empty((C, T, B, 2), np.int64)
    for c in range(C):
        for t0 in range(0, T, t_chunk):
            re, im = decode(b[c, t0:t0 + t_chunk])
            Y = (re + 1j * im).astype(np.complex128) @ W.T                # [t, B]
            out[c, t0:t0 + t_chunk, :, 0] = np.rint(Y.real).astype(np.int64)
            out[c, t0:t0 + t_chunk, :, 1] = np.rint(Y.imag).astype(np.int64)
    return out


def beam_cmac(N: int, T: int, C: int = 1, B: int = 1) -> float:
    """Complex multiply-accumulates of the beams: C * T * B * N."""
    return float(C) * T * B * N


def corner_turn(bundles: np.ndarray, n_cyl: int, n_freq: int, n_in: int, T: int) -> np.ndarray:
    """uint8 bundles [n_cyl][T][n_freq][n_in] -> frames uint8 [n_freq][T][n_cyl * n_in]."""
    b = np.ascontiguousarray(bundles, dtype=np.uint8).reshape(-1)
    if b.size != n_cyl * T * n_freq * n_in:
        raise ValueError("bundles must hold n_cyl * T * n_freq * n_in bytes")
    out = np.empty((n_freq, T, n_cyl * n_in), np.uint8)
    rc = _load().xe_oracle_corner_turn(_ptr(b), n_cyl, n_freq, n_in, T, _ptr(out))
    if rc != 0:
        raise ValueError("xe_oracle_corner_turn rejected its arguments")
    return out


def presum(frames: np.ndarray, N: int, T: int, C: int = 1) -> np.ndarray:
    """Per-input time sums of re and im: int64 [C, N, 2]."""
    b = _check_in(frames, N, T, C)
    out = np.empty((C, N, 2), np.int64)
    rc = _load().xe_oracle_presum(_ptr(b), N, T, C, _ptr(out))
    if rc != 0:
        raise ValueError("xe_oracle_presum rejected its arguments")
    return out
