"""Planted mistakes: each mutant of the C oracle must fail one of the golden pins.

The mutants are built on the CPU from a text-substituted copy of oracle/xe_oracle.c in a
temporary directory; nothing here touches a GPU or the CUDA library.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "xe_oracle.c")
GOLDEN = os.path.join(ROOT, "tests", "golden")

MUTANTS = {
    "im_sign_flipped": ("acc_im += b * p - a * q;", "acc_im += a * q - b * p;"),
    "dropped_imag_product": ("acc_re += a * p + b * q;", "acc_re += a * p;"),
    "re_product_sign": ("acc_re += a * p + b * q;", "acc_re += a * p - b * q;"),
    "nibbles_swapped": ("int64_t hi = (byte >> 4) & 0xF;", "int64_t hi = byte & 0xF; byte >>= 4;"),
    "offset_binary": ("*re = (hi >= 8) ? hi - 16 : hi;", "*re = hi - 8;"),
    "transposed_operand": ("decode_sample(chan[t * N + j], &p, &q);",
                           "decode_sample(chan[j * T + t < N * T ? j * T + t : 0], &p, &q);"),
    "triangle_index_lower": ("return i * N - (i * (i - 1)) / 2 + (j - i);",
                             "return j * (j + 1) / 2 + i;"),
    "no_autocorrelation": ("return N * (N + 1) / 2;", "return N * (N - 1) / 2;"),
}


def _golden_cases():
    with open(os.path.join(GOLDEN, "hand_visibilities.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    for row in rows:
        bar = [k for k, tok in enumerate(row) if tok == "|"]
        N, T = int(row[1]), int(row[2])
        b = np.array([int(x, 16) for x in row[bar[0] + 1:bar[1]]], np.uint8)
        want = np.array([[int(v) for v in p.split(",")] for p in row[bar[1] + 1:]], np.int64)
        yield N, T, b, want


def _passes_pins(lib) -> bool:
    i64, p = ctypes.c_int64, ctypes.c_void_p
    lib.xe_oracle_correlate.argtypes = [p, i64, i64, i64, p]
    lib.xe_oracle_n_baselines.argtypes = [i64]
    lib.xe_oracle_n_baselines.restype = i64
    for N, T, b, want in _golden_cases():
        if lib.xe_oracle_n_baselines(N) != N * (N + 1) // 2:
            return False
        out = np.full((want.shape[0] + 8, 2), -12345, np.int64)   # room for bad indexing
        lib.xe_oracle_correlate(b.ctypes.data, N, T, 1, out.ctypes.data)
        if not np.array_equal(out[:want.shape[0]], want):
            return False
    return True


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, f"mutation anchor for {name} not found"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(path)])
    return ctypes.CDLL(str(so))


def test_unmutated_passes(tmp_path):
    assert _passes_pins(_build(tmp_path, "clean", "int64_t", "int64_t"))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    assert not _passes_pins(_build(tmp_path, name, old, new))
