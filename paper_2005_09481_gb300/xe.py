"""Thin ctypes binding of libxe (include/xe.h).  Argument marshalling only: every step of
the correlation runs in the CUDA library.  There is no CPU fallback: if the library cannot
be built or loaded, every call raises.

Tensors: inputs are uint8 ``[C, T, N]`` (or ``[T, N]``) CUDA tensors of packed 4+4-bit
samples; outputs are int32 ``[C, N(N+1)/2, 2]`` CUDA tensors (row-major upper triangle,
{Re, Im}).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

XE_OK, XE_EINVAL, XE_EOVERFLOW, XE_ENOMEM, XE_EBUDGET = 0, -1, -2, -3, -4
XE_EAGAIN, XE_ETIMEOUT, XE_ECUDA, XE_ENODEV, XE_ECLOSED = -5, -6, -7, -8, -9
XE_ECHECK = -10
XE_MAX_T, XE_MAX_N = 16777215, 65536          # samples per integration (128 T < 2^31), inputs
ALGOS = {"auto": 0, "tc": 1, "imma": 2}

_lock = threading.Lock()
_lib = None


class XeError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {detail} (code {code})")
        self.code = code


class Job(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("vis", ctypes.c_void_p), ("N", ctypes.c_int),
                ("n_chan", ctypes.c_int), ("T", ctypes.c_int64)]


class MaskedJob(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("flags", ctypes.c_void_p), ("vis", ctypes.c_void_p),
                ("counts", ctypes.c_void_p), ("N", ctypes.c_int), ("n_chan", ctypes.c_int),
                ("T", ctypes.c_int64), ("encoding", ctypes.c_int), ("accumulate", ctypes.c_int)]


ENCODINGS = {"twos": 0, "offset": 1}


def lib_path() -> str:
    return _build.LIB


def load():
    """Build (if stale) and load libxe.so.  Raises if nvcc or the library is unavailable."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        L = ctypes.CDLL(path)
        i64, i32, p, d = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_double
        sigs = {
            "xe_strerror": ([i32], ctypes.c_char_p),
            "xe_last_error": ([], ctypes.c_char_p),
            "xe_version": ([], i32),
            "xe_cmac": ([i64, i64, i64], d),
            "xe_correlate": ([p, i32, i64, i32, p], i32),
            "xe_correlate_async": ([p, i32, i64, i32, p, i32, p], i32),
            "xe_correlate_host": ([p, i32, i64, i32, p, i32], i32),
            "xe_correlate_host_async": ([p, i32, i64, i32, p, i32], i32),
            "xe_host_wait": ([i32], i32),
            "xe_correlate_batch": ([p, i32, i32, p], i32),
            "xe_correlate_noalloc": ([p, i32, i64, i32, p, p], i32),
            "xe_noalloc_status": ([p], i32),
            "xe_correlate_accumulate": ([p, i32, p], i32),
            "xe_plan_stats": ([p, p, p, i32, i32, p, p, p], i32),
            "xe_set_option": ([ctypes.c_char_p, i64], i32),
            "xe_set_timing": ([i32], i32),
            "xe_last_timing": ([p, p], i32),
            "xe_last_timing_counts": ([p, p, p], i32),
            "xe_correlate_masked": ([p, p, i32, i64, i32, i32, p, p, i32, p], i32),
            "xe_correlate_masked_batch": ([p, i32, p], i32),
            "xe_beamform": ([p, i32, i64, i32, p, i32, p, p], i32),
            "xe_bundle_view": ([i32, i32, i32, i64, p], i32),
            "xe_correlate_view": ([p, p, i32, i64, i32, p, p], i32),
            "xe_corner_turn": ([p, i32, i32, i32, i64, p, p, p], i32),
            "xe_device_status": ([p], i32),
            "xe_release_stream": ([p], i32),
            "xe_debug_operand_code": ([i32, i32], ctypes.c_uint32),
            "xe_plan_dump": ([p, p, p, i32, i32, i32, i32, p, i64], i64),
            "xe_last_config": ([p, p, p], i32),
            "xe_peak_probe": ([i32, p, p], i32),
            "xe_device_info": ([p], i32),
            "xe_tune_cache": ([ctypes.c_char_p], i32),
            "xe_tune_store": ([ctypes.c_char_p, i32, p, p, p, i32, i32, i32, i32, i32], i32),
            "xe_tune_lookup": ([ctypes.c_char_p, i32, p, p, p, i32, i32, p, p, p], i32),
            "xe_tune_stats": ([p, p], i32),
            "xe_runtime_counters": ([p, i32], i32),
            "xe_stream_open": ([p, p], i32),
            "xe_stream_admit": ([p, i32], i32),
            "xe_stream_evict": ([p, i32], i32),
            "xe_stream_push": ([p, i32, p, i64, i64], i32),
            "xe_stream_push_frames": ([p, i32, p, p, p, i64, p], i32),
            "xe_stream_flush": ([p], i32),
            "xe_stream_poll": ([p, p, i32], i32),
            "xe_stream_release": ([p, i64], i32),
            "xe_stream_stats": ([p, p, p, p, p], i32),
            "xe_stream_close": ([p], None),
            "xe_stream_counters": ([p, p, i32], i32),
            "xe_stream_snapshot": ([p, i32, p, p, i32], i32),
            "xe_stream_restore": ([p, i32, p, p], i32),
        }
        for name, (args, res) in sigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


def _check(rc: int, where: str):
    if rc != XE_OK:
        L = load()
        raise XeError(rc, where, L.xe_last_error().decode(errors="replace"))


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def n_baselines(N: int) -> int:
    return N * (N + 1) // 2


def cmac(N: int, T: int, C: int = 1) -> float:
    return float(load().xe_cmac(N, T, C))


def set_option(key: str, value: int):
    _check(load().xe_set_option(key.encode(), int(value)), f"xe_set_option({key})")


def set_timing(enable: bool):
    _check(load().xe_set_timing(1 if enable else 0), "xe_set_timing")


def last_timing() -> tuple[float, float]:
    a, b = ctypes.c_float(), ctypes.c_float()
    _check(load().xe_last_timing(ctypes.byref(a), ctypes.byref(b)), "xe_last_timing")
    return a.value, b.value


def last_timing_counts() -> tuple[float, float, float]:
    """(stage, correlate, counts) device milliseconds of the last call on this thread."""
    a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
    _check(load().xe_last_timing_counts(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "xe_last_timing_counts")
    return a.value, b.value, c.value


def device_status(stream=None):
    _check(load().xe_device_status(_stream_handle(stream)), "xe_device_status")


def release_stream(stream=None):
    """Free the library's scratch memory for `stream` (a torch.cuda.Stream, or None for the
    current stream); call before the stream is destroyed."""
    _check(load().xe_release_stream(_stream_handle(stream)), "xe_release_stream")


def peak_probe(kind: str, with_aux: bool = False):
    """Measured dense TFLOP/s of 'tc_fp8' (tcgen05 e4m3), 'imma_s8' (mma.sync int8) or
    'tc_fp8_fill' (tcgen05 e4m3 with concurrent shared-memory fills; aux = fill GB/s)."""
    out, aux = ctypes.c_double(), ctypes.c_double(0.0)
    _check(load().xe_peak_probe({"tc_fp8": 0, "imma_s8": 1, "tc_fp8_fill": 2, "tc_fp8_fill_l2": 3}[kind],
                                ctypes.byref(out),
                                ctypes.byref(aux)), "xe_peak_probe")
    return (out.value, aux.value) if with_aux else out.value


def device_info():
    """SM count of the current device."""
    a = ctypes.c_int()
    _check(load().xe_device_info(ctypes.byref(a)), "xe_device_info")
    return a.value


def operand_code(v: int, elem_bytes: int) -> int:
    return int(load().xe_debug_operand_code(v, elem_bytes))


def plan_stats(shapes, n_cta: int):
    """shapes: list of (N, T, C).  Returns (n_tiles, n_iters, n_split_tiles)."""
    n = len(shapes)
    Ns = (ctypes.c_int * n)(*[s[0] for s in shapes])
    Ts = (ctypes.c_int64 * n)(*[s[1] for s in shapes])
    Cs = (ctypes.c_int * n)(*[s[2] for s in shapes])
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().xe_plan_stats(Ns, Ts, Cs, n, n_cta, ctypes.byref(a), ctypes.byref(b),
                                ctypes.byref(c)), "xe_plan_stats")
    return a.value, b.value, c.value


SCHEDULES = {"stream_k": 0, "split": 1, "hybrid": 2, "lpt": 3, "weighted": 4}


def plan_dump(shapes, n_cta: int, sched: int = -1, tile_n: int = 0):
    """Host-side plan for shapes [(N, T, C), ...]: dict with 'tiles' (job, chan, i0, j0, nj,
    kblocks) rows, 'segs' (cta, tile, k_lo, k_hi, slot) rows, 'n_cta', 'n_partial'."""
    import numpy as np
    n = len(shapes)
    Ns = (ctypes.c_int * n)(*[s[0] for s in shapes])
    Ts = (ctypes.c_int64 * n)(*[s[1] for s in shapes])
    Cs = (ctypes.c_int * n)(*[s[2] for s in shapes])
    L = load()
    need = L.xe_plan_dump(Ns, Ts, Cs, n, n_cta, sched, tile_n, None, 0)
    if need < 0:
        _check(int(need), "xe_plan_dump")
    buf = np.zeros(need, np.int32)
    got = L.xe_plan_dump(Ns, Ts, Cs, n, n_cta, sched, tile_n, buf.ctypes.data, need)
    _check(0 if got == need else int(got), "xe_plan_dump")
    nt, ns = int(buf[0]), int(buf[1])
    tiles = buf[4:4 + 6 * nt].reshape(nt, 6)
    segs = buf[4 + 6 * nt:4 + 6 * nt + 5 * ns].reshape(ns, 5)
    return {"tiles": tiles, "segs": segs, "n_cta": int(buf[2]), "n_partial": int(buf[3])}


def _shape_arrays(shapes):
    n = len(shapes)
    return ((ctypes.c_int * n)(*[s[0] for s in shapes]), (ctypes.c_int64 * n)(*[s[1] for s in shapes]),
            (ctypes.c_int * n)(*[s[2] for s in shapes]), n)


def tune_cache(path):
    """Use `path` as the tuning cache file (None: none)."""
    _check(load().xe_tune_cache(path.encode() if path else None), "xe_tune_cache")


def tune_store(gpu: str, n_sm: int, shapes, n_cta: int, tile_n: int, sched: int, operand_bytes: int = 1):
    """Record a plan configuration for shapes [(N, T, C), ...] on GPU `gpu` (no blanks)."""
    Ns, Ts, Cs, n = _shape_arrays(shapes)
    _check(load().xe_tune_store(gpu.encode(), n_sm, Ns, Ts, Cs, n, operand_bytes, n_cta, tile_n, sched),
           "xe_tune_store")


def tune_lookup(gpu: str, n_sm: int, shapes, operand_bytes: int = 1):
    """(n_cta, tile_n, sched) cached for shapes on GPU `gpu`, or None."""
    Ns, Ts, Cs, n = _shape_arrays(shapes)
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    L = load()
    rc = L.xe_tune_lookup(gpu.encode(), n_sm, Ns, Ts, Cs, n, operand_bytes, ctypes.byref(a), ctypes.byref(b),
                          ctypes.byref(c))
    if rc == XE_EAGAIN:
        return None
    _check(rc, "xe_tune_lookup")
    return a.value, b.value, c.value


def tune_stats():
    """(candidate plans timed by the autotuner in this process, shapes taken from the cache)."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().xe_tune_stats(ctypes.byref(a), ctypes.byref(b)), "xe_tune_stats")
    return a.value, b.value


def runtime_counters():
    """Host work that can stall a caller: batches built and their host ns, plans built for new
    shapes and their host ns, scratch regrowths and plan-cache trims (both synchronise)."""
    import numpy as np
    v = np.zeros(6, np.int64)
    n = load().xe_runtime_counters(v.ctypes.data, 6)
    if n < 0:
        _check(n, "xe_runtime_counters")
    return dict(zip(("batches", "build_ns", "plans_built", "plan_ns", "regrowths", "trims"), v.tolist()))


def last_config():
    """(n_cta, tile_n, schedule) of the last plan this thread launched."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    load().xe_last_config(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    return a.value, b.value, c.value


def _shape(inp, N, T, C):
    import torch
    if inp.dtype != torch.uint8:
        raise TypeError("input must be uint8 packed samples")
    if not inp.is_contiguous():
        raise ValueError("input must be contiguous")
    if inp.numel() != C * T * N:
        raise ValueError(f"input has {inp.numel()} bytes, expected C*T*N = {C * T * N}")


def _device_input(inp, what="input"):
    if not inp.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")


def _int32_out(out, n, on_device, what):
    """`out` must be a contiguous int32 tensor of n elements on the device (or on the host)."""
    import torch
    if out.dtype != torch.int32 or not out.is_contiguous() or bool(out.is_cuda) != on_device:
        raise ValueError(f"{what} must be a contiguous int32 {'CUDA' if on_device else 'host'} tensor")
    if out.numel() != n:
        raise ValueError(f"{what} has {out.numel()} elements, expected {n}")


def empty_vis(N: int, C: int = 1, device="cuda"):
    import torch
    return torch.empty((C, n_baselines(N), 2), dtype=torch.int32, device=device)


def correlate(inp, N: int, T: int, C: int = 1, out=None, algo: str = "auto", stream=None):
    """Visibilities of C channels: device input -> device int32 [C, B, 2] (async on stream)."""
    _shape(inp, N, T, C)
    if not inp.is_cuda:
        raise ValueError("input must be a CUDA tensor (use correlate_host for host buffers)")
    if out is None:
        out = empty_vis(N, C, inp.device)
    _int32_out(out, C * n_baselines(N) * 2, True, "out")
    rc = load().xe_correlate_async(ctypes.c_void_p(inp.data_ptr()), N, T, C,
                                   ctypes.c_void_p(out.data_ptr()), ALGOS[algo],
                                   _stream_handle(stream))
    _check(rc, "xe_correlate_async")
    return out


def correlate_host(inp, N: int, T: int, C: int = 1, out=None, algo: str = "auto"):
    """Host (CPU, ideally pinned) input -> host int32 [C, B, 2]; synchronous."""
    import torch
    _shape(inp, N, T, C)
    if inp.is_cuda:
        raise ValueError("correlate_host takes host tensors")
    if out is None:
        out = torch.empty((C, n_baselines(N), 2), dtype=torch.int32,
                          pin_memory=inp.is_pinned())
    _int32_out(out, C * n_baselines(N) * 2, False, "out")
    rc = load().xe_correlate_host(ctypes.c_void_p(inp.data_ptr()), N, T, C,
                                  ctypes.c_void_p(out.data_ptr()), ALGOS[algo])
    _check(rc, "xe_correlate_host")
    return out


HOST_SLOTS = 4


def correlate_host_async(inp, N: int, T: int, C: int = 1, out=None, slot: int = 0):
    """Enqueue a host-buffer correlation into `slot` and return (out, slot) at once; `out`
    (pinned host int32 [C, B, 2]) is valid after host_wait(slot).  Keep `inp` and `out`
    alive and untouched until then."""
    import torch
    _shape(inp, N, T, C)
    if inp.is_cuda:
        raise ValueError("correlate_host_async takes host tensors")
    if out is None:
        out = torch.empty((C, n_baselines(N), 2), dtype=torch.int32, pin_memory=True)
    _int32_out(out, C * n_baselines(N) * 2, False, "out")
    rc = load().xe_correlate_host_async(ctypes.c_void_p(inp.data_ptr()), N, T, C,
                                        ctypes.c_void_p(out.data_ptr()), slot)
    _check(rc, "xe_correlate_host_async")
    return out, slot


def host_wait(slot: int):
    _check(load().xe_host_wait(slot), "xe_host_wait")


def correlate_batch(jobs, use_graph: bool = False, stream=None):
    """jobs: list of (input, out, N, T, C) with device tensors; one persistent launch."""
    arr = (Job * len(jobs))()
    for k, (inp, out, N, T, C) in enumerate(jobs):
        _shape(inp, N, T, C)
        _device_input(inp)
        _int32_out(out, C * n_baselines(N) * 2, True, "out")
        arr[k] = Job(inp.data_ptr(), out.data_ptr(), N, C, T)
    rc = load().xe_correlate_batch(arr, len(jobs), 1 if use_graph else 0, _stream_handle(stream))
    _check(rc, "xe_correlate_batch")
    return [j[1] for j in jobs]


def correlate_accumulate(jobs, stream=None):
    """jobs: list of (input, out, N, T, C); adds each job's visibilities into its out."""
    arr = (Job * len(jobs))()
    for k, (inp, out, N, T, C) in enumerate(jobs):
        _shape(inp, N, T, C)
        _device_input(inp)
        _int32_out(out, C * n_baselines(N) * 2, True, "out")
        arr[k] = Job(inp.data_ptr(), out.data_ptr(), N, C, T)
    _check(load().xe_correlate_accumulate(arr, len(jobs), _stream_handle(stream)),
           "xe_correlate_accumulate")
    return [j[1] for j in jobs]


def correlate_noalloc(inp, N: int, T: int, C: int = 1, out=None, stream=None):
    """As correlate(algo="tc"), through the entry point that allocates nothing (its scratch
    is a fixed array inside the library; see include/xe.h for the limits)."""
    _shape(inp, N, T, C)
    _device_input(inp)
    if out is None:
        out = empty_vis(N, C, inp.device)
    _int32_out(out, C * n_baselines(N) * 2, True, "out")
    rc = load().xe_correlate_noalloc(ctypes.c_void_p(inp.data_ptr()), N, T, C,
                                     ctypes.c_void_p(out.data_ptr()), _stream_handle(stream))
    _check(rc, "xe_correlate_noalloc")
    return out


def noalloc_status(stream=None):
    """Raise XeError(XE_ETIMEOUT) if an allocation-free call since the last query timed out."""
    _check(load().xe_noalloc_status(_stream_handle(stream)), "xe_noalloc_status")


def flag_bytes(N: int) -> int:
    """Bytes of one sample row of validity bits (one bit per input)."""
    return (N + 7) // 8


def empty_counts(N: int, C: int = 1, device="cuda"):
    import torch
    return torch.empty((C, n_baselines(N)), dtype=torch.int32, device=device)


def _flags_shape(flags, N, T, C):
    import torch
    if flags is None:
        return
    if flags.dtype != torch.uint8 or not flags.is_contiguous() or not flags.is_cuda:
        raise ValueError("flags must be a contiguous uint8 CUDA tensor")
    if flags.numel() != C * T * flag_bytes(N):
        raise ValueError(f"flags has {flags.numel()} bytes, expected C*T*ceil(N/8) = "
                         f"{C * T * flag_bytes(N)}")


def correlate_masked(inp, flags, N: int, T: int, C: int = 1, encoding: str = "twos",
                     out=None, counts=None, with_counts: bool = True, accumulate: bool = False,
                     stream=None):
    """Flag-masked correlation: V_ij = sum_t f_i(t) f_j(t) x_i(t) conj(x_j(t)) and the
    valid-sample counts n_ij.  flags: uint8 [C, T, ceil(N/8)] validity bits or None (all
    valid); encoding 'twos' or 'offset'.  Returns (vis, counts or None)."""
    _shape(inp, N, T, C)
    _device_input(inp)
    _flags_shape(flags, N, T, C)
    if out is None:
        out = empty_vis(N, C, inp.device)
    if with_counts and counts is None:
        counts = empty_counts(N, C, inp.device)
    if not with_counts:
        counts = None
    _int32_out(out, C * n_baselines(N) * 2, True, "out")
    if counts is not None:
        _int32_out(counts, C * n_baselines(N), True, "counts")
    rc = load().xe_correlate_masked(
        ctypes.c_void_p(inp.data_ptr()), ctypes.c_void_p(flags.data_ptr() if flags is not None else 0),
        N, T, C, ENCODINGS[encoding], ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(counts.data_ptr() if counts is not None else 0), 1 if accumulate else 0,
        _stream_handle(stream))
    _check(rc, "xe_correlate_masked")
    return out, counts


def correlate_masked_batch(jobs, stream=None):
    """jobs: list of dicts with keys in, flags (or None), vis, counts (or None), N, T, C,
    encoding ('twos'/'offset'), accumulate (bool).  One staging + one correlation launch."""
    arr = (MaskedJob * len(jobs))()
    for k, j in enumerate(jobs):
        _shape(j["in"], j["N"], j["T"], j["C"])
        _device_input(j["in"])
        _flags_shape(j.get("flags"), j["N"], j["T"], j["C"])
        f, c = j.get("flags"), j.get("counts")
        _int32_out(j["vis"], j["C"] * n_baselines(j["N"]) * 2, True, "vis")
        if c is not None:
            _int32_out(c, j["C"] * n_baselines(j["N"]), True, "counts")
        arr[k] = MaskedJob(j["in"].data_ptr(), f.data_ptr() if f is not None else None,
                           j["vis"].data_ptr(), c.data_ptr() if c is not None else None,
                           j["N"], j["C"], j["T"], ENCODINGS[j.get("encoding", "twos")],
                           1 if j.get("accumulate") else 0)
    _check(load().xe_correlate_masked_batch(arr, len(jobs), _stream_handle(stream)),
           "xe_correlate_masked_batch")
    return [(j["vis"], j.get("counts")) for j in jobs]


class View(ctypes.Structure):
    _fields_ = [("chan_stride", ctypes.c_int64), ("time_stride", ctypes.c_int64),
                ("seg_inputs", ctypes.c_int64), ("seg_stride", ctypes.c_int64)]


def bundle_view(n_cyl: int, n_freq: int, n_in: int, T: int) -> View:
    """The input view of n_freq channels held as cylinder bundles [n_cyl][T][n_freq][n_in]."""
    v = View()
    _check(load().xe_bundle_view(n_cyl, n_freq, n_in, T, ctypes.byref(v)), "xe_bundle_view")
    return v


def correlate_view(inp, view: View, N: int, T: int, C: int = 1, out=None, stream=None):
    """Correlation of C channels whose samples are addressed through `view` (device uint8
    tensor `inp` holding them) -> int32 [C, B, 2]."""
    import torch
    if inp.dtype != torch.uint8 or not inp.is_cuda:
        raise ValueError("input must be a uint8 CUDA tensor")
    if out is None:
        out = empty_vis(N, C, inp.device)
    _int32_out(out, C * n_baselines(N) * 2, True, "out")
    rc = load().xe_correlate_view(ctypes.c_void_p(inp.data_ptr()), ctypes.byref(view), N, T, C,
                                  ctypes.c_void_p(out.data_ptr()), _stream_handle(stream))
    _check(rc, "xe_correlate_view")
    return out


def correlate_bundles(bundles, n_cyl: int, n_freq: int, n_in: int, T: int, out=None, stream=None):
    """Full-array correlation of n_freq channels straight from cylinder bundles
    uint8 [n_cyl, T, n_freq, n_in] (corner turn fused into the staging loads)."""
    if bundles.numel() != n_cyl * T * n_freq * n_in:
        raise ValueError("bundles must hold n_cyl * T * n_freq * n_in bytes")
    return correlate_view(bundles, bundle_view(n_cyl, n_freq, n_in, T), n_cyl * n_in, T, n_freq,
                          out=out, stream=stream)


def corner_turn(bundles, n_cyl: int, n_freq: int, n_in: int, T: int, frames=None, presums: bool = True,
                stream=None):
    """Bundles uint8 [n_cyl, T, n_freq, n_in] -> (frames uint8 [n_freq, T, n_cyl * n_in],
    pre-sums int32 [n_freq, N, 2] or None)."""
    import torch
    if bundles.dtype != torch.uint8 or not bundles.is_cuda or not bundles.is_contiguous():
        raise ValueError("bundles must be a contiguous uint8 CUDA tensor")
    if bundles.numel() != n_cyl * T * n_freq * n_in:
        raise ValueError("bundles must hold n_cyl * T * n_freq * n_in bytes")
    N = n_cyl * n_in
    if frames is None:
        frames = torch.empty((n_freq, T, N), dtype=torch.uint8, device=bundles.device)
    if frames.dtype != torch.uint8 or not frames.is_cuda or not frames.is_contiguous() or \
            frames.numel() != bundles.numel():
        raise ValueError("frames must be a contiguous uint8 CUDA tensor of n_freq * T * N bytes")
    ps = torch.empty((n_freq, N, 2), dtype=torch.int32, device=bundles.device) if presums else None
    rc = load().xe_corner_turn(ctypes.c_void_p(bundles.data_ptr()), n_cyl, n_freq, n_in, T,
                               ctypes.c_void_p(frames.data_ptr()),
                               ctypes.c_void_p(ps.data_ptr() if ps is not None else 0), _stream_handle(stream))
    _check(rc, "xe_corner_turn")
    return frames, ps


def empty_beams(T: int, B: int, C: int = 1, device="cuda"):
    import torch
    return torch.empty((C, T, B, 2), dtype=torch.int32, device=device)


def beamform(inp, weights, N: int, T: int, C: int = 1, out=None, stream=None):
    """Phased-array beams y_b(t) = sum_i w_{b,i} x_i(t): device uint8 input [C, T, N], int8
    weights [B, N, 2] -> int32 [C, T, B, 2] (async on stream)."""
    import torch
    _shape(inp, N, T, C)
    _device_input(inp)
    if weights.dtype != torch.int8 or not weights.is_cuda or not weights.is_contiguous():
        raise ValueError("weights must be a contiguous int8 CUDA tensor [B, N, 2]")
    if weights.numel() % (2 * N) != 0:
        raise ValueError("weights must hold B * N * 2 values")
    B = weights.numel() // (2 * N)
    if out is None:
        out = empty_beams(T, B, C, inp.device)
    _int32_out(out, C * T * B * 2, True, "out")
    rc = load().xe_beamform(ctypes.c_void_p(inp.data_ptr()), N, T, C, ctypes.c_void_p(weights.data_ptr()),
                            B, ctypes.c_void_p(out.data_ptr()), _stream_handle(stream))
    _check(rc, "xe_beamform")
    return out


class StreamCfg(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("frame_T", ctypes.c_int64), ("integ_T", ctypes.c_int64),
                ("max_chan", ctypes.c_int), ("hbm_budget", ctypes.c_int64),
                ("ring_frames", ctypes.c_int), ("sample_rate", ctypes.c_double),
                ("device_source", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("chan", ctypes.c_int), ("integ_index", ctypes.c_int64),
                ("n_samples", ctypes.c_int64), ("complete", ctypes.c_int),
                ("vis", ctypes.c_void_p), ("t_first_arrival_ns", ctypes.c_int64),
                ("t_last_arrival_ns", ctypes.c_int64), ("t_ready_ns", ctypes.c_int64),
                ("handle", ctypes.c_int64)]


class Snapshot(ctypes.Structure):
    _fields_ = [("integ_index", ctypes.c_int64), ("next_seq", ctypes.c_int64),
                ("frames", ctypes.c_int64), ("n_samples", ctypes.c_int64), ("lost", ctypes.c_int),
                ("t_first_arrival_ns", ctypes.c_int64)]


class Stream:
    """Streaming server (xe_stream_*): admit channels, push frames, poll integrations."""

    def __init__(self, N: int, frame_T: int, integ_T: int, max_chan: int, hbm_budget: int,
                 ring_frames: int = 3, sample_rate: float = 390625.0, device_source: bool = False):
        self.N, self.frame_T, self.integ_T = N, frame_T, integ_T
        self.B = n_baselines(N)
        self.device_source = device_source
        cfg = StreamCfg(N, frame_T, integ_T, max_chan, hbm_budget, ring_frames, sample_rate,
                        1 if device_source else 0)
        h = ctypes.c_void_p()
        _check(load().xe_stream_open(ctypes.byref(cfg), ctypes.byref(h)), "xe_stream_open")
        self.h = h

    def admit(self, chan: int) -> int:
        """XE_OK, or XE_EBUDGET when the HBM budget is full."""
        rc = load().xe_stream_admit(self.h, chan)
        if rc not in (XE_OK, XE_EBUDGET):
            _check(rc, "xe_stream_admit")
        return rc

    def evict(self, chan: int):
        _check(load().xe_stream_evict(self.h, chan), "xe_stream_evict")

    def push(self, chan: int, frame, seq: int, t_arrival_ns: int = 0) -> int:
        """frame: uint8 [frame_T, N] tensor (CUDA if device_source, else host).  Returns
        XE_OK or XE_EAGAIN (ring full)."""
        if frame.numel() != self.frame_T * self.N or not frame.is_contiguous():
            raise ValueError("frame must be a contiguous [frame_T, N] uint8 tensor")
        if bool(frame.is_cuda) != self.device_source:
            raise ValueError("frame memory does not match the stream's source kind")
        rc = load().xe_stream_push(self.h, chan, ctypes.c_void_p(frame.data_ptr()), seq,
                                   t_arrival_ns)
        if rc not in (XE_OK, XE_EAGAIN):
            _check(rc, "xe_stream_push")
        return rc

    def push_frames(self, chans, frames, seqs, t_arrival_ns: int = 0):
        """Push several frames in one call; returns the per-frame codes (numpy int32)."""
        import numpy as np
        n = len(chans)
        for f in frames:
            if f.numel() != self.frame_T * self.N or bool(f.is_cuda) != self.device_source:
                raise ValueError("bad frame")
        c = np.ascontiguousarray(chans, np.int32)
        q = np.ascontiguousarray(seqs, np.int64)
        ptrs = (ctypes.c_void_p * n)(*[f.data_ptr() for f in frames])
        rc = np.zeros(n, np.int32)
        got = load().xe_stream_push_frames(self.h, n, c.ctypes.data, ptrs, q.ctypes.data,
                                           t_arrival_ns, rc.ctypes.data)
        if got < 0:
            _check(got, "xe_stream_push_frames")
        return rc

    def flush(self):
        _check(load().xe_stream_flush(self.h), "xe_stream_flush")

    def poll(self, timeout_ms: int = 0, copy: bool = True):
        """Next completed integration as (meta dict, int32 numpy [B, 2] copy or None), or
        None if nothing is ready.  The result buffer is handed back to the stream."""
        import numpy as np
        r = Result()
        rc = load().xe_stream_poll(self.h, ctypes.byref(r), timeout_ms)
        if rc == XE_EAGAIN:
            return None
        _check(rc, "xe_stream_poll")
        vis = None
        if copy:
            buf = (ctypes.c_int32 * (2 * self.B)).from_address(r.vis)
            vis = np.frombuffer(buf, dtype=np.int32).reshape(self.B, 2).copy()
        _check(load().xe_stream_release(self.h, r.handle), "xe_stream_release")
        meta = {k: getattr(r, k) for k, _ in Result._fields_ if k != "vis"}
        return meta, vis

    def stats(self):
        v = [ctypes.c_int64() for _ in range(4)]
        _check(load().xe_stream_stats(self.h, *[ctypes.byref(x) for x in v]), "xe_stream_stats")
        return dict(zip(("admitted", "frames", "integrations", "dropped"), [x.value for x in v]))

    def counters(self):
        import numpy as np
        v = np.zeros(9, np.int64)
        n = load().xe_stream_counters(self.h, v.ctypes.data, 9)
        if n < 0:
            _check(n, "xe_stream_counters")
        keys = ("admitted", "frames", "integrations", "dropped", "launch_passes",
                "launch_groups", "held_passes", "launch_host_ns", "rejected")
        return dict(zip(keys, v.tolist()))

    def snapshot(self, chan: int, timeout_ms: int = 2000):
        """Checkpoint of a channel's open integration: (info dict, int32 numpy [B, 2])."""
        import numpy as np
        vis = np.zeros((self.B, 2), np.int32)
        info = Snapshot()
        _check(load().xe_stream_snapshot(self.h, chan, ctypes.c_void_p(vis.ctypes.data),
                                         ctypes.byref(info), timeout_ms), "xe_stream_snapshot")
        return {k: getattr(info, k) for k, _ in Snapshot._fields_}, vis

    def restore(self, chan: int, info: dict, vis=None):
        """Continue a checkpointed integration on a newly admitted channel."""
        import numpy as np
        snap = Snapshot(*[int(info[k]) for k, _ in Snapshot._fields_])
        ptr = None
        if vis is not None:
            vis = np.ascontiguousarray(vis, np.int32)
            if vis.size != 2 * self.B:
                raise ValueError("vis must hold B x 2 int32 values")
            ptr = ctypes.c_void_p(vis.ctypes.data)
        _check(load().xe_stream_restore(self.h, chan, ptr, ctypes.byref(snap)), "xe_stream_restore")

    def close(self):
        if self.h:
            load().xe_stream_close(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
