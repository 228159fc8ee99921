"""Real-time serving loop over the streaming server (xe_stream_*).

Frames of `frame_T` samples per channel arrive at the instrument's sample rate (CHIME:
390625 samples/s per channel, Denman et al. 2020, section 2.3 and Table tab:node-stats),
for `n_chan` channels at once.  A producer paces the pushes in real time; a consumer thread
polls completed integrations and records the frame-to-visibility latency (time from the
arrival of an integration's last frame to its visibilities being in host memory).  The
correlation itself runs in the CUDA library; this module only paces and measures.
"""
from __future__ import annotations

import gc
import threading
import time

from . import xe

CHIME_RATE = 390625.0
# Lower edges (ms) of the frame-to-visibility latency histogram's buckets; the last is open.
LATENCY_EDGES_MS = (0, 10, 20, 40, 80, 160, 320, 640)


def latency_histogram(lat_ns) -> list[int]:
    """Counts of latencies (ns) per bucket [LATENCY_EDGES_MS[k], LATENCY_EDGES_MS[k + 1]) ms,
    the last bucket open-ended."""
    edges = list(LATENCY_EDGES_MS) + [None]
    return [sum(1 for v in lat_ns if v / 1e6 >= lo and (hi is None or v / 1e6 < hi))
            for lo, hi in zip(edges[:-1], edges[1:])]


def per_channel_bytes(N: int, frame_T: int, ring_frames: int) -> int:
    """Device bytes one channel slot holds: accumulators + frame ring + staging share (up to
    min(4, ring_frames) frames of a channel are correlated as one job)."""
    n_pad = (N + 255) // 256 * 256
    merge = min(4, ring_frames)
    return (2 * N * (N + 1) * 4 + ring_frames * frame_T * N
            + merge * 2 * n_pad * ((frame_T + 63) // 64 * 64))


def run_realtime(n_chan: int, seconds: float, N: int = 2048, frame_T: int = 8192,
                 integ_T: int = 32768, rate: float = CHIME_RATE, device_source: bool = True,
                 ring_frames: int = 8, hbm_budget: int | None = None, n_distinct: int = 8,
                 seed: int = 20050948) -> dict:
    """Stream n_chan channels in real time for `seconds`; return throughput and latency.

    The producer and consumer are Python threads: the garbage collector is run first and kept
    off while they pace the frames (a collection pause in the producer would count as a late
    frame of the server's run)."""
    gc.collect()
    gc_was_enabled = gc.isenabled()
    gc.disable()
    try:
        return _run_realtime(n_chan, seconds, N, frame_T, integ_T, rate, device_source, ring_frames,
                             hbm_budget, n_distinct, seed)
    finally:
        if gc_was_enabled:
            gc.enable()


def _run_realtime(n_chan, seconds, N, frame_T, integ_T, rate, device_source, ring_frames, hbm_budget,
                  n_distinct, seed):
    import torch
    budget = hbm_budget if hbm_budget is not None else (n_chan + 1) * per_channel_bytes(N, frame_T, ring_frames)
    frame_period = frame_T / rate
    n_frames = max(integ_T // frame_T, int(round(seconds / frame_period)))
    n_frames = (n_frames + integ_T // frame_T - 1) // (integ_T // frame_T) * (integ_T // frame_T)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    # Distinct random frames (full-range packed bytes), reused cyclically across channels.
    frames = [torch.randint(0, 256, (frame_T, N), dtype=torch.uint8, device="cuda", generator=g)
              for _ in range(n_distinct)]
    if not device_source:
        frames = [f.cpu().pin_memory() for f in frames]
    lat_ns, results = [], [0, 0]
    stop = threading.Event()
    with xe.Stream(N, frame_T, integ_T, max_chan=n_chan, hbm_budget=budget,
                   ring_frames=ring_frames, sample_rate=rate, device_source=device_source) as st:
        admitted = 0
        for c in range(n_chan):
            if st.admit(c) != xe.XE_OK:
                break
            admitted += 1

        def consumer():
            while not stop.is_set() or results[0] < expected[0]:
                r = st.poll(timeout_ms=20, copy=False)
                if r is None:
                    if stop.is_set() and time.monotonic() > deadline[0]:
                        break
                    continue
                meta, _ = r
                results[0] += 1
                results[1] += 1 if meta["complete"] else 0
                lat_ns.append(meta["t_ready_ns"] - meta["t_last_arrival_ns"])

        expected = [admitted * (n_frames // (integ_T // frame_T))]
        deadline = [float("inf")]
        th = threading.Thread(target=consumer, daemon=True)
        th.start()
        overruns, late = 0, 0
        chans = list(range(admitted))
        t0 = time.monotonic() + 0.05
        for k in range(n_frames):
            target = t0 + k * frame_period
            now = time.monotonic()
            if target > now:
                time.sleep(target - now)
            elif now - target > frame_period:
                late += 1                      # the producer itself fell a frame behind
            t_arr = time.monotonic_ns()
            rc = st.push_frames(chans, [frames[(k + c) % n_distinct] for c in chans],
                                [k] * admitted, t_arr)
            overruns += int((rc != xe.XE_OK).sum())
        t_last_push = time.monotonic()
        st.flush()
        deadline[0] = time.monotonic() + 5.0
        stop.set()
        th.join(timeout=10.0)
        t_end = time.monotonic()
        stats = st.stats()
        counters = st.counters()
    lat = sorted(lat_ns)
    pct = (lambda q: lat[min(len(lat) - 1, int(q * len(lat)))] / 1e6) if lat else (lambda q: None)
    hist = latency_histogram(lat)
    cmac_frame = N * (N + 1) / 2 * frame_T
    span = t_last_push - t0 + frame_period
    realtime = span <= n_frames * frame_period * 1.02 + 0.01
    return {
        "channels": admitted, "frames_per_channel": n_frames, "seconds": span,
        "frames_processed": stats["frames"], "frames_dropped": stats["dropped"],
        "push_overruns": overruns, "integrations": results[0], "complete_integrations": results[1],
        "expected_integrations": expected[0],
        "sustained": bool(realtime and late == 0 and overruns == 0 and stats["dropped"] == 0
                          and results[0] == expected[0] and results[1] == expected[0]),
        "producer_late_frames": late, "realtime_pace": bool(realtime),
        "cmac_per_s": stats["frames"] * cmac_frame / span,
        "p50_latency_ms": pct(0.50), "p99_latency_ms": pct(0.99),
        "max_latency_ms": (lat[-1] / 1e6) if lat else None,
        "latency_hist_ms": {"edges": list(LATENCY_EDGES_MS), "counts": hist},
        "drain_s": t_end - t_last_push, "device_source": device_source, "counters": counters,
        "frame_T": frame_T, "integ_T": integ_T, "N": N, "rate": rate,
    }
