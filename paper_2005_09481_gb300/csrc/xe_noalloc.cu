// xe_noalloc.cu -- an entry point of the tensor-core correlation that allocates nothing.
//
// Some callers cannot call cudaMalloc: a real-time pipeline that forbids allocation once
// it is running (an allocation can block on the driver and stall a frame deadline), a host
// application or plugin framework that owns all device memory through its own pool, or
// code that must not change the device's memory footprint after start-up.  For them,
// xe_correlate_noalloc runs the same staging and tcgen05 kernels as xe_correlate_async, but
// takes all of its scratch memory (staged operand planes, tile table, status words) from
// one fixed array compiled into this library, instead of allocating it.  Integrations
// longer than one window of staged planes run as several windows, each added into the
// visibilities (int32 sums of exact partial sums are exact).
//
// The array is a file-scope __device__ array of XE_NOALLOC_SCRATCH_BYTES (32 MiB): every
// GPU that loads the library holds it until the process exits.  Every call shares it, and
// it keeps the last call's contents; calls that overlap on the GPU (different streams, or
// different host threads without ordering) race on it and corrupt each other's results.
//
// A bounded wait that gives up sets the live status word; the next call moves a set live
// word into a latched word before it clears the live one, so a timeout stays visible until
// xe_noalloc_status reads (and clears) both.
//
// Host code cannot use the array's name as a device address: in host code the name is a
// host-side stand-in.  So the first call on each device (with that device current) looks up
// its device address with cudaGetSymbolAddress and caches it; that first call should come
// before any stream capture.  Device code here could name the array directly; the kernels
// receive the looked-up address as an argument.
#include <algorithm>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "xe.h"
#include "xe_host.h"
#include "xe_internal.h"

namespace xe {

static __device__ __align__(256) uint8_t g_noalloc_scratch[XE_NOALLOC_SCRATCH_BYTES];

// Layout of the array: [status | pad][tiles][segments][segment offsets][planes].
constexpr size_t kNaStatusBytes = 256;
constexpr size_t kNaTileBytes = size_t(XE_NOALLOC_MAX_TILES) * sizeof(Tile);
constexpr size_t kNaSegOffset = kNaStatusBytes + kNaTileBytes;
constexpr size_t kNaSegBytes = size_t(XE_NOALLOC_MAX_TILES) * sizeof(Seg);
constexpr size_t kNaOffOffset = kNaSegOffset + kNaSegBytes;
constexpr size_t kNaOffBytes = size_t(XE_NOALLOC_MAX_TILES + 1) * sizeof(int);
constexpr size_t kNaPlaneOffset = (kNaOffOffset + kNaOffBytes + 1023) / 1024 * 1024;
constexpr size_t kNaPlaneBytes = size_t(XE_NOALLOC_SCRATCH_BYTES) - kNaPlaneOffset;
static_assert(kNaPlaneOffset < size_t(XE_NOALLOC_SCRATCH_BYTES), "scratch layout");

constexpr int kMaxDevices = 64;
static uint8_t *g_na_ptr[kMaxDevices] = {nullptr};
static std::mutex g_na_mu;
static int na_fail(int code, const char *msg) { return record_error(code, msg); }

// Enumerate the triangle tiles of one job (same cover and order as the allocating path:
// row blocks of 128, 256-wide column tiles aligned to 256, a 128-wide half tile where a row
// block starts mid-way through a column block) straight into the scratch tile table, with
// one whole-tile segment per CTA.  One thread: at most XE_NOALLOC_MAX_TILES entries.
// status[0] is the live word the kernels of a call set on a timeout; status[1] latches the
// first code left in it by an earlier call until the host reads it.
__global__ void na_tiles_kernel(Tile *tiles, Seg *segs, int *seg_off, int N, int C, int kb,
                                int *status, int first_window) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (first_window) {
        if (status[0] != 0 && status[1] == 0) status[1] = status[0];
        status[0] = 0;
    }
    int k = 0;
    for (int c = 0; c < C; ++c)
        for (int i0 = 0; i0 < N; i0 += kBM) {
            int j0 = i0;
            if (j0 % kBN != 0) {
                tiles[k] = Tile{0, c, i0, j0, kBM, kb, 0, 0};
                segs[k] = Seg{k, 0, kb, -1};
                seg_off[k] = k;
                ++k;
                j0 += kBM;
            }
            for (; j0 < N; j0 += kBN) {
                tiles[k] = Tile{0, c, i0, j0, kBN, kb, 0, 0};
                segs[k] = Seg{k, 0, kb, -1};
                seg_off[k] = k;
                ++k;
            }
        }
    seg_off[k] = k;
}

static int64_t na_tile_count(int N, int C) {
    int64_t n = 0;
    for (int i0 = 0; i0 < N; i0 += kBM) {
        int j0 = i0;
        if (j0 % kBN != 0) { ++n; j0 += kBM; }
        if (j0 < N) n += (N - j0 + kBN - 1) / kBN;
    }
    return n * C;
}

// Device address of the array on the current device (looked up once per device).
static int na_scratch(uint8_t **out) {
    int dev = 0;
    const cudaError_t ge = cudaGetDevice(&dev);
    if (ge == cudaErrorNoDevice || ge == cudaErrorInsufficientDriver)
        return na_fail(XE_ENODEV, "no usable CUDA device (no device or no driver)");
    if (ge != cudaSuccess) return na_fail(XE_ECUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return na_fail(XE_ENODEV, "device index out of range");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        int major = 0, minor = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        if (!(major == 10 && minor == 3)) return na_fail(XE_ENODEV, "not an sm_103 device");
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return na_fail(XE_ECUDA, "cudaGetSymbolAddress of the no-alloc scratch failed");
        // Both status words start at zero (set-up only: a blocking memset, then a wait).
        e = cudaMemset(p, 0, 2 * sizeof(int));
        if (e == cudaSuccess) e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) return na_fail(XE_ECUDA, "clearing the no-alloc status words failed");
        g_na_ptr[dev] = static_cast<uint8_t *>(p);
    }
    *out = g_na_ptr[dev];
    return XE_OK;
}

}  // namespace xe

using namespace xe;

extern "C" {

int xe_correlate_noalloc(const uint8_t *in, int N, int64_t T, int n_chan, int32_t *vis,
                         void *stream) {
    if (!in || !vis) return na_fail(XE_EINVAL, "null input or output pointer");
    if (N < 1 || T < 1 || n_chan < 1) return na_fail(XE_EINVAL, "N, T and n_chan must be >= 1");
    if (reinterpret_cast<uintptr_t>(vis) & 7) return na_fail(XE_EINVAL, "vis must be 8-byte aligned");
    if (T > XE_MAX_T)
        return na_fail(XE_EOVERFLOW, "xe_correlate_noalloc: T exceeds XE_MAX_T: int32 visibilities could overflow");
    if (N > XE_MAX_N) return na_fail(XE_EINVAL, "xe_correlate_noalloc: N too large");
    const int eb = 1;
    const int ks = samples_per_stage(eb);
    const int n_pad = (N + kNPad - 1) / kNPad * kNPad;
    // Staged planes of one 64-sample block of every channel; the window is as many blocks as
    // the array holds, at most one exact f32 accumulation (option "exact_chunk_t").
    const int64_t block_bytes = int64_t(2) * n_pad * kRowBytes * n_chan;
    const int64_t fit_blocks = int64_t(kNaPlaneBytes) / block_bytes;
    if (fit_blocks < 1)
        return na_fail(XE_EINVAL,
                       "xe_correlate_noalloc: 2 * n_chan * ceil(N/256)*256 * 64 bytes of staged "
                       "operands (one 64-sample block) exceed the fixed scratch");
    const int64_t n_tiles = na_tile_count(N, n_chan);
    if (n_tiles > XE_NOALLOC_MAX_TILES)
        return na_fail(XE_EINVAL, "xe_correlate_noalloc: too many triangle tiles for the fixed scratch");
    const int64_t win_blocks = std::min<int64_t>(fit_blocks, option_exact_chunk_t() / ks);
    const int64_t wt = win_blocks * ks;

    uint8_t *base = nullptr;
    int rc = na_scratch(&base);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int *status = reinterpret_cast<int *>(base);
    Tile *tiles = reinterpret_cast<Tile *>(base + kNaStatusBytes);
    Seg *segs = reinterpret_cast<Seg *>(base + kNaSegOffset);
    int *seg_off = reinterpret_cast<int *>(base + kNaOffOffset);
    uint8_t *planes = base + kNaPlaneOffset;
    const int stall = take_inject_stall();

    int table_kb = -1;            // k-blocks per tile in the tile table now in the array
    for (int64_t t0 = 0; t0 < T; t0 += wt) {
        const int64_t Tw = std::min(T - t0, wt);
        const int64_t kb = (Tw + ks - 1) / ks;
        JobTable jt{};
        jt.n_jobs = 1;
        jt.accumulate = t0 > 0 ? 1 : 0;
        JobDev &jd = jt.jobs[0];
        jd.in = in;
        jd.vis = vis;
        jd.planes = planes;
        jd.T = Tw;
        jd.t0 = t0;
        jd.T_in = T;
        jd.s_c = T * int64_t(N);
        jd.s_t = N;
        jd.s_seg = 0;
        jd.seg = N;
        jd.N = N;
        jd.n_pad = n_pad;
        jd.C = n_chan;
        jd.kblocks = int(kb);
        jd.plane_chan_bytes = kb * 2 * n_pad * kRowBytes;
        jd.vis_chan_elems = int64_t(N) * (N + 1);
        jd.stage_block0 = 0;
        jt.total_stage_blocks = int64_t(n_chan) * kb * (n_pad / 256);

        // One CTA per tile, each covering its whole tile: no tile is split across CTAs, so the
        // split-tile workspace and arrival counters of the allocating path are never touched.
        PlanDev pd{};
        pd.tiles = tiles;
        pd.segs = segs;
        pd.seg_off = seg_off;
        pd.tile_slots = seg_off;      // never read: no tile has partial segments
        pd.n_tiles = int(n_tiles);
        pd.n_cta = int(n_tiles);
        pd.ws = nullptr;
        pd.counters = nullptr;
        pd.status = status;
        pd.inject_stall = t0 == 0 ? stall : 0;

        // The table is rewritten only when the window length changes (the last window), in
        // stream order after the previous window's correlation has read it.
        if (int(kb) != table_kb) {
            na_tiles_kernel<<<1, 32, 0, s>>>(tiles, segs, seg_off, N, n_chan, int(kb), status, t0 == 0 ? 1 : 0);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return na_fail(XE_ECUDA, cudaGetErrorString(e));
            table_kb = int(kb);
        }
        cudaError_t e = launch_stage(jt, eb, s);
        if (e != cudaSuccess) return na_fail(XE_ECUDA, cudaGetErrorString(e));
        e = launch_tc(jt, pd, eb, s);
        if (e != cudaSuccess) return na_fail(XE_ECUDA, cudaGetErrorString(e));
    }
    return XE_OK;
}

int xe_noalloc_status(void *stream) {
    uint8_t *base = nullptr;
    int rc = na_scratch(&base);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return na_fail(XE_ECUDA, cudaGetErrorString(e));
    int st[2] = {0, 0};
    e = cudaMemcpy(st, base, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return na_fail(XE_ECUDA, cudaGetErrorString(e));
    if (st[0] == 0 && st[1] == 0) return XE_OK;
    e = cudaMemsetAsync(base, 0, sizeof st, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return na_fail(XE_ECUDA, cudaGetErrorString(e));
    return na_fail(XE_ETIMEOUT, st[1] != 0 ? "xe_correlate_noalloc: a bounded wait of an earlier call timed out"
                                           : "xe_correlate_noalloc: a bounded wait of the last call timed out");
}

}  // extern "C"
