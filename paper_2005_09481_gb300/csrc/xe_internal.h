// xe_internal.h -- structures shared by the libxe kernels and the host runtime.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "xe.h"

namespace xe {

// ---- tensor-core tiling (tcgen05 path) ------------------------------------------------
constexpr int kBM = 128;           // inputs i per tile (MMA M)
constexpr int kBN = 256;           // inputs j per tile (MMA N; 128 on half tiles)
constexpr int kRowBytes = 64;      // bytes of one operand row per pipeline stage
constexpr int kStages = 4;         // shared-memory pipeline depth
constexpr int kPrefetchStages = 8; // L2 prefetch distance of the plane tiles, in stages
constexpr int kNPad = 256;         // inputs are padded to a multiple of this (zeros)
constexpr int kAPlane = kBM * kRowBytes;              // 8 KB
constexpr int kBPlane = kBN * kRowBytes;              // 16 KB
constexpr int kStageBytes = 2 * kAPlane + 2 * kBPlane;  // 48 KB
constexpr int kTcThreads = 256;    // 4 epilogue warps, 1 producer warp, 1 MMA warp, 2 warps that
                                   // join the eight-warp pair-exchange epilogue
constexpr int kEpiStageBytes = 4 * 32 * 33 * 8;  // per epilogue warp: 32 x 33 int2 transpose buffer
constexpr int kTcSmem = kStages * kStageBytes + kEpiStageBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr int kMaxJobs = 208;      // jobs per launch (passed by value, within the 32 KB limit)

// Samples per stage: 64 with 1-byte (e4m3) operands, 32 with 2-byte (f16) operands.
__host__ __device__ constexpr int samples_per_stage(int elem_bytes) {
    return kRowBytes / elem_bytes;
}

// Largest sample count one f32 tensor-memory accumulator may sum before its partial sums
// could leave the exactly-representable integer range (|partial| <= 128 per sample,
// kept below 2^24).
constexpr int64_t kExactChunkT = (1LL << 24) / 128;  // 131072

// One job as the kernels see it.
struct JobDev {
    const uint8_t *in;        // packed input [C][T][N]
    const uint8_t *planes;    // staged operands [C][kblocks][2][n_pad][64 B]
    int32_t *vis;             // output [C][B][2]
    int64_t T;                // samples in this launch (time window)
    int64_t t0;               // first sample of the window within `in`
    int64_t T_in;             // samples per channel in `in` (row stride over channels)
    int64_t plane_chan_bytes; // bytes of planes per channel
    int64_t vis_chan_elems;   // int32 elements of vis per channel (= 2B)
    int N;
    int n_pad;
    int C;
    int kblocks;              // ceil(T / samples_per_stage)
    int accumulate;           // 1: this job adds into vis (vis += V) even if the launch overwrites
    int mode;                 // kModeMasked | kModeOffsetBinary bits (masked staging only)
    int64_t stage_block0;     // first block of this job in the stage (or anchor) grid
    const uint8_t *flags;     // validity bits [C][T_in][ceil(N/8)] (bit n%8 of byte n/8,
                              // 1 = valid), or null = every sample valid
    uint8_t *count_planes;    // masked job with counts: where the staging kernel writes the
                              // validity planes of its count job (same layout as `planes`,
                              // re slots only), else null
    // Input view: sample (c, t, n) of the job (t counted from the job's first sample) is the
    // byte in + c * s_c + t * s_t + (n / seg) * s_seg + n % seg.  A plain [C][T][N] input has
    // s_c = T N, s_t = N, seg = N; cylinder bundles [n_cyl][T][C][n_in] (the corner turn done
    // by the staging kernel's loads) have s_c = n_in, s_t = C n_in, seg = n_in, s_seg = T C n_in.
    int64_t s_c;
    int64_t s_t;
    int64_t s_seg;
    int seg;
    int tile0;                // implicit plans: tiles of the jobs before this one in the launch
    int tiles_per_chan;       // implicit plans: 256-wide triangle tiles of one channel
};

// Byte address of sample (c, t, n) of a job's input (see JobDev).
__host__ __device__ __forceinline__ int64_t view_offset(const JobDev &jb, int c, int64_t t, int n) {
    return int64_t(c) * jb.s_c + t * jb.s_t + int64_t(n / jb.seg) * jb.s_seg + (n % jb.seg);
}

// JobDev::mode bits.  A masked job is staged by the masking variant of the staging kernel:
// each sample byte becomes (byte ^ key) & valid, where key = 0x88 for offset-binary input
// (nibble u encodes u - 8; XOR with 8 gives the two's-complement nibble of the same value)
// and valid = 0xFF if the sample's flag bit is set and it lies inside [0,T) x [0,N).
// A count job correlates the 0/1 validity planes written by its masked job, n_ij =
// sum_t f_i(t) f_j(t), the same contraction over real 0/1 operands (exact for the same
// reason as the visibilities): each k-iteration holds two sample blocks in its re and im
// slots, the MMAs accumulate F_I F_J^T of both into the Re accumulator, and the epilogue
// writes that Re part, n_ij, straight into the caller's int32 [C][B] counts (the count
// job's vis pointer; vis_chan_elems = B).  Its Im accumulator is never formed nor read.
constexpr int kModeMasked = 1;
constexpr int kModeOffsetBinary = 2;
constexpr int kModeCount = 4;

struct JobTable {
    int n_jobs;
    int accumulate;           // 1: add into vis instead of overwriting
    int64_t total_stage_blocks;
    JobDev jobs[kMaxJobs];
    int *status;              // device status word of the launch's stream
    int checks;               // 1 (option "checks"): a descriptor check ran before this launch;
                              // the kernels do nothing once the status word is set
    int reserved;
};

// One output tile of the triangle: rows [i0, i0+128), columns [j0, j0+nj).
struct Tile {
    int job;
    int chan;
    int i0;
    int j0;
    int nj;                   // 256 or 128
    int kblocks;              // k-iterations (pipeline stages) of this tile
    int n_parts;              // segments that each cover part of the tile (0: one whole segment)
    int part_off;             // their workspace slots: tile_slots[part_off .. part_off + n_parts)
};

// A contiguous k-range of one tile processed by one CTA.
struct Seg {
    int tile;
    int k_lo;
    int k_hi;
    int slot;                 // workspace slot if the segment is partial, else -1
};

// Device-resident plan of one persistent launch: CTA b processes segs[seg_off[b] ..
// seg_off[b+1]) in order.
struct PlanDev {
    const Tile *tiles;
    const Seg *segs;
    const int *seg_off;
    const int *tile_slots;
    int n_tiles;
    int n_cta;
    int32_t *ws;              // partial-tile workspace, one slot per partial segment
    int *counters;            // one arrival counter per tile, zero between launches
    int *status;              // device status word (0 = ok)
    int inject_stall;         // test hook: 1 = the producer issues no copies, so waits time out
    int pair_exchange;        // 1: every split tile has 2, 4 or 8 parts (each at least 32
                              // columns wide) and every CTA one segment, all resident: the parts
                              // exchange column slices instead of a last-arriver sum
    int implicit;             // 1: no tile or segment arrays: CTA b takes whole tiles b, b + grid,
                              // ... of the launch, decoded from the job table (implicit_tile)
};

// Triangle schedules (host-side choice; the kernel just follows the segment lists).
enum Sched : int {
    kSchedStreamK = 0,        // equal contiguous ranges of the concatenated k-iterations
    kSchedSplit = 1,          // each tile split into s equal k-parts, parts dealt round-robin;
                              // s from a cost model (mainloop saved against fix-up)
    kSchedHybrid = 2,         // whole tiles in full waves, the last partial wave's tiles split
                              // as in kSchedSplit over the CTAs
    kSchedLPT = 3,            // whole tiles, longest first, to the least-loaded CTA
    kSchedWeighted = 4,       // tiles cut into k-aligned parts of about equal weighted cost
                              // (count jobs weigh less than data jobs), longest part first
                              // to the least-loaded CTA
    kNumSched = 5,
};

constexpr int64_t kWsSlotElems = 2LL * kBN * kBM;  // re and im planes, [col][row] int32

enum DeviceStatus : int {
    kStatusOk = 0,
    kStatusTimeoutProducer = 1,
    kStatusTimeoutMma = 2,
    kStatusTimeoutEpilogue = 3,
    kStatusCheck = 16,        // + the number (0..15) of the descriptor check that failed
};

// What a launch's descriptors may address (option "checks"): the staging scratch and the
// lengths of the plan's device arrays, as allocated on the host.
struct CheckLimits {
    const uint8_t *planes;    // staged operands live in [planes, planes + planes_bytes)
    int64_t planes_bytes;
    int64_t ws_slots;         // workspace slots of kWsSlotElems int32
    int64_t n_counters;       // per-tile arrival counters
    int n_tiles;              // entries of pd.tiles
    int n_segs;               // entries of pd.segs
    int n_seg_off;            // entries of pd.seg_off
    int n_tile_slots;         // entries of pd.tile_slots
};

cudaError_t launch_check(const JobTable &jt, const PlanDev &pd, const CheckLimits &lim, cudaStream_t s);
const void *check_kernel_fn();

// ---- phased-array beams (xe_beam.cu) ---------------------------------------------------

constexpr int kBeamRows = 128;          // time samples per CTA (MMA M)
constexpr int kBeamChunk = 64;          // inputs per pipeline stage (K = 128 e4m3: re, im)
constexpr int kBeamMaxBeams = 128;      // per call
constexpr int kBeamMaxPerLaunch = 64;   // 4 MMA columns per beam (Re/Im x hi/lo), N <= 256

struct BeamDev {
    const uint8_t *in;        // packed input [C][T][N]
    const uint8_t *wt;        // weights as MMA B tiles: [n_chunks][2][ncols][64 B] e4m3, swizzled
    int32_t *y;               // beams [C][T][B_total][2]
    int *status;              // device status word (0 = ok)
    int64_t T;
    int N;
    int C;
    int B_total;              // beams per sample row of y
    int b0;                   // first beam of this launch
    int B;                    // beams of this launch (<= kBeamMaxPerLaunch)
    int ncols;                // MMA N: 4B rounded up to a multiple of 16
    int k_lo, k_hi;           // input chunks [k_lo, k_hi) summed by this launch
};

cudaError_t launch_beam_weights(const int8_t *w, int b0, int nb, int N, int ncols, uint8_t *wt, cudaStream_t s);
cudaError_t launch_beam(const BeamDev &bd, cudaStream_t s);
int beam_ncols(int B);
size_t beam_wt_bytes(int B, int N);

// ---- corner turn (xe_corner.cu) ---------------------------------------------------------

cudaError_t launch_corner_turn(const uint8_t *bundles, int n_cyl, int n_freq, int n_in, int64_t T,
                               uint8_t *frames, int32_t *partial, int32_t *presums, cudaStream_t s);
int64_t corner_partial_elems(int n_cyl, int n_freq, int n_in, int64_t T);

// Kernel launchers (xe_stage.cu, xe_tc.cu, xe_imma.cu).  `masked` selects the masking
// variant of the e4m3 staging kernel (any job with kModeMasked).
cudaError_t launch_stage(const JobTable &jt, int elem_bytes, cudaStream_t s, bool masked = false);
cudaError_t launch_tc(const JobTable &jt, const PlanDev &plan, int elem_bytes, cudaStream_t s);
cudaError_t launch_imma(const JobTable &jt, cudaStream_t s);
int64_t imma_blocks(int N, int C);
int tc_smem_bytes();
const void *stage_kernel_fn(int elem_bytes, bool masked = false);
unsigned stage_grid(const JobTable &jt, int elem_bytes, bool masked = false);
int stage_smem_bytes(int elem_bytes, bool masked = false);
cudaError_t stage_prepare();
const void *tc_kernel_fn(int elem_bytes);
const void *imma_kernel_fn();
cudaError_t tc_prepare();

// Enqueue jobs on stream s in accumulate mode (vis += V), tensor-core path; takes the
// runtime lock.  Used by the streaming server.  Returns an XE_* code.
int run_jobs_accumulate(const struct ::xe_job *jobs, int n_jobs, cudaStream_t s);
// Same, with a per-job choice: accumulate[k] = 1 adds into job k's vis, 0 overwrites it.
int run_jobs_mixed(const struct ::xe_job *jobs, const int *accumulate, int n_jobs, cudaStream_t s);

// Record a failure for xe_last_error() on this thread; returns `code`.
int record_error(int code, const char *msg);

// Host encoders of a small integer as an MMA operand (e4m3 for 1 byte, f16 for 2 bytes).
uint32_t operand_code(int v, int elem_bytes);

// Every kernel takes its JobTable (and PlanDev) by value: keep them within the 32764-byte
// kernel parameter limit.
static_assert(sizeof(JobTable) + sizeof(PlanDev) <= 32000, "kernel parameters too large");

}  // namespace xe
