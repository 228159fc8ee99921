// xe_beam.cu -- phased-array beams on the tensor cores.
//
// Besides the correlation, the X-engine nodes form phased-array beams for pulsar timing
// (Denman et al. 2020, section 2.1; "Pulsar Beamforming" in Table tab:computing):
//     y_b(t) = sum_i w_{b,i} x_i(t),   b < B,
// a dense complex contraction over the N inputs for every time sample.  In real form, with
// x = a + i c and w = wr + i wi,
//     Re y_b = sum_i (wr a - wi c),    Im y_b = sum_i (wi a + wr c).
// Each int8 weight component is split exactly as w = 16 w_hi + w_lo with w_lo in [-8, 7] and
// w_hi in [-8, 8], so every operand is an integer of magnitude <= 16, exact in FP8 e4m3:
//     D[t][col] = sum_k X'[t][k] W'[col][k],   K = 2N (per input: im at 2n, re at 2n + 1),
//     col = 4b + {0: Re hi, 1: Im hi, 2: Re lo, 3: Im lo},   y_b = 16 D[hi] + D[lo],
// one tcgen05 kind::f8f6f4 MMA chain per 128 time samples, f32 accumulation in tensor memory.
// Exact: every partial sum is an integer of magnitude <= 128 N < 2^24 (N <= 65536).
//
// beam_weight_kernel  int8 w[B][N][2] -> e4m3 B-operand tiles [chunk][2][ncols][64 B] in the
//                     64-byte-swizzled image the MMA reads (one bulk copy per stage).
// beam_kernel         one CTA per (channel, 128 samples).  Eight converter warps, each owning
//                     half of every stage's bytes for 32 sample rows end to end, stream the
//                     packed bytes into a 3-deep shared-memory ring with cp.async (whole
//                     32-byte sectors) and convert them into a ring of four e4m3 A tiles held
//                     in tensor memory (tcgen05.st; the MMA reads A from there, so the A tiles
//                     cost no shared-memory bandwidth); a ninth warp streams the weight tiles
//                     through a ring of bulk copies and issues the MMAs; the roles meet on
//                     mbarriers.  The converter warps then read the accumulator and write
//                     y[c][t][b][re, im].
#include <cstdint>
#include <cuda_runtime.h>

#include "xe_codes.cuh"
#include "xe_internal.h"
#include "xe_ptx.cuh"

namespace xe {

constexpr int kBeamSub = 2;                         // weight sub-tiles of 32 inputs (64 B of e4m3) per stage
constexpr int kBeamACols = 32;                      // tensor-memory columns of one A tile (128 B per row)
constexpr int kBeamABufs = 4;                       // A tiles: conversion waits for stage i - 4
constexpr int kBeamRawSlot = kBeamRows * 64;        // raw ring slot: 64-byte rows, 16-byte pieces
                                                    // XOR-swizzled by (row >> 1) & 3
constexpr int kBeamRawDepth = 3;                    // raw slots: stages in flight = depth - 1
constexpr int kBeamConvThreads = 256;               // 8 converter warps, two per tensor-memory lane quarter
constexpr int kBeamThreads = kBeamConvThreads + 32; // + 1 MMA / weight-copy warp

int beam_ncols(int B) { return (4 * (B < kBeamMaxPerLaunch ? B : kBeamMaxPerLaunch) + 15) / 16 * 16; }

size_t beam_wt_bytes(int B, int N) {
    const size_t chunks = size_t((N + kBeamChunk - 1) / kBeamChunk);
    return chunks * kBeamSub * size_t(beam_ncols(B)) * 64;
}

// Weight ring: 5 slots, copies issued 2 stages early.  The copy of stage j reuses the slot of
// stage j - 5, so issuing it (at stage j - 2) waits for the MMAs of stage j - 5, 3 stages
// back.  Up to 128 columns two CTAs fit on an SM (<= 106 KB of shared memory and 256
// tensor-memory columns each).
constexpr int kBeamWDepth = 5, kBeamWAhead = 2;

static int beam_smem_bytes(int ncols) {
    return 1024 /*align*/ + kBeamRawDepth * kBeamRawSlot + kBeamWDepth * kBeamSub * ncols * 64 +
           128 /*barriers, tensor-memory slot*/;
}

// Tensor-memory columns: the accumulator (ncols rounded up to a power of two, >= 32), then
// the ring of A tiles; the allocation is the next power of two.
__host__ __device__ constexpr uint32_t beam_acc_cols(int ncols) {
    return ncols <= 32 ? 32u : ncols <= 64 ? 64u : ncols <= 128 ? 128u : 256u;
}
__host__ __device__ constexpr uint32_t beam_tmem_cols(int ncols) {
    return beam_acc_cols(ncols) + kBeamABufs * kBeamACols <= 256u ? 256u : 512u;
}

// ---- weights -> B operand tiles --------------------------------------------------------

// Exact split of an int8 weight component: w = 16 hi + lo, lo in [-8, 7], hi in [-8, 8].
__device__ __forceinline__ int w_lo(int w) { return ((w + 8) & 15) - 8; }
__device__ __forceinline__ int w_hi(int w) { return (w - w_lo(w)) / 16; }

// One thread per 32-bit word of the tile image: word u of 16-byte piece q of row col of
// (chunk k, sub-tile s) holds inputs n = 64k + 32s + 8q + 2u and n + 1, each as two e4m3
// codes {K = (n, im), K = (n, re)} (the order the converters produce, the nibble order of a
// packed sample):
//   Re rows (col % 4 = 0 hi, 2 lo):  { -w_i, w_r }     Im rows (col % 4 = 1 hi, 3 lo): { w_r, w_i }
// of weight beam b0 + col / 4.  Rows past the launch's nb beams and inputs n >= N are zero.
// The four weight bytes of the two inputs are one aligned 32-bit load where they can be.
__global__ void beam_weight_kernel(const int8_t *__restrict__ w, int b0, int nb, int N, int ncols,
                                   int n_chunks, uint8_t *__restrict__ wt) {
    const int64_t total = int64_t(n_chunks) * kBeamSub * ncols * 16;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int u2 = int(e & 3), q = int((e >> 2) & 3);
        const int col = int((e >> 4) % ncols);
        const int64_t ks = (e >> 4) / ncols;                 // k * kBeamSub + s
        const int b = col >> 2, part = col & 3;
        const int64_t n0 = ks * 32 + 8 * q + 2 * u2;
        int wv[2][2] = {{0, 0}, {0, 0}};                     // [input][re, im]
        if (b < nb && n0 < N) {
            const int8_t *src = w + (int64_t(b0 + b) * N + n0) * 2;
            if (n0 + 1 < N && (reinterpret_cast<uintptr_t>(src) & 3) == 0) {
                const uint32_t x = *reinterpret_cast<const uint32_t *>(src);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    wv[h][0] = int(int8_t(x >> (16 * h)));
                    wv[h][1] = int(int8_t(x >> (16 * h + 8)));
                }
            } else {
                wv[0][0] = src[0];
                wv[0][1] = src[1];
                if (n0 + 1 < N) {
                    wv[1][0] = src[2];
                    wv[1][1] = src[3];
                }
            }
        }
        const bool hi = part < 2, im_row = part & 1;
        uint32_t pair = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int wr = wv[h][0], wi = wv[h][1];
            const int pr = hi ? w_hi(wr) : w_lo(wr), pi = hi ? w_hi(wi) : w_lo(wi);
            const int k_re = im_row ? pi : pr;      // coefficient of the input's re part
            const int k_im = im_row ? pr : -pi;     // coefficient of its im part
            pair |= (encode_small_int(k_im, 1) | (encode_small_int(k_re, 1) << 8)) << (16 * h);
        }
        uint8_t *dst = wt + (ks * ncols + col) * 64 + ((q ^ ((col >> 1) & 3)) << 4) + 4 * u2;
        *reinterpret_cast<uint32_t *>(dst) = pair;
    }
}

cudaError_t launch_beam_weights(const int8_t *w, int b0, int nb, int N, int ncols, uint8_t *wt, cudaStream_t s) {
    const int n_chunks = (N + kBeamChunk - 1) / kBeamChunk;
    const int64_t total = int64_t(n_chunks) * kBeamSub * ncols * 16;
    const int64_t blocks = (total + 255) / 256;
    beam_weight_kernel<<<unsigned(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(w, b0, nb, N, ncols, n_chunks, wt);
    return cudaGetLastError();
}

// ---- the beam kernel -------------------------------------------------------------------

__device__ __forceinline__ void beam_cp_async16(void *dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

// D (tensor memory) [+]= A (tensor memory: row m in lane m, 4 e4m3 values of K per 32-bit
// column) x B (shared-memory descriptor), kind::f8f6f4, f32 accumulation.
__device__ __forceinline__ void mma_f8f6f4_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                                  uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Warp-collective store of 16 consecutive 32-bit columns: thread l writes lane
// (taddr lane) + l, register i to column (taddr column) + i.
__device__ __forceinline__ void tmem_st_32x32b_x16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Roles (see the file header).  Barriers:
//   a_full[buf]   8 converter warps arrive when A tile `buf` (tensor memory) holds its stage
//   w_full[slot]  the weight tile of a stage has landed (transaction count)
//   mma_done[buf] the MMAs that read A tile `buf` (and the stage's weight slot) completed
__global__ void __launch_bounds__(kBeamThreads) beam_kernel(const __grid_constant__ BeamDev bd) {
    extern __shared__ uint8_t beam_smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(beam_smem_raw) + 1023) & ~uintptr_t(1023));
    const int w_bytes = kBeamSub * bd.ncols * 64;
    uint8_t *raw = smem;                                           // [3][128][64], swizzled
    uint8_t *w_buf = raw + kBeamRawDepth * kBeamRawSlot;           // [5][2][ncols][64]
    uint64_t *mma_done = reinterpret_cast<uint64_t *>(w_buf + kBeamWDepth * w_bytes);   // [4]
    uint64_t *a_full = mma_done + kBeamABufs;                                            // [4]
    uint64_t *w_full = a_full + kBeamABufs;                                              // [5]
    uint64_t *drain = w_full + kBeamWDepth;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tiles_per_chan = (bd.T + kBeamRows - 1) / kBeamRows;
    const int c = int(blockIdx.x / tiles_per_chan);
    const int64_t t0 = (blockIdx.x % tiles_per_chan) * kBeamRows;
    volatile int *status = bd.status;
    const uint32_t tmem_cols = beam_tmem_cols(bd.ncols);
    const uint32_t a_col0 = beam_acc_cols(bd.ncols);       // first column of the A ring
    const int nk = bd.k_hi - bd.k_lo;

    if (tid == 0) {
        for (int i = 0; i < kBeamABufs; ++i) {
            mbar_init(&mma_done[i], 1);
            mbar_init(&a_full[i], kBeamConvThreads / 32);
        }
        for (int i = 0; i < kBeamWDepth; ++i) mbar_init(&w_full[i], 1);
        mbar_init(drain, 1);
        fence_mbar_init();
    }
    if (warp == 8) {
        tmem_alloc(tmem_slot, tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 8) {
        // ---------------- weight copies + MMA issue (one thread) ----------------
        if (lane == 0) {
            auto issue_w = [&](int i) {
                const int slot = i % kBeamWDepth;
                mbar_arrive_expect_tx(&w_full[slot], uint32_t(w_bytes));
                bulk_g2s(w_buf + slot * w_bytes, bd.wt + int64_t(bd.k_lo + i) * w_bytes, uint32_t(w_bytes),
                         &w_full[slot]);
            };
            // The weight tiles are written by the preceding kernel in the stream, which this
            // grid may overlap (programmatic dependent launch): wait for its completion first.
            asm volatile("griddepcontrol.wait;" ::: "memory");
            for (int i = 0; i < kBeamWAhead && i < nk; ++i) issue_w(i);
            const uint32_t idesc = idesc_dense(kBeamRows, uint32_t(bd.ncols), 0, 0, false);
            bool ok = true;
            for (int i = 0; i < nk && ok; ++i) {
                const int buf = i % kBeamABufs, slot = i % kBeamWDepth;
                // The weight copy of stage j = i + 2 reuses the slot of stage j - 5.
                const int j = i + kBeamWAhead;
                if (j < nk) {
                    const int prev = j - kBeamWDepth;
                    if (prev >= 0 && !mbar_wait(&mma_done[prev % kBeamABufs],
                                                uint32_t(prev / kBeamABufs) & 1u, status)) {
                        ok = false;
                        break;
                    }
                    issue_w(j);
                }
                if (!mbar_wait(&a_full[buf], uint32_t(i / kBeamABufs) & 1u, status) ||
                    !mbar_wait(&w_full[slot], uint32_t(i / kBeamWDepth) & 1u, status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // MMA (s, h) covers inputs 32 s + 16 h .. +15: A columns 16 s + 8 h .. +7 of the
                // tile, B bytes 32 h .. +31 of weight sub-tile s.
                const uint32_t a0 = tmem + a_col0 + uint32_t(buf * kBeamACols);
                const uint32_t b0 = smem_u32(w_buf + slot * w_bytes);
#pragma unroll
                for (int s2 = 0; s2 < kBeamSub; ++s2)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        mma_f8f6f4_tmem_a(tmem, a0 + uint32_t(16 * s2 + 8 * h),
                                          sdesc_k_sw64(b0 + s2 * bd.ncols * 64 + 32 * h), idesc,
                                          (i > 0 || s2 > 0 || h > 0) ? 1u : 0u);
                mma_commit(&mma_done[buf]);
            }
            if (!ok) {
                atomicCAS(bd.status, 0, kStatusTimeoutMma);
                // Bounded wait for MMAs and copies in flight before the CTA may exit.
                mma_commit(drain);
                const long long c0 = clock64();
                while (!mbar_try_wait(drain, 0) && clock64() - c0 < kWaitBudgetCycles) {}
            }
        }
    } else {
        // ---------------- converters (and the epilogue) ----------------
        const bool vec = (bd.N & 15) == 0 && (reinterpret_cast<uintptr_t>(bd.in) & 15) == 0;
        const uint8_t *chan = bd.in + int64_t(c) * bd.T * bd.N;
        // Warp w serves tensor-memory lanes 32 (w % 4) .. +31 (the lane quarter it may access)
        // and part p = w / 4 of every stage: inputs 32 p .. 32 p + 31, raw bytes 32 p .. +31 of
        // each of its 32 sample rows.  It copies those bytes into the raw ring, converts them
        // and stores them to tensor memory itself, so the warps never wait on each other.
        // Copies: lane l takes rows 32 (w % 4) + (l % 16) + 16 jj, 16-byte piece 2 p + l / 16
        // (lanes l and l + 16 read one whole 32-byte sector).  Outside [0,T) x [0,N) the bytes
        // are zero (value 0 + 0i).
        const int quarter = warp & 3, part = warp >> 2;
        const int r = 32 * quarter + lane;                       // conversion: sample row r
        auto issue_raw = [&](int k, int slot) {
            uint8_t *dst = raw + slot * kBeamRawSlot;
            if (vec) {
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) {
                    const int row = 32 * quarter + (lane & 15) + 16 * jj, piece = 2 * part + (lane >> 4);
                    const int64_t t = t0 + row;
                    const int64_t n = int64_t(k) * kBeamChunk + 16 * piece;
                    const bool ok = t < bd.T && n < bd.N;
                    beam_cp_async16(dst + row * 64 + ((piece ^ ((row >> 1) & 3)) << 4),
                                    ok ? static_cast<const void *>(chan + t * bd.N + n) : static_cast<const void *>(bd.in),
                                    ok ? 16u : 0u);
                }
            } else {
                const int64_t t = t0 + r;
                for (int b = 0; b < 32; ++b) {
                    const int col = 32 * part + b;
                    const int64_t n = int64_t(k) * kBeamChunk + col;
                    dst[r * 64 + ((((col >> 4) ^ ((r >> 1) & 3))) << 4) + (col & 15)] =
                        (t < bd.T && n < bd.N) ? chan[t * bd.N + n] : uint8_t(0);
                }
            }
        };
        constexpr int kAhead = kBeamRawDepth - 1;
        for (int i = 0; i < kAhead; ++i) {
            if (i < nk) issue_raw(bd.k_lo + i, i);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        bool ok = true;
        const int sw = (r >> 1) & 3;
        const uint32_t lane_base = uint32_t(32 * quarter) << 16;
        for (int i = 0; i < nk; ++i) {
            const int buf = i % kBeamABufs;
            asm volatile("cp.async.wait_group %0;" ::"n"(kAhead - 1) : "memory");
            // The warp's copies of stage i have landed (byte stores of the scalar path
            // included) and its lanes have finished reading stage i - 1 from the slot that is
            // refilled below.
            __syncwarp();
            if (i + kAhead < nk) issue_raw(bd.k_lo + i + kAhead, (i + kAhead) % kBeamRawDepth);
            asm volatile("cp.async.commit_group;" ::: "memory");
            // Row r, inputs 32 part .. +31: 8 raw words -> 16 columns of {im, re} e4m3 pairs.
            const uint8_t *src = raw + (i % kBeamRawDepth) * kBeamRawSlot + r * 64;
            const uint4 w0 = *reinterpret_cast<const uint4 *>(src + (((2 * part) ^ sw) << 4));
            const uint4 w1 = *reinterpret_cast<const uint4 *>(src + (((2 * part + 1) ^ sw) << 4));
            const uint32_t rw[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
            uint32_t o[16];
#pragma unroll
            for (int q = 0; q < 8; ++q) e4m3_of_bytes_nibble_order(rw[q], o[2 * q], o[2 * q + 1]);
            // A tile `buf` is free once the MMAs of stage i - 4 have completed; the warp
            // decides together (a lane that gave up stops the whole warp).
            const bool free_ok = i < kBeamABufs ||
                                 mbar_wait(&mma_done[buf], uint32_t((i - kBeamABufs) / kBeamABufs) & 1u, status);
            if (__any_sync(0xffffffffu, !free_ok)) {
                ok = false;
                break;
            }
            tc_fence_after();
            tmem_st_32x32b_x16(tmem + lane_base + a_col0 + uint32_t(buf * kBeamACols + 16 * part), o);
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_full[buf]);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        // Every MMA of this CTA has completed once the last stage's commit has arrived.
        if (ok && nk > 0 &&
            !mbar_wait(&mma_done[(nk - 1) % kBeamABufs], uint32_t((nk - 1) / kBeamABufs) & 1u, status))
            ok = false;
        if (!ok) atomicCAS(bd.status, 0, kStatusTimeoutEpilogue);
        tc_fence_after();
        if (ok && *status == 0) {
            // Tensor-memory lane = row = sample t; column 4b + {Re hi, Im hi, Re lo, Im lo}.
            // Warp w reads lanes 32 (w % 4) .. +31 (lane l: row 32 (w % 4) + l); warps w and
            // w + 4 split the 32-column groups.
            const int64_t t = t0 + r;
            int32_t *yrow = bd.y + ((int64_t(c) * bd.T + t) * bd.B_total + bd.b0) * 2;
            for (int c0 = 32 * part; c0 < bd.ncols; c0 += 64) {
                uint32_t v[32];
                tmem_ld_32x32b_x32(tmem + lane_base + uint32_t(c0), v);
                tmem_ld_wait();
                if (t < bd.T) {
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) {
                        const int b = c0 / 4 + jj;
                        if (b < bd.B) {
                            yrow[2 * b] = 16 * __float2int_rn(__uint_as_float(v[4 * jj + 0])) +
                                          __float2int_rn(__uint_as_float(v[4 * jj + 2]));
                            yrow[2 * b + 1] = 16 * __float2int_rn(__uint_as_float(v[4 * jj + 1])) +
                                              __float2int_rn(__uint_as_float(v[4 * jj + 3]));
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc_fence_after();
        tmem_dealloc(tmem, tmem_cols);
    }
}

cudaError_t launch_beam(const BeamDev &bd, cudaStream_t s) {
    if (bd.ncols < 16 || bd.ncols > 256 || (bd.ncols & 15) || bd.B > kBeamMaxPerLaunch) return cudaErrorInvalidValue;
    const int64_t blocks = int64_t(bd.C) * ((bd.T + kBeamRows - 1) / kBeamRows);
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int smem = beam_smem_bytes(bd.ncols);
    cudaError_t e = cudaFuncSetAttribute(beam_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // Programmatic dependent launch: the grid is set up as soon as the weight preparation ends
    // (no launch gap), and only the weight-copy thread waits for that grid's memory to be
    // visible.  The preparation does not trigger the launch early: beam CTAs running beside
    // its few blocks slowed it down more than the overlap gained (10 beams: 39.1 -> 49.1 us).
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(blocks));
    cfg.blockDim = dim3(kBeamThreads);
    cfg.dynamicSmemBytes = size_t(smem);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, beam_kernel, bd);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace xe
