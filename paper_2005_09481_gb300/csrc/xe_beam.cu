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
//                     16 sample rows end to end, stream the packed bytes of each stage into a
//                     3-deep shared-memory ring with coalesced cp.async (4 lanes per 64-byte
//                     row piece) and convert them to a triple-buffered e4m3 A tile; a ninth warp
//                     streams the weight tiles through a ring of bulk copies and issues the
//                     MMAs; the roles meet on mbarriers.  The converter warps then read tensor
//                     memory and write y[c][t][b][re, im].
#include <cstdint>
#include <cuda_runtime.h>

#include "xe_codes.cuh"
#include "xe_internal.h"
#include "xe_ptx.cuh"

namespace xe {

constexpr int kBeamSub = 2;                         // sub-tiles of 32 inputs (64 B of e4m3) per stage
constexpr int kBeamASub = kBeamRows * 64;           // 8 KB
constexpr int kBeamABuf = kBeamSub * kBeamASub;     // 16 KB
constexpr int kBeamABufs = 3;                       // A tiles: conversion waits for stage i - 3
constexpr int kBeamRawSlot = kBeamRows * 64;        // raw ring slot: 64-byte rows, 16-byte pieces
                                                    // XOR-swizzled by (row >> 1) & 3
constexpr int kBeamRawDepth = 3;                    // raw slots: stages in flight = depth - 1
constexpr int kBeamConvThreads = 256;               // 8 converter warps, two threads per row
constexpr int kBeamThreads = kBeamConvThreads + 32; // + 1 MMA / weight-copy warp

int beam_ncols(int B) { return (4 * (B < kBeamMaxPerLaunch ? B : kBeamMaxPerLaunch) + 15) / 16 * 16; }

size_t beam_wt_bytes(int B, int N) {
    const size_t chunks = size_t((N + kBeamChunk - 1) / kBeamChunk);
    return chunks * kBeamSub * size_t(beam_ncols(B)) * 64;
}

// Weight ring for an MMA width: `depth` slots, copies issued `ahead` stages early.  The copy
// of stage j reuses the slot of stage j - depth, so issuing it (at stage j - ahead) waits for
// the MMAs of stage j - depth, depth - ahead = 3 stages back.  Up to 64 columns two CTAs fit
// on an SM (<= 114 KB each, the 1 KB per-CTA reservation included); wider MMAs run one CTA
// per SM and take the deeper ring.
__host__ __device__ constexpr int beam_w_depth(int ncols) {
    return ncols <= 48 ? 5 : ncols <= 64 ? 4 : ncols <= 128 ? 5 : 4;
}
__host__ __device__ constexpr int beam_w_ahead(int ncols) { return beam_w_depth(ncols) - 3; }

static int beam_smem_bytes(int ncols) {
    return 1024 /*align*/ + kBeamABufs * kBeamABuf + kBeamRawDepth * kBeamRawSlot +
           beam_w_depth(ncols) * kBeamSub * ncols * 64 + 128 /*barriers, tensor-memory slot*/;
}

// ---- weights -> B operand tiles --------------------------------------------------------

// Exact split of an int8 weight component: w = 16 hi + lo, lo in [-8, 7], hi in [-8, 8].
__device__ __forceinline__ int w_lo(int w) { return ((w + 8) & 15) - 8; }
__device__ __forceinline__ int w_hi(int w) { return (w - w_lo(w)) / 16; }

// One thread per 16-byte piece of the tile image: (chunk k, sub-tile s, row col, piece q)
// holds inputs n = 64k + 32s + 8q .. +7, each as two e4m3 codes {K = (n, im), K = (n, re)}
// (the order the converters produce, the nibble order of a packed sample):
//   Re rows (col % 4 = 0 hi, 2 lo):  { -w_i, w_r }     Im rows (col % 4 = 1 hi, 3 lo): { w_r, w_i }
// of weight beam b0 + col / 4.  Rows past the launch's nb beams and inputs n >= N are zero.
__global__ void beam_weight_kernel(const int8_t *__restrict__ w, int b0, int nb, int N, int ncols,
                                   int n_chunks, uint8_t *__restrict__ wt) {
    const int64_t total = int64_t(n_chunks) * kBeamSub * ncols * 4;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += int64_t(gridDim.x) * blockDim.x) {
        const int q = int(e & 3);
        const int col = int((e >> 2) % ncols);
        const int64_t ks = (e >> 2) / ncols;                 // k * 2 + s
        const int b = col >> 2, part = col & 3;
        uint32_t v[4];
#pragma unroll
        for (int u2 = 0; u2 < 4; ++u2) {
            uint32_t pair = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t n = ks * 32 + 8 * q + 2 * u2 + h;
                int wr = 0, wi = 0;
                if (b < nb && n < N) {
                    wr = w[(int64_t(b0 + b) * N + n) * 2 + 0];
                    wi = w[(int64_t(b0 + b) * N + n) * 2 + 1];
                }
                const bool hi = part < 2;
                const int pr = hi ? w_hi(wr) : w_lo(wr), pi = hi ? w_hi(wi) : w_lo(wi);
                const bool im_row = part & 1;
                const int k_re = im_row ? pi : pr;      // coefficient of the input's re part
                const int k_im = im_row ? pr : -pi;     // coefficient of its im part
                pair |= (encode_small_int(k_im, 1) | (encode_small_int(k_re, 1) << 8)) << (16 * h);
            }
            v[u2] = pair;
        }
        uint8_t *dst = wt + (ks * ncols + col) * 64 + ((q ^ ((col >> 1) & 3)) << 4);
        *reinterpret_cast<uint4 *>(dst) = make_uint4(v[0], v[1], v[2], v[3]);
    }
}

cudaError_t launch_beam_weights(const int8_t *w, int b0, int nb, int N, int ncols, uint8_t *wt, cudaStream_t s) {
    const int n_chunks = (N + kBeamChunk - 1) / kBeamChunk;
    const int64_t total = int64_t(n_chunks) * kBeamSub * ncols * 4;
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

// Roles (see the file header).  Barriers:
//   a_full[buf]   8 converter warps arrive when A tile `buf` holds its stage
//   w_full[slot]  the weight tile of a stage has landed (transaction count)
//   mma_done[buf] the MMAs that read A tile `buf` (and the stage's weight slot) completed
__global__ void __launch_bounds__(kBeamThreads) beam_kernel(const __grid_constant__ BeamDev bd) {
    extern __shared__ uint8_t beam_smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(beam_smem_raw) + 1023) & ~uintptr_t(1023));
    const int w_depth = beam_w_depth(bd.ncols);
    const int w_bytes = kBeamSub * bd.ncols * 64;
    uint8_t *a_buf = smem;                                         // [3][2][128][64]
    uint8_t *raw = smem + kBeamABufs * kBeamABuf;                  // [3][128][64], swizzled
    uint8_t *w_buf = raw + kBeamRawDepth * kBeamRawSlot;           // [w_depth][2][ncols][64]
    uint64_t *mma_done = reinterpret_cast<uint64_t *>(w_buf + w_depth * w_bytes);   // [3]
    uint64_t *a_full = mma_done + kBeamABufs;                                        // [3]
    uint64_t *w_full = a_full + kBeamABufs;                                          // [5]
    uint64_t *drain = w_full + 5;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tiles_per_chan = (bd.T + kBeamRows - 1) / kBeamRows;
    const int c = int(blockIdx.x / tiles_per_chan);
    const int64_t t0 = (blockIdx.x % tiles_per_chan) * kBeamRows;
    volatile int *status = bd.status;
    const uint32_t tmem_cols = bd.ncols <= 32 ? 32u : bd.ncols <= 64 ? 64u : bd.ncols <= 128 ? 128u : 256u;
    const int nk = bd.k_hi - bd.k_lo;

    if (tid == 0) {
        for (int i = 0; i < kBeamABufs; ++i) {
            mbar_init(&mma_done[i], 1);
            mbar_init(&a_full[i], kBeamConvThreads / 32);
        }
        for (int i = 0; i < 5; ++i) mbar_init(&w_full[i], 1);
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
            const int w_ahead = beam_w_ahead(bd.ncols);
            auto issue_w = [&](int i) {
                const int slot = i % w_depth;
                mbar_arrive_expect_tx(&w_full[slot], uint32_t(w_bytes));
                bulk_g2s(w_buf + slot * w_bytes, bd.wt + int64_t(bd.k_lo + i) * w_bytes, uint32_t(w_bytes),
                         &w_full[slot]);
            };
            for (int i = 0; i < w_ahead && i < nk; ++i) issue_w(i);
            const uint32_t idesc = idesc_dense(kBeamRows, uint32_t(bd.ncols), 0, 0, false);
            bool ok = true;
            for (int i = 0; i < nk && ok; ++i) {
                const int buf = i % kBeamABufs, slot = i % w_depth;
                // The weight copy of stage j = i + w_ahead reuses the slot of stage j - w_depth.
                const int j = i + w_ahead;
                if (j < nk) {
                    const int prev = j - w_depth;
                    if (prev >= 0 && !mbar_wait(&mma_done[prev % kBeamABufs],
                                                uint32_t(prev / kBeamABufs) & 1u, status)) {
                        ok = false;
                        break;
                    }
                    issue_w(j);
                }
                if (!mbar_wait(&a_full[buf], uint32_t(i / kBeamABufs) & 1u, status) ||
                    !mbar_wait(&w_full[slot], uint32_t(i / w_depth) & 1u, status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(a_buf + buf * kBeamABuf), b0 = smem_u32(w_buf + slot * w_bytes);
#pragma unroll
                for (int s2 = 0; s2 < kBeamSub; ++s2)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        mma_f8f6f4(tmem, sdesc_k_sw64(a0 + s2 * kBeamASub + 32 * h),
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
        // Converter warp w owns time rows 16w .. 16w + 15 end to end: it copies their bytes
        // into the raw ring, converts them and arrives on a_full, so the warps never wait on
        // each other.  Stage k -> raw slot: row = time sample, 64 bytes = inputs
        // 64k..64k+63.  Vector path: the warp's 64 pieces of 16 B, piece p = lane + 32 j
        // covers row 16w + p / 4, bytes 16 (p % 4) .. +15 (four adjacent lanes read one row's
        // 64 contiguous bytes).  Outside [0,T) x [0,N) the slot holds zeros (value 0 + 0i).
        const int r = 16 * warp + (lane >> 1), half = lane & 1;   // conversion: row r, sub-tile `half`
        auto issue_raw = [&](int k, int slot) {
            uint8_t *dst = raw + slot * kBeamRawSlot;
            if (vec) {
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int p = lane + 32 * j;
                    const int row = 16 * warp + (p >> 2), col = (p & 3) * 16;
                    const int64_t t = t0 + row;
                    const int64_t n = int64_t(k) * kBeamChunk + col;
                    const bool ok = t < bd.T && n < bd.N;
                    beam_cp_async16(dst + row * 64 + ((col >> 4) ^ ((row >> 1) & 3)) * 16,
                                    ok ? static_cast<const void *>(chan + t * bd.N + n) : static_cast<const void *>(bd.in),
                                    ok ? 16u : 0u);
                }
            } else {
                const int64_t t = t0 + r;
                for (int b = 0; b < 32; ++b) {
                    const int col = 32 * half + b;
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
        for (int i = 0; i < nk; ++i) {
            const int buf = i % kBeamABufs;
            asm volatile("cp.async.wait_group %0;" ::"n"(kAhead - 1) : "memory");
            // The warp's copies of stage i have landed (byte stores of the scalar path
            // included) and its lanes have finished reading stage i - 1 from the slot that is
            // refilled below.
            __syncwarp();
            if (i + kAhead < nk) issue_raw(bd.k_lo + i + kAhead, (i + kAhead) % kBeamRawDepth);
            asm volatile("cp.async.commit_group;" ::: "memory");
            // A tile `buf` is free once the MMAs of stage i - 3 have completed; the warp
            // decides together (a lane that gave up stops the whole warp).
            const bool free_ok = i < kBeamABufs ||
                                 mbar_wait(&mma_done[buf], uint32_t((i - kBeamABufs) / kBeamABufs) & 1u, status);
            if (__any_sync(0xffffffffu, !free_ok)) {
                ok = false;
                break;
            }
            // Row r, inputs 32 half .. +31: 8 raw words -> 16 words of {im, re} e4m3 pairs;
            // 16-byte piece q = inputs 8q..8q+7, XOR-swizzled by row.
            const uint8_t *src = raw + (i % kBeamRawDepth) * kBeamRawSlot + r * 64;
            const int sw = (r >> 1) & 3;
            const uint4 w0 = *reinterpret_cast<const uint4 *>(src + (((2 * half) ^ sw) << 4));
            const uint4 w1 = *reinterpret_cast<const uint4 *>(src + (((2 * half + 1) ^ sw) << 4));
            const uint32_t rw[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
            uint8_t *dst = a_buf + buf * kBeamABuf + half * kBeamASub + r * 64;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t o[4];
#pragma unroll
                for (int u = 0; u < 2; ++u) e4m3_of_bytes_nibble_order(rw[2 * q + u], o[2 * u], o[2 * u + 1]);
                *reinterpret_cast<uint4 *>(dst + ((q ^ ((r >> 1) & 3)) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
            }
            fence_proxy_async_smem();
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
            const int64_t t = t0 + 32 * (warp & 3) + lane;
            int32_t *yrow = bd.y + ((int64_t(c) * bd.T + t) * bd.B_total + bd.b0) * 2;
            for (int c0 = 32 * (warp >> 2); c0 < bd.ncols; c0 += 64) {
                uint32_t v[32];
                tmem_ld_32x32b_x32(tmem + (uint32_t((warp & 3) * 32) << 16) + uint32_t(c0), v);
                tmem_ld_wait();
                if (t < bd.T) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int b = c0 / 4 + j;
                        if (b < bd.B) {
                            yrow[2 * b] = 16 * __float2int_rn(__uint_as_float(v[4 * j + 0])) +
                                          __float2int_rn(__uint_as_float(v[4 * j + 2]));
                            yrow[2 * b + 1] = 16 * __float2int_rn(__uint_as_float(v[4 * j + 1])) +
                                              __float2int_rn(__uint_as_float(v[4 * j + 3]));
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
    beam_kernel<<<unsigned(blocks), kBeamThreads, smem, s>>>(bd);
    return cudaGetLastError();
}

}  // namespace xe
