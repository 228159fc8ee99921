// xe_imma.cu -- exact int8 warp-level tensor-core correlation (legacy mma.sync path).
//
// Same operation as the tcgen05 path (Denman et al. 2020, sections 1 and 2.2:
// V_ij = sum_t x_i(t) conj(x_j(t)) for i <= j), written as two real GEMMs over K = 2T by
// interleaving the real and imaginary parts of each sample along K:
//     u_i(t) = (a_i(t), b_i(t)),  w_j(t) = (-b_j(t), a_j(t)),
//     Re V_ij = sum_k u_i[k] u_j[k],   Im V_ij = sum_k u_i[k] w_j[k].
// mma.sync.m16n8k32 s8 x s8 -> s32 accumulates in int32, so the path is exact by
// construction.  It decodes the packed bytes itself (no staging pass) and serves as the
// integer-exact anchor for the tensor-core kernel and as the int8 mma.sync baseline.
//
// One CTA computes a 64 x 64 block of baselines of one channel over all T; 4 warps, each a
// 32 x 32 quadrant.  Grid: every (job, channel, I-block <= J-block).
#include <cstdint>
#include <cuda_runtime.h>

#include "xe_internal.h"

namespace xe {

constexpr int kImmaB = 64;     // inputs per block side
constexpr int kImmaKT = 32;    // samples per iteration (64 int8 K-elements)
constexpr int kImmaRow = 80;   // padded shared row (64 bytes + 16)

__device__ __forceinline__ void mma_s8(int (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int sext4(uint32_t nib) { return int(nib ^ 8u) - 8; }

__global__ void __launch_bounds__(128) imma_kernel(const __grid_constant__ JobTable jt) {
    __shared__ __align__(16) int8_t Ui[kImmaB][kImmaRow];
    __shared__ __align__(16) int8_t Uj[kImmaB][kImmaRow];
    __shared__ __align__(16) int8_t Wj[kImmaB][kImmaRow];

    // Locate (job, channel, I, J).
    const int64_t blk = blockIdx.x;
    int q = 0;
    {
        int lo = 0, hi = jt.n_jobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jt.jobs[mid].stage_block0 <= blk) lo = mid; else hi = mid - 1;
        }
        q = lo;
    }
    const JobDev &jb = jt.jobs[q];
    const int nb = (jb.N + kImmaB - 1) / kImmaB;
    const int64_t per_chan = int64_t(nb) * (nb + 1) / 2;
    int64_t local = blk - jb.stage_block0;
    const int c = int(local / per_chan);
    int64_t rem = local % per_chan;
    int I = 0;
    while (rem >= nb - I) { rem -= nb - I; ++I; }
    const int J = I + int(rem);
    const int i0 = I * kImmaB, j0 = J * kImmaB;
    const uint8_t *src = jb.in + (int64_t(c) * jb.T_in + jb.t0) * jb.N;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, tig = lane & 3;
    const int wm = warp >> 1, wn = warp & 1;

    int acc_re[2][4][4], acc_im[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int e = 0; e < 4; ++e) { acc_re[a][b][e] = 0; acc_im[a][b][e] = 0; }

    const int ln = tid & 63, th = tid >> 6;
    for (int64_t t0 = 0; t0 < jb.T; t0 += kImmaKT) {
        for (int tt = 0; tt < 16; ++tt) {
            const int tl = th * 16 + tt;
            const int64_t t = t0 + tl;
            uint32_t bi = 0, bj = 0;
            if (t < jb.T) {
                if (i0 + ln < jb.N) bi = src[t * jb.N + i0 + ln];
                if (j0 + ln < jb.N) bj = src[t * jb.N + j0 + ln];
            }
            const int ar = sext4(bi >> 4), ai = sext4(bi & 15u);
            const int br = sext4(bj >> 4), bim = sext4(bj & 15u);
            Ui[ln][2 * tl] = int8_t(ar);
            Ui[ln][2 * tl + 1] = int8_t(ai);
            Uj[ln][2 * tl] = int8_t(br);
            Uj[ln][2 * tl + 1] = int8_t(bim);
            Wj[ln][2 * tl] = int8_t(-bim);
            Wj[ln][2 * tl + 1] = int8_t(br);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const int k0 = ks * 32;
            uint32_t af[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int rb = wm * 32 + mt * 16;
                af[mt][0] = *reinterpret_cast<const uint32_t *>(&Ui[rb + g][k0 + 4 * tig]);
                af[mt][1] = *reinterpret_cast<const uint32_t *>(&Ui[rb + g + 8][k0 + 4 * tig]);
                af[mt][2] = *reinterpret_cast<const uint32_t *>(&Ui[rb + g][k0 + 16 + 4 * tig]);
                af[mt][3] = *reinterpret_cast<const uint32_t *>(&Ui[rb + g + 8][k0 + 16 + 4 * tig]);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int cb = wn * 32 + nt * 8;
                const uint32_t u0 = *reinterpret_cast<const uint32_t *>(&Uj[cb + g][k0 + 4 * tig]);
                const uint32_t u1 = *reinterpret_cast<const uint32_t *>(&Uj[cb + g][k0 + 16 + 4 * tig]);
                const uint32_t w0 = *reinterpret_cast<const uint32_t *>(&Wj[cb + g][k0 + 4 * tig]);
                const uint32_t w1 = *reinterpret_cast<const uint32_t *>(&Wj[cb + g][k0 + 16 + 4 * tig]);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma_s8(acc_re[mt][nt], af[mt], u0, u1);
                    mma_s8(acc_im[mt][nt], af[mt], w0, w1);
                }
            }
        }
        __syncthreads();
    }

    const int64_t N = jb.N;
    int32_t *vis = jb.vis + int64_t(c) * jb.vis_chan_elems;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = i0 + wm * 32 + mt * 16 + g + (e >= 2 ? 8 : 0);
                const int j = j0 + wn * 32 + nt * 8 + 2 * tig + (e & 1);
                if (i < N && j < N && j >= i) {
                    const int64_t k = int64_t(i) * N - (int64_t(i) * (i - 1)) / 2 + (j - i);
                    int2 *p = reinterpret_cast<int2 *>(vis + 2 * k);
                    if (jt.accumulate | jb.accumulate) {
                        const int2 o = *p;
                        *p = make_int2(o.x + acc_re[mt][nt][e], o.y + acc_im[mt][nt][e]);
                    } else {
                        *p = make_int2(acc_re[mt][nt][e], acc_im[mt][nt][e]);
                    }
                }
            }
}

// Blocks of the anchor grid for one job: C * nb(nb+1)/2 with nb = ceil(N / 64).
int64_t imma_blocks(int N, int C) {
    const int64_t nb = (N + kImmaB - 1) / kImmaB;
    return int64_t(C) * nb * (nb + 1) / 2;
}

const void *imma_kernel_fn() { return reinterpret_cast<const void *>(imma_kernel); }

cudaError_t launch_imma(const JobTable &jt, cudaStream_t s) {
    if (jt.total_stage_blocks <= 0) return cudaSuccess;
    if (jt.total_stage_blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    imma_kernel<<<unsigned(jt.total_stage_blocks), 128, 0, s>>>(jt);
    return cudaGetLastError();
}

}  // namespace xe
