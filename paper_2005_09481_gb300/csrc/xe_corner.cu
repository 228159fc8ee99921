// xe_corner.cu -- corner turn of cylinder bundles into full-array frames, and pre-sums.
//
// The F-engine's last transpose stage leaves the data as bundles of four frequency channels,
// each holding the inputs of one cylinder only; every X-engine node combines four bundles into
// full-array data for its frequencies (Denman et al. 2020, section 2.1; section 2.3: the node
// completes the transpose; Table tab:computing: "Re-Order and Pre-Sum").  Layouts (readings):
//     bundles  uint8 [n_cyl][T][n_freq][n_in]       one cylinder per bundle
//     frames   uint8 [n_freq][T][n_cyl * n_in]      input n = cyl * n_in + i
//     presums  int32 [n_freq][N][2]                 sum over t of {re, im} of x_n(t)
// The correlation does not need the materialised frames: its staging kernel reads bundles
// through an input view (see JobDev), which performs the same corner turn inside its loads.
//
// corner_turn_kernel  one block per (cylinder, 256-sample block); thread p copies the 16-byte
//                     pieces p of every sample row (contiguous in the bundle and in the frame)
//                     and accumulates the pieces' per-input sums; each block writes its partial
//                     sums to its own slot (no atomics).
// presum_reduce_kernel sums the partial slots per (frequency, input): eight slices of the
//                     slots per element, eight loads in flight each, one atomic add per slice.
#include <cstdint>
#include <cuda_runtime.h>

#include "xe_internal.h"

namespace xe {

constexpr int kCornerTBlock = 256;   // samples per block
constexpr int kCornerRows = 8;       // sample rows per copy iteration

struct CornerDev {
    const uint8_t *bundles;
    uint8_t *frames;
    int32_t *partial;        // [n_tb][n_freq][N][2] or null
    int64_t T;
    int n_cyl, n_freq, n_in;
};

__device__ __forceinline__ void add_sample(uint32_t byte, int &sr, int &si) {
    sr += int(int8_t(byte & 0xF0u)) >> 4;            // high nibble, sign-extended
    si += int(uint32_t(byte) << 28) >> 28;           // low nibble, sign-extended
}

template <int PER>
__global__ void __launch_bounds__(256) corner_turn_kernel(const __grid_constant__ CornerDev cd) {
    const int cyl = int(blockIdx.x % cd.n_cyl);
    const int64_t tb = blockIdx.x / cd.n_cyl;
    const int64_t t_lo = tb * kCornerTBlock;
    const int64_t t_hi = t_lo + kCornerTBlock < cd.T ? t_lo + kCornerTBlock : cd.T;
    const int N = cd.n_cyl * cd.n_in;
    const int per_row = cd.n_in / PER;
    const int P = cd.n_freq * per_row;
    const int64_t in_row = int64_t(cd.n_freq) * cd.n_in;     // bundle bytes per sample
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const int f = p / per_row;
        const int i = (p % per_row) * PER;
        const uint8_t *src = cd.bundles + ((int64_t(cyl) * cd.T + t_lo) * cd.n_freq + f) * cd.n_in + i;
        uint8_t *dst = cd.frames + (int64_t(f) * cd.T + t_lo) * N + int64_t(cyl) * cd.n_in + i;
        int sr[PER], si[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) sr[u] = si[u] = 0;
        const bool sums = cd.partial != nullptr;
        int64_t t = t_lo;
        if (PER == 16) {
            // Packed sums: nibble v XOR 8 = v + 8 in [0, 15]; for each 32-bit word of the
            // piece, the even and odd bytes of the re (and im) nibbles add into 16-bit lanes,
            // which hold at least 4369 samples (a block has 256).  acc[word][0..3] = re even,
            // re odd, im even, im odd.
            uint32_t acc[4][4];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0u;
            auto add_word = [&](uint32_t w, uint32_t (&a)[4]) {
                const uint32_t re = ((w >> 4) & 0x0F0F0F0Fu) ^ 0x08080808u;
                const uint32_t im = (w & 0x0F0F0F0Fu) ^ 0x08080808u;
                a[0] += re & 0x00FF00FFu;
                a[1] += (re >> 8) & 0x00FF00FFu;
                a[2] += im & 0x00FF00FFu;
                a[3] += (im >> 8) & 0x00FF00FFu;
            };
            // kCornerRows rows per iteration: 16 * kCornerRows bytes of loads in flight per
            // thread (the blocks have 128 threads at CHIME's 4 x 512 bundle rows).
            for (; t + kCornerRows <= t_hi; t += kCornerRows) {
                uint4 v[kCornerRows];
#pragma unroll
                for (int r = 0; r < kCornerRows; ++r) v[r] = __ldcs(reinterpret_cast<const uint4 *>(src + r * in_row));
#pragma unroll
                for (int r = 0; r < kCornerRows; ++r) __stcs(reinterpret_cast<uint4 *>(dst + r * int64_t(N)), v[r]);
                if (sums) {
#pragma unroll
                    for (int r = 0; r < kCornerRows; ++r) {
                        add_word(v[r].x, acc[0]);
                        add_word(v[r].y, acc[1]);
                        add_word(v[r].z, acc[2]);
                        add_word(v[r].w, acc[3]);
                    }
                }
                src += kCornerRows * in_row;
                dst += kCornerRows * int64_t(N);
            }
            for (; t < t_hi; ++t) {
                const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(src));
                __stcs(reinterpret_cast<uint4 *>(dst), v);
                if (sums) {
                    add_word(v.x, acc[0]);
                    add_word(v.y, acc[1]);
                    add_word(v.z, acc[2]);
                    add_word(v.w, acc[3]);
                }
                src += in_row;
                dst += N;
            }
            // Unpack: byte u of word q is input 4q + u; lanes hold sum(v + 8).
            const int bias = 8 * int(t_hi - t_lo);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int lane = (u & 1) ? 1 : 0, sh = (u >> 1) * 16;
                    sr[4 * q + u] = int((acc[q][lane] >> sh) & 0xFFFFu) - bias;
                    si[4 * q + u] = int((acc[q][2 + lane] >> sh) & 0xFFFFu) - bias;
                }
        } else {
            for (; t < t_hi; ++t) {
                const uint8_t b = *src;
                *dst = b;
                if (sums) add_sample(b, sr[0], si[0]);
                src += in_row;
                dst += N;
            }
        }
        if (sums) {
            int32_t *out = cd.partial + ((tb * cd.n_freq + f) * N + int64_t(cyl) * cd.n_in + i) * 2;
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                out[2 * u] = sr[u];
                out[2 * u + 1] = si[u];
            }
        }
    }
}

// Thread (e, slice): the partial sums of element e over block slots slice, slice + S, ...
// (eight loads in flight), added into the zeroed pre-sums (S atomics per element).
constexpr int kPresumSlices = 8;

__global__ void presum_reduce_kernel(const int32_t *__restrict__ partial, int64_t n_tb, int64_t per_tb,
                                     int32_t *__restrict__ presums) {
    const int slice = int(blockIdx.y);
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < per_tb;
         e += int64_t(gridDim.x) * blockDim.x) {
        int32_t s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int64_t b = slice;
        for (; b + 7 * kPresumSlices < n_tb; b += 8 * kPresumSlices) {
#pragma unroll
            for (int u = 0; u < 8; ++u) s[u] += __ldcs(partial + (b + u * kPresumSlices) * per_tb + e);
        }
        for (; b < n_tb; b += kPresumSlices) s[0] += __ldcs(partial + b * per_tb + e);
        const int32_t tot = s[0] + s[1] + s[2] + s[3] + s[4] + s[5] + s[6] + s[7];
        if (tot != 0) atomicAdd(presums + e, tot);
    }
}

int64_t corner_partial_elems(int n_cyl, int n_freq, int n_in, int64_t T) {
    const int64_t n_tb = (T + kCornerTBlock - 1) / kCornerTBlock;
    return n_tb * n_freq * int64_t(n_cyl) * n_in * 2;
}

cudaError_t launch_corner_turn(const uint8_t *bundles, int n_cyl, int n_freq, int n_in, int64_t T,
                               uint8_t *frames, int32_t *partial, int32_t *presums, cudaStream_t s) {
    CornerDev cd{bundles, frames, presums ? partial : nullptr, T, n_cyl, n_freq, n_in};
    const int64_t n_tb = (T + kCornerTBlock - 1) / kCornerTBlock;
    const int64_t blocks = n_tb * n_cyl;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    const bool vec = (n_in % 16) == 0 && (reinterpret_cast<uintptr_t>(bundles) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(frames) & 15) == 0 && (int64_t(n_freq) * n_in) % 16 == 0 &&
                     (int64_t(n_cyl) * n_in) % 16 == 0;
    const int P = n_freq * (vec ? n_in / 16 : n_in);
    const int threads = P >= 256 ? 256 : (P + 31) / 32 * 32;
    if (vec) corner_turn_kernel<16><<<unsigned(blocks), threads, 0, s>>>(cd);
    else corner_turn_kernel<1><<<unsigned(blocks), threads, 0, s>>>(cd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !presums) return e;
    const int64_t per_tb = int64_t(n_freq) * n_cyl * n_in * 2;
    e = cudaMemsetAsync(presums, 0, size_t(per_tb) * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int64_t rb = (per_tb + 255) / 256;
    presum_reduce_kernel<<<dim3(unsigned(rb < 4096 ? rb : 4096), kPresumSlices), 256, 0, s>>>(partial, n_tb, per_tb,
                                                                                             presums);
    return cudaGetLastError();
}

}  // namespace xe
