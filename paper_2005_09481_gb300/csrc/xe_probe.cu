// xe_probe.cu -- measured tensor-core ceilings for the roofline of the correlation kernels.
//
// Two microbenchmarks, each a tight loop of the instructions the correlation kernels issue:
//   kind 0: tcgen05.mma kind::f8f6f4, e4m3 x e4m3 -> f32, M=128, N=256, K=32, operands
//           resident in shared memory (no loads in the loop), one CTA per SM;
//   kind 1: mma.sync m16n8k32 s8 x s8 -> s32, register operands, 8 warps per SM;
//   kind 2: kind 0 while bulk copies stream into shared memory at full speed from a 1 MB
//           source; kind 3: the same from a 64 MB source spread over the whole L2.
// They measure what the instruction streams of the exact correlators can reach on this
// GPU at its current clocks and power limit; the headline roofline still uses the
// measured bf16 peak (x 2 for FP8).
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "xe.h"
#include "xe_internal.h"
#include "xe_ptx.cuh"

namespace xe {

constexpr int kProbeA = 128 * kRowBytes;   // one 128 x 64-byte operand tile
constexpr int kProbeB = 256 * kRowBytes;   // one 256 x 64-byte operand tile

__global__ void __launch_bounds__(128, 1) tc_peak_kernel(int iters, int *status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *A = smem, *Bm = smem + kProbeA;
    uint64_t *done = reinterpret_cast<uint64_t *>(smem + kProbeA + kProbeB);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    // Operands: e4m3 codes of small nonzero integers (values do not change the rate).
    for (int k = threadIdx.x; k < (kProbeA + kProbeB) / 4; k += blockDim.x)
        reinterpret_cast<uint32_t *>(smem)[k] = 0x4A44C038u ^ (uint32_t(k) * 0x01000100u & 0x80008000u);
    if (threadIdx.x == 0) {
        mbar_init(done, 1);
        fence_mbar_init();
    }
    fence_proxy_async_smem();
    if ((threadIdx.x >> 5) == 0) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (threadIdx.x == 0) {
        const uint32_t idesc = idesc_dense(128, 256, 0, 0, false);
        const uint32_t a = smem_u32(A), b = smem_u32(Bm);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const uint64_t ad = sdesc_k_sw64(a + 32u * s), bd = sdesc_k_sw64(b + 32u * s);
                mma_f8f6f4(tmem, ad, bd, idesc, (it | s) ? 1u : 0u);
                mma_f8f6f4(tmem + 256, ad, bd, idesc, (it | s) ? 1u : 0u);
            }
        }
        mma_commit(done);
        const long long t0 = clock64();
        bool ok = true;
        while (!mbar_try_wait(done, 0)) {
            if (clock64() - t0 > kWaitBudgetCycles) { ok = false; break; }
        }
        if (!ok) atomicCAS(status, 0, kStatusTimeoutMma);
    }
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// The same MMA loop while a second thread streams bulk copies (48 KB per round, the
// correlation kernel's bytes per pipeline stage) from an L2-resident buffer into a separate
// two-slot shared ring, as fast as they complete: shows how much concurrent shared-memory
// fill traffic costs the tensor pipe.  copies[blockIdx] receives the number of rounds done.
__global__ void __launch_bounds__(128, 1) tc_peak_fill_kernel(int iters, const uint8_t *src, int64_t span,
                                                              int *status, int *copies) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *A = smem, *Bm = smem + kProbeA;
    uint8_t *ring = smem + kProbeA + kProbeB;                 // 2 x 48 KB
    uint64_t *bars = reinterpret_cast<uint64_t *>(ring + 2 * kStageBytes);
    uint64_t *done = bars + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile uint32_t *stop = tmem_slot + 1;
    for (int k = threadIdx.x; k < (kProbeA + kProbeB) / 4; k += blockDim.x)
        reinterpret_cast<uint32_t *>(smem)[k] = 0x4A44C038u;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(done, 1);
        fence_mbar_init();
        *stop = 0;
    }
    fence_proxy_async_smem();
    if ((threadIdx.x >> 5) == 0) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (threadIdx.x == 0) {
        const uint32_t idesc = idesc_dense(128, 256, 0, 0, false);
        const uint32_t a = smem_u32(A), b = smem_u32(Bm);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const uint64_t ad = sdesc_k_sw64(a + 32u * s), bd = sdesc_k_sw64(b + 32u * s);
                mma_f8f6f4(tmem, ad, bd, idesc, (it | s) ? 1u : 0u);
                mma_f8f6f4(tmem + 256, ad, bd, idesc, (it | s) ? 1u : 0u);
            }
        }
        mma_commit(done);
        const long long t0 = clock64();
        bool ok = true;
        while (!mbar_try_wait(done, 0)) {
            if (clock64() - t0 > kWaitBudgetCycles) { ok = false; break; }
        }
        if (!ok) atomicCAS(status, 0, kStatusTimeoutMma);
        *stop = 1;
    } else if (threadIdx.x == 32) {
        uint32_t ph[2] = {0, 0};
        int rounds = 0;
        for (int slot = 0; *stop == 0; slot ^= 1, ++rounds) {
            if (rounds >= 2) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&bars[slot], ph[slot])) {
                    if (clock64() - t0 > kWaitBudgetCycles) { atomicCAS(status, 0, kStatusTimeoutProducer); break; }
                }
                ph[slot] ^= 1u;
            }
            mbar_arrive_expect_tx(&bars[slot], kStageBytes);
            const int64_t base = (int64_t(blockIdx.x) * 2654435761LL + int64_t(rounds) * kStageBytes) %
                                 (span - kStageBytes) / 1024 * 1024;
            for (int c = 0; c < 3; ++c)
                bulk_g2s(ring + slot * kStageBytes + c * 16384, src + base + c * 16384, 16384, &bars[slot]);
        }
        // Drain the copies still in flight.
        for (int k = 0; k < 2 && k < rounds; ++k) {
            const int slot = (rounds - 1 - k) & 1;
            const long long t0 = clock64();
            while (!mbar_try_wait(&bars[slot], ph[slot]) && clock64() - t0 < kWaitBudgetCycles) {}
            ph[slot] ^= 1u;
        }
        copies[blockIdx.x] = rounds;
    }
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

__global__ void __launch_bounds__(256) imma_peak_kernel(int iters, int *sink) {
    uint32_t a[4] = {threadIdx.x * 0x01010101u, 0x02030405u, 0x0708090Au, 0x0B0C0D0Eu};
    uint32_t b0 = 0x01FF01FFu ^ threadIdx.x, b1 = 0x03050709u;
    int acc[8][4] = {};
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+r"(acc[k][0]), "+r"(acc[k][1]), "+r"(acc[k][2]), "+r"(acc[k][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
    int s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += acc[k][0] + acc[k][1] + acc[k][2] + acc[k][3];
    if (s == 0x7fffffff) sink[threadIdx.x] = s;   // keep the loop alive
}

}  // namespace xe

using namespace xe;

extern "C" int xe_peak_probe(int kind, double *tflops_out, double *aux_out) {
    if (!tflops_out || kind < 0 || kind > 3) return record_error(XE_EINVAL, "bad probe request");
    int dev = 0, n_sm = 0;
    const cudaError_t ge = cudaGetDevice(&dev);
    if (ge == cudaErrorNoDevice || ge == cudaErrorInsufficientDriver)
        return record_error(XE_ENODEV, "no usable CUDA device (no device or no driver)");
    if (ge != cudaSuccess) return record_error(XE_ECUDA, "cudaGetDevice failed");
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    int *status = nullptr;
    uint8_t *src = nullptr;
    const size_t src_bytes = kind == 3 ? (size_t(64) << 20) : (size_t(1) << 20) + 65536;
    if (cudaMalloc(&status, 2048 * sizeof(int)) != cudaSuccess) return record_error(XE_ENOMEM, "probe scratch");
    if (kind >= 2 && cudaMalloc(&src, src_bytes) != cudaSuccess) {
        cudaFree(status);
        return record_error(XE_ENOMEM, "probe scratch");
    }
    cudaMemset(status, 0, 2048 * sizeof(int));
    if (src) cudaMemset(src, 0x38, src_bytes);
    int *copies = status + 1024;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double flops = 0;
    float ms = 0;
    int rc = XE_OK;
    const int iters = 20000;
    if (kind == 0) {
        const int smem = kProbeA + kProbeB + 1024 + 64;
        cudaFuncSetAttribute(tc_peak_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        tc_peak_kernel<<<n_sm, 128, smem>>>(200, status);   // warm-up
        cudaEventRecord(e0);
        tc_peak_kernel<<<n_sm, 128, smem>>>(iters, status);
        cudaEventRecord(e1);
        flops = double(n_sm) * iters * 4.0 * 2.0 * 128 * 256 * 32;
    } else if (kind >= 2) {
        const int smem = kProbeA + kProbeB + 2 * kStageBytes + 1024 + 64;
        cudaFuncSetAttribute(tc_peak_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        tc_peak_fill_kernel<<<n_sm, 128, smem>>>(200, src, int64_t(src_bytes), status, copies);
        cudaEventRecord(e0);
        tc_peak_fill_kernel<<<n_sm, 128, smem>>>(iters, src, int64_t(src_bytes), status, copies);
        cudaEventRecord(e1);
        flops = double(n_sm) * iters * 4.0 * 2.0 * 128 * 256 * 32;
    } else {
        const int blocks = n_sm * 4;
        imma_peak_kernel<<<blocks, 256>>>(200, status);
        cudaEventRecord(e0);
        imma_peak_kernel<<<blocks, 256>>>(iters, status);
        cudaEventRecord(e1);
        flops = double(blocks) * 8 * iters * 8.0 * 2.0 * 16 * 8 * 32;
    }
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        rc = record_error(XE_ECUDA, cudaGetErrorString(e));
    } else {
        cudaEventElapsedTime(&ms, e0, e1);
        int st = 0;
        cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
        if (st != 0) rc = record_error(XE_ETIMEOUT, "probe wait timed out");
        *tflops_out = flops / (double(ms) * 1e-3) / 1e12;
        if (aux_out && kind >= 2) {
            std::vector<int> rounds(size_t(n_sm), 0);
            cudaMemcpy(rounds.data(), copies, size_t(n_sm) * sizeof(int), cudaMemcpyDeviceToHost);
            double total = 0;
            for (int r : rounds) total += double(r) * kStageBytes;
            *aux_out = total / (double(ms) * 1e-3) / 1e9;   // GB/s of shared-memory fill
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(status);
    if (src) cudaFree(src);
    return rc;
}
