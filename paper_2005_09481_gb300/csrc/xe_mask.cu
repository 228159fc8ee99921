// xe_mask.cu -- valid-sample counts of a flag-masked correlation.
//
// Flags travel with the voltages (Denman et al. 2020, section 2.2 and Table tab:data-flow)
// and RFI excision runs on the GPU ahead of the correlation (Table tab:computing).  With
// per-(sample, input) validity bits f_i(t), a masked correlation sums only the samples
// where both inputs are valid, and its normalisation needs the count of those samples for
// every baseline:
//     n_ij = sum_t f_i(t) f_j(t),   0 <= i <= j < N.
// That is the same contraction as the correlation, over real 0/1 operands.  The masked
// staging kernel writes the validity as an e4m3 operand plane (1.0 / 0), and a "count job"
// of the tensor-core kernel (JobDev::mode & kModeCount) contracts it with one MMA per K
// step instead of four; exact for the same reason as the visibilities (integer partial sums
// below 2^24 per window).  Its Re output holds n_ij; count_extract_kernel below copies (or
// adds) that Re part into the caller's int32 [C][B] counts.
//
// (The 1-bit mma.sync AND + popcount form of the same contraction issues on the legacy
// integer tensor pipe of this part and measured about 30x slower than the count job.)
#include <cstdint>
#include <cuda_runtime.h>

#include "xe_internal.h"

namespace xe {

__global__ void __launch_bounds__(256) count_extract_kernel(const __grid_constant__ CountDev cd) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < cd.n; e += stride) {
        const int32_t v = __ldcs(cd.src + 2 * e);
        cd.counts[e] = cd.accumulate ? cd.counts[e] + v : v;
    }
}

cudaError_t launch_counts(const CountDev &cd, cudaStream_t s) {
    if (cd.n <= 0) return cudaSuccess;
    int dev = 0, n_sm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (cd.n + 255) / 256;
    const int64_t cap = int64_t(n_sm) * 8;
    count_extract_kernel<<<unsigned(want < cap ? want : cap), 256, 0, s>>>(cd);
    return cudaGetLastError();
}

}  // namespace xe
