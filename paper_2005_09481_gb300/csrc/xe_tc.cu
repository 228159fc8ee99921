// xe_tc.cu -- the tensor-core X-engine: operand staging and the tcgen05 correlation kernel.
//
// The X stage of an FX correlator (Denman et al. 2020, sections 1 and 2.2): for every
// channel, V_ij = sum_t x_i(t) conj(x_j(t)) over all i <= j, autocorrelations included.
// With x = a + ib this is four real products,
//     Re V = A_I A_J^T + B_I B_J^T,     Im V = B_I A_J^T - A_I B_J^T,
// where A and B are the real and imaginary planes (inputs x time).  Each is a dense
// integer contraction over time, run here on the 5th-generation tensor cores.
//
// sm_103a has no integer tcgen05 kind, so the operands are carried as FP8 e4m3 (or f16):
// every sample component is an integer in [-8, 7], exactly representable, every product
// is an integer of magnitude <= 64, and every partial sum is an integer of magnitude
// below 2^24 as long as one accumulation covers at most 131072 samples, so the f32
// tensor-memory accumulator holds the exact integer.  The host splits longer integrations.
//
// Kernels:
//   stage_kernel  packed 4+4-bit bytes [T][N] -> per-stage operand planes [kb][re|im][n][64 B]
//                 in the exact shared-memory image the MMA reads (64-byte swizzle), so the
//                 correlation kernel fetches each plane tile with one bulk copy.
//   tc_kernel     persistent, at most one CTA per SM; each CTA follows its list of
//                 segments (a k-range of one triangle tile of one job) from the host plan:
//                 warp 4 streams planes into a 4-stage shared-memory ring with bulk copies,
//                 warp 5 issues tcgen05.mma (M=128, N=256/128, K=32 bytes) into two f32
//                 accumulators in tensor memory (Re: columns 0-255, Im: 256-511),
//                 warps 0-3 drain them (tcgen05.ld), convert to int32 and store the packed
//                 upper triangle.  A tile split into several segments is summed exactly
//                 through a workspace by the last segment to finish (arrival counter, no
//                 spinning on other CTAs).
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "xe_codes.cuh"
#include "xe_internal.h"
#include "xe_ptx.cuh"

namespace xe {

// ---- operand encodings ---------------------------------------------------------------

uint32_t operand_code(int v, int elem_bytes) { return encode_small_int(v, elem_bytes); }

struct NibbleCodes {
    uint16_t c[16];
};
__host__ __device__ constexpr NibbleCodes make_codes(int elem_bytes) {
    NibbleCodes t{};
    for (int n = 0; n < 16; ++n) t.c[n] = uint16_t(encode_small_int(nibble_value(n), elem_bytes));
    return t;
}
__constant__ NibbleCodes c_codes_e4m3 = make_codes(1);
__constant__ NibbleCodes c_codes_f16 = make_codes(2);

// ---- staging kernel ----------------------------------------------------------------------

// Every 16-byte piece of the job's input (16 consecutive inputs of one sample) starts 16-byte
// aligned and lies inside one segment, so the vector load paths apply.
__device__ __forceinline__ bool view_vec_ok(const JobDev &jb) {
    return (jb.N & 15) == 0 && (jb.seg & 15) == 0 && ((jb.s_c | jb.s_t | jb.s_seg) & 15) == 0 &&
           (reinterpret_cast<uintptr_t>(jb.in) & 15) == 0;
}

__device__ __forceinline__ int find_job(const JobTable &jt, int64_t blk) {
    int lo = 0, hi = jt.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jt.jobs[mid].stage_block0 <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One block: KS samples x 256 inputs of one channel -> the re and im plane tiles
// (256 rows x 64 bytes each) of pipeline stage kb.
template <int EB>
__global__ void __launch_bounds__(256) stage_kernel(const __grid_constant__ JobTable jt) {
    constexpr int KS = samples_per_stage(EB);
    __shared__ __align__(16) uint8_t raw[KS][256];
    __shared__ uint32_t lut[256];

    const int tid = threadIdx.x;
    {
        const NibbleCodes &nc = EB == 1 ? c_codes_e4m3 : c_codes_f16;
        lut[tid] = uint32_t(nc.c[tid >> 4]) | (uint32_t(nc.c[tid & 15]) << 16);
    }

    const int64_t blk = blockIdx.x;
    const JobDev &jb = jt.jobs[find_job(jt, blk)];
    const int64_t local = blk - jb.stage_block0;
    const int nblk = jb.n_pad / 256;
    const int nb = int(local % nblk);
    const int64_t rest = local / nblk;
    const int kb = int(rest % jb.kblocks);
    const int c = int(rest / jb.kblocks);
    const int n0 = nb * 256;
    const int64_t t0 = int64_t(kb) * KS;

    // Load the packed [KS][256] tile; zeros outside [0,T) x [0,N) (value 0 + 0i, exact).
    if (view_vec_ok(jb)) {
        const int seg = tid & 15;          // 16-byte segment of the 256-byte row
        for (int r = tid >> 4; r < KS; r += 16) {
            const int64_t t = t0 + r;
            const int n = n0 + seg * 16;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (t < jb.T && n < jb.N)
                v = __ldg(reinterpret_cast<const uint4 *>(jb.in + view_offset(jb, c, jb.t0 + t, n)));
            *reinterpret_cast<uint4 *>(&raw[r][seg * 16]) = v;
        }
    } else {
        for (int r = 0; r < KS; ++r) {
            const int64_t t = t0 + r;
            const int n = n0 + tid;
            raw[r][tid] = (t < jb.T && n < jb.N) ? jb.in[view_offset(jb, c, jb.t0 + t, n)] : uint8_t(0);
        }
    }
    __syncthreads();

    uint8_t *plane0 = const_cast<uint8_t *>(jb.planes) + int64_t(c) * jb.plane_chan_bytes +
                      (int64_t(kb) * 2 * jb.n_pad + n0) * kRowBytes;
    const int64_t im_off = int64_t(jb.n_pad) * kRowBytes;
    if (EB == 1) {
        // Thread: rows n0 + 4g .. +3 (g = tid % 64), 16-sample chunk q = tid / 64 of each.
        // Four 32-bit shared loads give a 4x4 byte block (4 samples x 4 inputs); a byte
        // transpose turns it into 4 samples of each input, and the nibble -> e4m3 table
        // (held in registers) converts them.
        const int g = tid & 63, q = tid >> 6;
        uint32_t re[4][4], im[4][4];                 // [input][word of the 16-byte chunk]
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t w[4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
                w[r] = *reinterpret_cast<const uint32_t *>(&raw[q * 16 + kk * 4 + r][4 * g]);
            const uint32_t a = __byte_perm(w[0], w[1], 0x5140), b = __byte_perm(w[2], w[3], 0x5140);
            const uint32_t cc = __byte_perm(w[0], w[1], 0x7362), d = __byte_perm(w[2], w[3], 0x7362);
            const uint32_t v[4] = {__byte_perm(a, b, 0x5410), __byte_perm(a, b, 0x7632),
                                   __byte_perm(cc, d, 0x5410), __byte_perm(cc, d, 0x7632)};
#pragma unroll
            for (int i = 0; i < 4; ++i) e4m3_of_bytes(v[i], re[i][kk], im[i][kk]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = 4 * g + i;
            uint8_t *pre = plane0 + int64_t(row) * kRowBytes + ((q ^ ((row >> 1) & 3)) << 4);
            *reinterpret_cast<uint4 *>(pre) = make_uint4(re[i][0], re[i][1], re[i][2], re[i][3]);
            *reinterpret_cast<uint4 *>(pre + im_off) = make_uint4(im[i][0], im[i][1], im[i][2], im[i][3]);
        }
    } else {
        // f16 operands: row n0+tid of both planes, 4 chunks of 8 samples each.
        const int row = tid;
        uint8_t *pre = plane0 + int64_t(row) * kRowBytes;
        const int sw = (row >> 1) & 3;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t wr[4], wi[4];
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const uint32_t c0 = lut[raw[q * 8 + w * 2 + 0][tid]];
                const uint32_t c1 = lut[raw[q * 8 + w * 2 + 1][tid]];
                wr[w] = (c0 & 0xFFFFu) | (c1 << 16);
                wi[w] = (c0 >> 16) | (c1 & 0xFFFF0000u);
            }
            const int off = ((q ^ sw) << 4);
            *reinterpret_cast<uint4 *>(pre + off) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
            *reinterpret_cast<uint4 *>(pre + im_off + off) = make_uint4(wi[0], wi[1], wi[2], wi[3]);
        }
    }
}

// Persistent e4m3 staging kernel: each block walks the (job, channel, k-block, 256-input)
// items with a grid stride; the packed [64][256] input tile of the next item streams into
// the other half of a double buffer (cp.async, zero-filled outside [0,T) x [0,N)) while
// the current one is converted, so HBM reads, conversion and plane writes overlap.
constexpr int kStageBlocksPerSm = 4;

__device__ __forceinline__ void cp_async16(void *dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }

struct StageItem {
    int job;                  // index into the job table (read from the kernel parameters at
                              // each use, never through a pointer kept in a register)
    int c, kb, n0;
};

// Decode item blk (32-bit arithmetic: the host keeps every staging grid below 2^31 items).
__device__ __forceinline__ StageItem stage_item(const JobTable &jt, int64_t blk) {
    const int job = find_job(jt, blk);
    const JobDev &jb = jt.jobs[job];
    const uint32_t local = uint32_t(blk - jb.stage_block0);
    const uint32_t nblk = uint32_t(jb.n_pad) / 256u;
    StageItem it;
    it.job = job;
    const uint32_t rest = local / nblk;
    it.n0 = int(local - rest * nblk) * 256;
    const uint32_t c = rest / uint32_t(jb.kblocks);
    it.kb = int(rest - c * uint32_t(jb.kblocks));
    it.c = int(c);
    return it;
}

// Shared layout of one packed input tile: sample t of the 64 is stored at row
// 4 * (t % 16) + t / 16, rows 288 bytes apart, so that the four 16-sample chunks read by the
// four lanes of one input group fall in distinct banks.
constexpr int kRawStride = 288;
__device__ __forceinline__ int raw_row(int t) { return 4 * (t & 15) + (t >> 4); }

constexpr int kStageSmem = 3 * 64 * kRawStride;   // three packed input tiles (dynamic smem)
// The masking variant also rings the validity bits of each tile: 64 rows x 32 bytes
// (256 inputs), rows in the same permuted order as the packed tile.
constexpr int kFlagRowBytes = 32;
constexpr int kStageSmemMasked = kStageSmem + 3 * 64 * kFlagRowBytes;
constexpr int kStageBlocksPerSmMasked = 3;

// Four validity bits (inputs 4g..4g+3) -> a byte mask (bit k -> 0xFF in byte k).  The
// multiply moves bit k to bit 8k (k <= 3, no carries), the AND keeps those bits.
__device__ __forceinline__ uint32_t byte_mask_of_nibble(uint32_t nib) {
    return ((nib * 0x00204081u) & 0x01010101u) * 0xFFu;
}

// MASK = false: the plain conversion.  MASK = true (jobs with kModeMasked): every sample
// byte b becomes (b ^ key) & valid (offset-binary key 0x88; valid from the job's flag bits
// and the [0,T) x [0,N) range), and if the job asks for counts the validity itself is also
// written as an operand plane (e4m3 1.0 or 0) for its count job.
template <bool MASK>
__global__ void __launch_bounds__(256) stage_e4m3_kernel(const __grid_constant__ JobTable jt) {
    constexpr int KS = 64;
    extern __shared__ __align__(16) uint8_t stage_smem[];
    auto raw = reinterpret_cast<uint8_t (*)[KS][kRawStride]>(stage_smem);
    auto fl = reinterpret_cast<uint8_t (*)[KS][kFlagRowBytes]>(stage_smem + kStageSmem);
    const int tid = threadIdx.x;
    const int64_t total = jt.total_stage_blocks;
    // The correlation grid that follows may be set up now: its CTAs need more shared memory
    // than an SM has beside even one staging block, so they only start on SMs this grid has
    // left, and they wait for it to complete before reading the planes.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    auto vec_ok = [&](const JobDev &jb) { return view_vec_ok(jb); };
    // Flag rows can be copied 16 bytes at a time when every row starts 16-byte aligned.
    auto flag_vec_ok = [&](const JobDev &jb) {
        const int64_t frow = (jb.N + 7) / 8;
        return (frow & 15) == 0 && (reinterpret_cast<uintptr_t>(jb.flags) & 15) == 0;
    };
    // Issue the loads of one (decoded) item into buffer b (vector path: N % 16 == 0, aligned
    // input).
    auto issue = [&](const StageItem &it, int b) {
        const JobDev &jb = jt.jobs[it.job];
        const int seg = tid & 15;
        const int n = it.n0 + seg * 16;
        // Inputs n..n+15 lie in one segment: one base per item row, rows s_t apart.
        const uint8_t *src = n < jb.N ? jb.in + view_offset(jb, it.c, jb.t0, n) : jb.in;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = (tid >> 4) + 16 * j;
            const int64_t t = int64_t(it.kb) * KS + r;
            const bool ok = t < jb.T && n < jb.N;
            cp_async16(&raw[b][raw_row(r)][seg * 16], ok ? static_cast<const void *>(src + t * jb.s_t)
                                                 : static_cast<const void *>(jb.in), ok ? 16u : 0u);
        }
        if (MASK && jb.flags && flag_vec_ok(jb) && tid < 128) {
            // Row r, 16-byte half h of the tile's 32 flag bytes; bytes past the end of the
            // flag row are not read (zero-filled), rows past T are zero.
            const int r = tid >> 1, h = tid & 1;
            const int64_t frow = (jb.N + 7) / 8;
            const int64_t t = int64_t(it.kb) * KS + r;
            const int64_t byte0 = it.n0 / 8 + 16 * h;
            const int64_t left = frow - byte0;
            const uint32_t nbytes = (t < jb.T && left > 0) ? uint32_t(left < 16 ? left : 16) : 0u;
            const uint8_t *fsrc = jb.flags + (int64_t(it.c) * jb.T_in + jb.t0 + t) * frow + byte0;
            cp_async16(&fl[b][raw_row(r)][16 * h], nbytes ? static_cast<const void *>(fsrc)
                                                          : static_cast<const void *>(jb.flags), nbytes);
        }
    };

    // Three buffers: the tiles of the next two items are in flight while one is converted.
    // Each item is decoded once, when its loads are issued, and carried to its conversion
    // (it0: the item converted now, it1 and it2: the two behind it).
    int b = 0;
    int64_t blk = blockIdx.x;
    StageItem it0{}, it1{};
    if (blk < total) it0 = stage_item(jt, blk);
    if (blk + gridDim.x < total) it1 = stage_item(jt, blk + gridDim.x);
    if (blk < total && vec_ok(jt.jobs[it0.job])) issue(it0, 0);
    cp_async_commit();
    if (blk + gridDim.x < total && vec_ok(jt.jobs[it1.job])) issue(it1, 1);
    cp_async_commit();
    for (; blk < total; blk += gridDim.x) {
        const StageItem it = it0;
        const JobDev &jb = jt.jobs[it.job];
        const int64_t next = blk + 2 * int64_t(gridDim.x);
        StageItem it2{};
        if (next < total) {
            it2 = stage_item(jt, next);
            if (vec_ok(jt.jobs[it2.job])) issue(it2, b == 0 ? 2 : b - 1);
        }
        cp_async_commit();
        it0 = it1;
        it1 = it2;
        if (!vec_ok(jb)) {
            // Scalar path (unaligned rows or segments, or an unaligned input): byte loads.
            const int n = it.n0 + tid;
            const uint8_t *src = n < jb.N ? jb.in + view_offset(jb, it.c, jb.t0, n) : jb.in;
            for (int r = 0; r < KS; ++r) {
                const int64_t t = int64_t(it.kb) * KS + r;
                raw[b][raw_row(r)][tid] = (t < jb.T && n < jb.N) ? src[t * jb.s_t] : uint8_t(0);
            }
        }
        if (MASK && jb.flags && !(vec_ok(jb) && flag_vec_ok(jb))) {
            // Scalar flag loads: 64 rows x 32 bytes, zero outside the row and past T.
            const int64_t frow = (jb.N + 7) / 8;
            for (int idx = tid; idx < KS * kFlagRowBytes; idx += 256) {
                const int r = idx / kFlagRowBytes, col = idx % kFlagRowBytes;
                const int64_t t = int64_t(it.kb) * KS + r;
                const int64_t byte = it.n0 / 8 + col;
                fl[b][raw_row(r)][col] =
                    (t < jb.T && byte < frow)
                        ? jb.flags[(int64_t(it.c) * jb.T_in + jb.t0 + t) * frow + byte] : uint8_t(0);
            }
        }
        cp_async_wait2();
        __syncthreads();

        uint8_t *plane0 = const_cast<uint8_t *>(jb.planes) + int64_t(it.c) * jb.plane_chan_bytes +
                          (int64_t(it.kb) * 2 * jb.n_pad + it.n0) * kRowBytes;
        const int64_t im_off = int64_t(jb.n_pad) * kRowBytes;
        // Lane l of warp w: input group g = 8w + l/4 (inputs 4g..4g+3), 16-sample chunk q = l%4;
        // the four lanes of a group write the four chunks of a row together (full sectors).
        const int g = (tid >> 5) * 8 + ((tid & 31) >> 2), q = tid & 3;
        // Masking: key, and the validity of inputs 4g..4g+3 inside [0, N).
        uint32_t key = 0, range_nib = 0xFu;
        bool use_flags = false;
        uint32_t vbits[4] = {0u, 0u, 0u, 0u};   // [input]: validity of this lane's 16 samples
                                                // (bit 4 kk + r = sample 16 q + 4 kk + r)
        if (MASK) {
            key = (jb.mode & kModeOffsetBinary) ? 0x88888888u : 0u;
            const int left = jb.N - (it.n0 + 4 * g);
            range_nib = left >= 4 ? 0xFu : left > 0 ? (1u << left) - 1u : 0u;
            use_flags = jb.flags != nullptr;
        }
        const bool want_counts = MASK && jb.count_planes != nullptr;
        uint32_t re[4][4], im[4][4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t w[4], mk[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int tl = q * 16 + kk * 4 + r;
                w[r] = *reinterpret_cast<const uint32_t *>(&raw[b][raw_row(tl)][4 * g]);
                if (MASK) {
                    uint32_t nib = (int64_t(it.kb) * KS + tl < jb.T) ? range_nib : 0u;
                    if (use_flags) nib &= uint32_t(fl[b][raw_row(tl)][g >> 1]) >> ((g & 1) * 4);
                    mk[r] = byte_mask_of_nibble(nib & 0xFu);    // byte i: input 4g + i valid
                    w[r] = (w[r] ^ key) & mk[r];
                }
            }
            if (want_counts) {
                // The same 4x4 byte transpose as the samples below turns the four masks into
                // one word per input (byte s: sample 4 kk + s); the multiply gathers the
                // bytes' low bits into a nibble (bit s lands on bit 28 + s, no carries).
                const uint32_t ma = __byte_perm(mk[0], mk[1], 0x5140), mb = __byte_perm(mk[2], mk[3], 0x5140);
                const uint32_t mc = __byte_perm(mk[0], mk[1], 0x7362), md = __byte_perm(mk[2], mk[3], 0x7362);
                const uint32_t vm[4] = {__byte_perm(ma, mb, 0x5410), __byte_perm(ma, mb, 0x7632),
                                        __byte_perm(mc, md, 0x5410), __byte_perm(mc, md, 0x7632)};
#pragma unroll
                for (int i = 0; i < 4; ++i) vbits[i] |= (((vm[i] & 0x01010101u) * 0x10204080u) >> 28) << (4 * kk);
            }
            const uint32_t a = __byte_perm(w[0], w[1], 0x5140), bb = __byte_perm(w[2], w[3], 0x5140);
            const uint32_t cc = __byte_perm(w[0], w[1], 0x7362), d = __byte_perm(w[2], w[3], 0x7362);
            const uint32_t v[4] = {__byte_perm(a, bb, 0x5410), __byte_perm(a, bb, 0x7632),
                                   __byte_perm(cc, d, 0x5410), __byte_perm(cc, d, 0x7632)};
#pragma unroll
            for (int i = 0; i < 4; ++i) e4m3_of_bytes(v[i], re[i][kk], im[i][kk]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = 4 * g + i;
            uint8_t *pre = plane0 + int64_t(row) * kRowBytes + ((q ^ ((row >> 1) & 3)) << 4);
            *reinterpret_cast<uint4 *>(pre) = make_uint4(re[i][0], re[i][1], re[i][2], re[i][3]);
            *reinterpret_cast<uint4 *>(pre + im_off) = make_uint4(im[i][0], im[i][1], im[i][2], im[i][3]);
        }
        if (want_counts) {
            // Validity plane of the count job: the same rows, chunks and swizzle as the re
            // plane above, one e4m3 byte per sample (0x38 = 1.0 where valid, else 0).  Sample
            // block kb is plane kb of the count job, i.e. slot kb % 2 of its k-iteration kb / 2
            // (a count k-iteration covers two sample blocks); with an odd number of blocks the
            // last block also zeroes the unused slot after it.
            const int64_t cchan = int64_t((jb.kblocks + 1) >> 1) * 2 * jb.n_pad * kRowBytes;
            uint8_t *cplane0 = jb.count_planes + int64_t(it.c) * cchan +
                               (int64_t(it.kb) * jb.n_pad + it.n0) * kRowBytes;
            const bool zero_next = (jb.kblocks & 1) && it.kb == jb.kblocks - 1;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int row = 4 * g + i;
                uint32_t wv[4];
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    wv[kk] = byte_mask_of_nibble((vbits[i] >> (4 * kk)) & 0xFu) & 0x38383838u;
                uint8_t *pc = cplane0 + int64_t(row) * kRowBytes + ((q ^ ((row >> 1) & 3)) << 4);
                *reinterpret_cast<uint4 *>(pc) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                if (zero_next)
                    *reinterpret_cast<uint4 *>(pc + int64_t(jb.n_pad) * kRowBytes) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        __syncthreads();   // raw[b] is refilled by the next iteration's prefetch
        b = b == 2 ? 0 : b + 1;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

static int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

// Grid of the staging launch (also used when the launch is placed in a CUDA graph).
unsigned stage_grid(const JobTable &jt, int elem_bytes, bool masked) {
    if (elem_bytes == 2) return unsigned(jt.total_stage_blocks);
    const int64_t cap = int64_t(sm_count()) * (masked ? kStageBlocksPerSmMasked : kStageBlocksPerSm);
    return unsigned(jt.total_stage_blocks < cap ? jt.total_stage_blocks : cap);
}

int stage_smem_bytes(int elem_bytes, bool masked) {
    return elem_bytes == 1 ? (masked ? kStageSmemMasked : kStageSmem) : 0;
}

cudaError_t stage_prepare() {
    static int done_dev[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done_dev[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(stage_e4m3_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(stage_e4m3_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kStageSmemMasked);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) done_dev[dev] = 1;
    return cudaSuccess;
}

cudaError_t launch_stage(const JobTable &jt, int elem_bytes, cudaStream_t s, bool masked) {
    if (jt.total_stage_blocks <= 0) return cudaSuccess;
    if (jt.total_stage_blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (masked && elem_bytes != 1) return cudaErrorInvalidValue;
    const dim3 grid(stage_grid(jt, elem_bytes, masked));
    if (elem_bytes == 1) {
        cudaError_t e = stage_prepare();
        if (e != cudaSuccess) return e;
        if (masked)
            stage_e4m3_kernel<true><<<grid, 256, kStageSmemMasked, s>>>(jt);
        else
            stage_e4m3_kernel<false><<<grid, 256, kStageSmem, s>>>(jt);
    } else {
        stage_kernel<2><<<grid, 256, 0, s>>>(jt);
    }
    return cudaGetLastError();
}

// ---- persistent tensor-core correlation kernel -----------------------------------------------

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ void set_status(int *status, int code) { atomicCAS(status, 0, code); }

// Store (or add) a 32 x 32 block of final visibilities held by one warp (lane = row
// i0 + lane, register k = column jbase + k).  The block is transposed through the warp's
// shared buffer so that each global access covers 32 consecutive baselines of one row
// (256 contiguous bytes); in accumulate mode all 32 row loads are issued before any add.
// A count job (kModeCount) writes only the Re part, n_ij, into its int32 [C][B] counts (its
// vis pointer and vis_chan_elems = B), 128 contiguous bytes per row.
__device__ __forceinline__ void store_block(const JobDev &jb, int chan, int i0, int jbase,
                                            const int (&re)[32], const int (&im)[32], int acc,
                                            int2 *stage) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 32; ++k) stage[lane * 33 + k] = make_int2(re[k], im[k]);
    __syncwarp();
    const int64_t N = jb.N;
    int32_t *vis = jb.vis + int64_t(chan) * jb.vis_chan_elems;
    const int j = jbase + lane;
    if (jb.mode & kModeCount) {
        // Counts: element k of the row-major upper triangle, Re part only.
        int old[32];
        if (acc) {
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int i = i0 + r;
                old[r] = 0;
                if (i < jb.N && j >= i && j < jb.N) {
                    const int64_t k = int64_t(i) * N - (int64_t(i) * (i - 1)) / 2 + (j - i);
                    old[r] = __ldcg(vis + k);
                }
            }
        }
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const int i = i0 + r;
            if (i < jb.N && j >= i && j < jb.N) {
                const int64_t k = int64_t(i) * N - (int64_t(i) * (i - 1)) / 2 + (j - i);
                vis[k] = (acc ? old[r] : 0) + stage[r * 33 + lane].x;
            }
        }
    } else if (acc) {
        int2 old[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            const int i = i0 + r;
            old[r] = make_int2(0, 0);
            if (i < jb.N && j >= i && j < jb.N) {
                const int64_t k = int64_t(i) * N - (int64_t(i) * (i - 1)) / 2 + (j - i);
                old[r] = __ldcg(reinterpret_cast<const int2 *>(vis + 2 * k));
            }
        }
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            const int i = i0 + r;
            if (i < jb.N && j >= i && j < jb.N) {
                const int64_t k = int64_t(i) * N - (int64_t(i) * (i - 1)) / 2 + (j - i);
                const int2 v = stage[r * 33 + lane];
                *reinterpret_cast<int2 *>(vis + 2 * k) = make_int2(old[r].x + v.x, old[r].y + v.y);
            }
        }
    } else {
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const int i = i0 + r;
            if (i < jb.N && j >= i && j < jb.N) {
                const int64_t k = int64_t(i) * N - (int64_t(i) * (i - 1)) / 2 + (j - i);
                *reinterpret_cast<int2 *>(vis + 2 * k) = stage[r * 33 + lane];
            }
        }
    }
    __syncwarp();
}

// MC = the clustered variant: the two CTAs of a cluster walk equally shaped segment lists
// in lockstep; for `multicast` segments CTA rank r fetches B plane r (re or im) of the shared
// column block for both CTAs, so each CTA reads 2/3 of the B bytes it would read alone.
// Each CTA's MMA completion for a stage arrives on the stage's `empty` barrier of BOTH CTAs
// (multicast commit, barrier count 2), so a producer refills a stage -- its own copies and
// its multicast into the partner -- only after both tensor cores have finished reading it.
template <int EB, bool MC>
__device__ __forceinline__ void tc_body(const JobTable &jt, const PlanDev &plan) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    uint64_t *empty = full + kStages;
    uint64_t *acc_full = empty + kStages;
    uint64_t *acc_empty = acc_full + 1;
    uint64_t *drain = acc_empty + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *epi_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    uint64_t *xfer = drain + 2;    // bulk copy of a partner's share into the idle stages
    int2 *epi_stage = reinterpret_cast<int2 *>(smem + kStages * kStageBytes + 256) + (threadIdx.x >> 5) * 32 * 33;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    volatile int *status = plan.status;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], MC ? 2 : 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 128);
        mbar_init(drain, 1);
        mbar_init(xfer, 1);
        fence_mbar_init();
    }
    if (warp == 5) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (MC) cluster_sync();     // the partner's barriers are initialised before any remote use
    const uint32_t tmem = *tmem_slot;
    const uint32_t rank = MC ? cluster_ctarank() : 0u;   // which B plane this CTA multicasts

    // This CTA's work: segments [q0, q1) of the plan, each a k-range of one tile.
    const int q0 = plan.seg_off[blockIdx.x];
    const int q1 = plan.seg_off[blockIdx.x + 1];
    // A CTA whose only segment is one part of a pair-exchanged tile finishes it with eight
    // warps: the producer and MMA warps are idle by then, and two more warps wait for it.
    const bool wide = !MC && plan.pair_exchange && q1 - q0 == 1 && plan.segs[q0].slot >= 0;
    constexpr uint32_t kFmt = 0;  // E4M3 for kind::f8f6f4, F16 for kind::f16

    if (warp == 4) {
        // ---------------- producer: bulk copies of plane tiles ----------------
        if (lane == 0) {
            // The planes come from the staging kernel just before this one in the stream,
            // which this grid may overlap (programmatic dependent launch): every read of
            // them follows this wait.  Without the launch attribute it returns at once.
            asm volatile("griddepcontrol.wait;" ::: "memory");
            int stage = 0;
            uint32_t ph = 0;
            int64_t fills = 0;
            bool ok = true;
            // Test hook: issue nothing, so the MMA warp's bounded wait runs out.
            for (int q = (!MC && plan.inject_stall) ? q1 : q0; ok && q < q1; ++q) {
                const Seg sg = plan.segs[q];
                const bool null_seg = MC && sg.tile < 0;
                const Tile tl = plan.tiles[null_seg ? 0 : sg.tile];
                const JobDev &jb = jt.jobs[tl.job];
                const uint8_t *pl = jb.planes + int64_t(tl.chan) * jb.plane_chan_bytes;
                const uint32_t bbytes = uint32_t(tl.nj) * kRowBytes;
                for (int64_t k = sg.k_lo; k < sg.k_hi; ++k) {
                    if (!mbar_wait(&empty[stage], ph ^ 1u, status)) {
                        set_status(plan.status, kStatusTimeoutProducer);
                        ok = false;
                        break;
                    }
                    if (null_seg) {
                        mbar_arrive(&full[stage]);     // nothing to load: complete the phase
                        ++fills;
                        if (++stage == kStages) { stage = 0; ph ^= 1u; }
                        continue;
                    }
                    uint8_t *st = smem + stage * kStageBytes;
                    const uint8_t *pre = pl + (k * 2 + 0) * jb.n_pad * int64_t(kRowBytes);
                    const uint8_t *pim = pre + int64_t(jb.n_pad) * kRowBytes;
                    mbar_arrive_expect_tx(&full[stage], 2 * kAPlane + 2 * bbytes);
                    if (k + kPrefetchStages < sg.k_hi) {
                        // Bring the plane tiles of a later stage into L2 ahead of their copy.
                        const uint8_t *fre = pre + int64_t(kPrefetchStages) * 2 * jb.n_pad * kRowBytes;
                        const uint8_t *fim = fre + int64_t(jb.n_pad) * kRowBytes;
                        bulk_prefetch_l2(fre + int64_t(tl.i0) * kRowBytes, kAPlane);
                        bulk_prefetch_l2(fim + int64_t(tl.i0) * kRowBytes, kAPlane);
                        if (!(MC && sg.multicast) || rank == 0) bulk_prefetch_l2(fre + int64_t(tl.j0) * kRowBytes, bbytes);
                        if (!(MC && sg.multicast) || rank == 1) bulk_prefetch_l2(fim + int64_t(tl.j0) * kRowBytes, bbytes);
                    }
                    bulk_g2s(st, pre + int64_t(tl.i0) * kRowBytes, kAPlane, &full[stage]);
                    bulk_g2s(st + kAPlane, pim + int64_t(tl.i0) * kRowBytes, kAPlane, &full[stage]);
                    if (MC && sg.multicast) {
                        // B plane `rank` of the shared column block, into both CTAs.
                        const uint8_t *pb = (rank == 0 ? pre : pim) + int64_t(tl.j0) * kRowBytes;
                        bulk_g2s_multicast(st + 2 * kAPlane + rank * kBPlane, pb, bbytes, &full[stage], 0x3);
                    } else {
                        bulk_g2s(st + 2 * kAPlane, pre + int64_t(tl.j0) * kRowBytes, bbytes, &full[stage]);
                        bulk_g2s(st + 2 * kAPlane + kBPlane, pim + int64_t(tl.j0) * kRowBytes, bbytes,
                                 &full[stage]);
                    }
                    ++fills;
                    if (++stage == kStages) { stage = 0; ph ^= 1u; }
                }
            }
            if (!ok) {
                // Let copies already in flight land before the CTA can exit.
                const int64_t n = fills < kStages ? fills : kStages;
                int s = stage;
                uint32_t p = ph;
                for (int64_t r = 0; r < n; ++r) {
                    if (--s < 0) { s = kStages - 1; p ^= 1u; }
                    const long long t0 = clock64();
                    while (!mbar_try_wait(&full[s], p) && clock64() - t0 < kWaitBudgetCycles) {}
                }
            }
        }
    } else if (warp == 5) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t ph = 0, acc_ph = 0;
            bool ok = true;
            const uint32_t d_re = tmem, d_im = tmem + 256;
            for (int q = q0; ok && q < q1; ++q) {
                const Seg sg = plan.segs[q];
                if (MC && sg.tile < 0) {
                    // Partner-only segment: pass each stage straight back to the producer.
                    for (int64_t k = sg.k_lo; k < sg.k_hi; ++k) {
                        if (!mbar_wait(&full[stage], ph, status)) {
                            set_status(plan.status, kStatusTimeoutMma);
                            ok = false;
                            break;
                        }
                        mma_commit_multicast(&empty[stage], 0x3);
                        if (++stage == kStages) { stage = 0; ph ^= 1u; }
                    }
                    continue;
                }
                const Tile tl = plan.tiles[sg.tile];
                // Count job (plain kernel only): its two slots hold the validity of two
                // consecutive sample blocks, and only the Re accumulator is formed.
                const bool re_only = !MC && (jt.jobs[tl.job].mode & kModeCount);
                const uint32_t idesc = idesc_dense(kBM, uint32_t(tl.nj), kFmt, kFmt, false);
                const uint32_t idesc_neg = idesc_dense(kBM, uint32_t(tl.nj), kFmt, kFmt, true);
                if (!mbar_wait(acc_empty, acc_ph ^ 1u, status)) {
                    set_status(plan.status, kStatusTimeoutMma);
                    ok = false;
                    break;
                }
                acc_ph ^= 1u;
                tc_fence_after();
                // The k-loop, compiled once per operand set: RO = count job.
                auto mainloop = [&](auto ro_tag) {
                    constexpr bool RO = decltype(ro_tag)::value;
                    for (int64_t k = sg.k_lo; k < sg.k_hi; ++k) {
                        if (!mbar_wait(&full[stage], ph, status)) {
                            set_status(plan.status, kStatusTimeoutMma);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t base = smem_u32(smem + stage * kStageBytes);
#pragma unroll
                        for (int s = 0; s < 2; ++s) {
                            const uint32_t off = 32u * s;
                            const uint64_t a_re = sdesc_k_sw64(base + off);
                            const uint64_t a_im = sdesc_k_sw64(base + kAPlane + off);
                            const uint64_t b_re = sdesc_k_sw64(base + 2 * kAPlane + off);
                            const uint64_t b_im = sdesc_k_sw64(base + 2 * kAPlane + kBPlane + off);
                            const uint32_t acc = (k > sg.k_lo || s > 0) ? 1u : 0u;
                            if constexpr (RO) {
                                if (EB == 1) {
                                    mma_f8f6f4(d_re, a_re, b_re, idesc, acc);   // + F_I F_J^T, block 2k
                                    mma_f8f6f4(d_re, a_im, b_im, idesc, 1u);    // + block 2k + 1
                                } else {
                                    mma_f16(d_re, a_re, b_re, idesc, acc);
                                    mma_f16(d_re, a_im, b_im, idesc, 1u);
                                }
                            } else if (EB == 1) {
                                mma_f8f6f4(d_re, a_re, b_re, idesc, acc);      // + A_I A_J^T
                                mma_f8f6f4(d_re, a_im, b_im, idesc, 1u);       // + B_I B_J^T
                                mma_f8f6f4(d_im, a_im, b_re, idesc, acc);      // + B_I A_J^T
                                mma_f8f6f4(d_im, a_re, b_im, idesc_neg, 1u);   // - A_I B_J^T
                            } else {
                                mma_f16(d_re, a_re, b_re, idesc, acc);
                                mma_f16(d_re, a_im, b_im, idesc, 1u);
                                mma_f16(d_im, a_im, b_re, idesc, acc);
                                mma_f16(d_im, a_re, b_im, idesc_neg, 1u);
                            }
                        }
                        if (MC) mma_commit_multicast(&empty[stage], 0x3);
                        else mma_commit(&empty[stage]);
                        if (++stage == kStages) { stage = 0; ph ^= 1u; }
                    }
                };
                if (re_only) mainloop(std::true_type{});
                else mainloop(std::false_type{});
                if (ok) mma_commit(acc_full);
            }
            if (!ok) {
                // Wait (bounded) for every MMA already issued before TMEM is released.
                mma_commit(drain);
                const long long t0 = clock64();
                while (!mbar_try_wait(drain, 0) && clock64() - t0 < kWaitBudgetCycles) {}
            }
        }
    } else if (warp < 4 && !wide) {
        // ---------------- epilogue: TMEM -> int32 -> packed triangle ----------------
        uint32_t acc_ph = 0, xph = 0;
        const int r = warp * 32 + lane;
        const uint32_t lane_base = uint32_t(warp * 32) << 16;
        for (int q = q0; q < q1; ++q) {
            const Seg sg = plan.segs[q];
            if (MC && sg.tile < 0) continue;      // partner-only segment: nothing to drain
            const Tile tl = plan.tiles[sg.tile];
            const JobDev &jb = jt.jobs[tl.job];
            if (threadIdx.x == 0) {
                const bool ok = mbar_wait(acc_full, acc_ph, status);
                if (!ok) set_status(plan.status, kStatusTimeoutEpilogue);
                *epi_flag = ok ? 1 : 0;
            }
            epi_bar();
            if (*epi_flag == 0) break;
            acc_ph ^= 1u;
            tc_fence_after();

            if (sg.slot < 0) {
                for (int cc = 0; cc < tl.nj; cc += 32) {
                    uint32_t fre[32], fim[32];
                    tmem_ld_32x32b_x32(tmem + lane_base + cc, fre);
                    tmem_ld_32x32b_x32(tmem + lane_base + 256 + cc, fim);
                    tmem_ld_wait();
                    int re[32], im[32];
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        re[k] = __float2int_rn(__uint_as_float(fre[k]));
                        im[k] = __float2int_rn(__uint_as_float(fim[k]));
                    }
                    store_block(jb, tl.chan, tl.i0 + warp * 32, tl.j0 + cc, re, im, jt.accumulate | jb.accumulate, epi_stage);
                }
            } else if (!MC && plan.pair_exchange) {
                // Two-part tile, both parts running now on two CTAs: part p finalises column
                // half p.  Publish my share of the partner's half, count myself in, wait
                // (bounded) for the partner's share of mine, then add it to my own sums.
                const int part = sg.k_lo == 0 ? 0 : 1;
                const int half = tl.nj / 2;
                const int mine0 = part * half, theirs0 = (1 - part) * half;
                int32_t *ws = plan.ws + int64_t(sg.slot) * kWsSlotElems;
                for (int cc = 0; cc < half; cc += 32) {
                    uint32_t fre[32], fim[32];
                    tmem_ld_32x32b_x32(tmem + lane_base + theirs0 + cc, fre);
                    tmem_ld_32x32b_x32(tmem + lane_base + 256 + theirs0 + cc, fim);
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        __stcg(ws + int64_t(cc + k) * kBM + r, __float2int_rn(__uint_as_float(fre[k])));
                        __stcg(ws + int64_t(kBN + cc + k) * kBM + r, __float2int_rn(__uint_as_float(fim[k])));
                    }
                }
                __threadfence();
                epi_bar();
                if (threadIdx.x == 0) {
                    atomicAdd(&plan.counters[sg.tile], 1);
                    volatile int *cnt = plan.counters + sg.tile;
                    const long long t0 = clock64();
                    bool ok = true;
                    while (*cnt < 2) {
                        if (*status != 0 || clock64() - t0 > kWaitBudgetCycles) { ok = false; break; }
                    }
                    if (!ok) set_status(plan.status, kStatusTimeoutEpilogue);
                    *epi_flag = ok ? 1 : 0;
                }
                epi_bar();
                if (*epi_flag == 1) {
                    __threadfence();
                    const int32_t *w = plan.ws + int64_t(plan.tile_slots[tl.part_off + (1 - part)]) * kWsSlotElems;
                    // On the CTA's last segment the operand stages are idle (its MMAs have
                    // completed, the producer has nothing left to fetch): one pair of bulk
                    // copies brings the partner's whole share (re and im, half x 128 int32
                    // each) into them, so the chunks below read shared memory instead of
                    // waiting on L2 loads chunk by chunk.
                    const bool staged = q == q1 - 1;
                    const int32_t *sh = reinterpret_cast<const int32_t *>(smem);
                    if (staged) {
                        const uint32_t bytes = uint32_t(half) * kBM * 4u;
                        if (threadIdx.x == 0) {
                            // The share was written through the generic proxy on another SM.
                            asm volatile("fence.proxy.async.global;" ::: "memory");
                            mbar_arrive_expect_tx(xfer, 2u * bytes);
                            bulk_g2s(smem, w, bytes, xfer);
                            bulk_g2s(smem + bytes, w + int64_t(kBN) * kBM, bytes, xfer);
                        }
                        // Bounded wait that does not stop on another CTA's error: the copies
                        // must land before this CTA may exit.
                        const long long t0 = clock64();
                        bool got = false;
                        while (!(got = mbar_try_wait(xfer, xph)) && clock64() - t0 < kWaitBudgetCycles) {}
                        if (!got) set_status(plan.status, kStatusTimeoutEpilogue);
                        xph ^= 1u;
                    }
                    for (int cc = 0; cc < half; cc += 32) {
                        uint32_t fre[32], fim[32];
                        tmem_ld_32x32b_x32(tmem + lane_base + mine0 + cc, fre);
                        tmem_ld_32x32b_x32(tmem + lane_base + 256 + mine0 + cc, fim);
                        int re[32], im[32];
                        if (staged) {
#pragma unroll
                            for (int k = 0; k < 32; ++k) {
                                re[k] = sh[(cc + k) * kBM + r];
                                im[k] = sh[(half + cc + k) * kBM + r];
                            }
                        } else {
#pragma unroll
                            for (int k = 0; k < 32; ++k) {
                                re[k] = __ldcg(w + int64_t(cc + k) * kBM + r);
                                im[k] = __ldcg(w + int64_t(kBN + cc + k) * kBM + r);
                            }
                        }
                        tmem_ld_wait();
#pragma unroll
                        for (int k = 0; k < 32; ++k) {
                            re[k] += __float2int_rn(__uint_as_float(fre[k]));
                            im[k] += __float2int_rn(__uint_as_float(fim[k]));
                        }
                        store_block(jb, tl.chan, tl.i0 + warp * 32, tl.j0 + mine0 + cc, re, im,
                                    jt.accumulate | jb.accumulate, epi_stage);
                    }
                    epi_bar();
                    // Both parts have read each other's share: the second to finish resets the
                    // counter for the next launch.
                    if (threadIdx.x == 0 && atomicAdd(&plan.counters[sg.tile], 1) == 3) plan.counters[sg.tile] = 0;
                }
            } else {
                // Partial tile: publish this segment's share; the last one to arrive sums all.
                int32_t *ws = plan.ws + int64_t(sg.slot) * kWsSlotElems;
                for (int cc = 0; cc < tl.nj; cc += 32) {
                    uint32_t fre[32], fim[32];
                    tmem_ld_32x32b_x32(tmem + lane_base + cc, fre);
                    tmem_ld_32x32b_x32(tmem + lane_base + 256 + cc, fim);
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        __stcg(ws + int64_t(cc + k) * kBM + r, __float2int_rn(__uint_as_float(fre[k])));
                        __stcg(ws + int64_t(kBN + cc + k) * kBM + r,
                               __float2int_rn(__uint_as_float(fim[k])));
                    }
                }
                __threadfence();
                epi_bar();
                if (threadIdx.x == 0) {
                    const int old = atomicAdd(&plan.counters[sg.tile], 1);
                    const bool last = old == tl.n_parts - 1;
                    if (last) plan.counters[sg.tile] = 0;  // ready for the next launch
                    *epi_flag = last ? 2 : 1;
                }
                epi_bar();
                if (*epi_flag == 2) {
                    // Last share to arrive: its own part is still in tensor memory; add the
                    // other shares from the workspace.
                    __threadfence();
                    for (int cc = 0; cc < tl.nj; cc += 32) {
                        uint32_t fre[32], fim[32];
                        tmem_ld_32x32b_x32(tmem + lane_base + cc, fre);
                        tmem_ld_32x32b_x32(tmem + lane_base + 256 + cc, fim);
                        tmem_ld_wait();
                        int re[32], im[32];
#pragma unroll
                        for (int k = 0; k < 32; ++k) {
                            re[k] = __float2int_rn(__uint_as_float(fre[k]));
                            im[k] = __float2int_rn(__uint_as_float(fim[k]));
                        }
                        for (int p = 0; p < tl.n_parts; ++p) {
                            const int slot = plan.tile_slots[tl.part_off + p];
                            if (slot == sg.slot) continue;
                            const int32_t *w = plan.ws + int64_t(slot) * kWsSlotElems;
#pragma unroll
                            for (int k = 0; k < 32; ++k) {
                                re[k] += __ldcg(w + int64_t(cc + k) * kBM + r);
                                im[k] += __ldcg(w + int64_t(kBN + cc + k) * kBM + r);
                            }
                        }
                        store_block(jb, tl.chan, tl.i0 + warp * 32, tl.j0 + cc, re, im, jt.accumulate | jb.accumulate, epi_stage);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acc_empty);
        }
    }

    if (wide) {
        // ---------------- eight-warp pair-exchange epilogue (see `wide`) ----------------
        // Warp w serves tensor-memory lane quarter w % 4 (rows 32 (w % 4) ..) and column share
        // w / 4 of each half; the eight warps meet on named barrier 2 only, every thread
        // taking the same barriers (the conditions are flags read after a barrier).  The
        // steps are those of the four-warp pair exchange in the epilogue role above, with
        // the partner's share always staged through the idle operand stages.
        auto wbar = []() { asm volatile("bar.sync 2, 256;" ::: "memory"); };
        const Seg sg = plan.segs[q0];
        const Tile tl = plan.tiles[sg.tile];
        const JobDev &jb = jt.jobs[tl.job];
        const int quarter = warp & 3, share = warp >> 2;
        const int r = quarter * 32 + lane;
        const uint32_t lane_base = uint32_t(quarter * 32) << 16;
        if (threadIdx.x == 0) {
            const bool ok = mbar_wait(acc_full, 0, status);
            if (!ok) set_status(plan.status, kStatusTimeoutEpilogue);
            *epi_flag = ok ? 1 : 0;
        }
        wbar();
        if (*epi_flag == 1) {
            tc_fence_after();
            const int part = sg.k_lo == 0 ? 0 : 1;
            const int half = tl.nj / 2, cols = half / 2;
            const int mine0 = part * half, theirs0 = (1 - part) * half;
            const int c_lo = share * cols, c_hi = c_lo + cols;
            int32_t *ws = plan.ws + int64_t(sg.slot) * kWsSlotElems;
            for (int cc = c_lo; cc < c_hi; cc += 32) {
                uint32_t fre[32], fim[32];
                tmem_ld_32x32b_x32(tmem + lane_base + theirs0 + cc, fre);
                tmem_ld_32x32b_x32(tmem + lane_base + 256 + theirs0 + cc, fim);
                tmem_ld_wait();
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                    __stcg(ws + int64_t(cc + k) * kBM + r, __float2int_rn(__uint_as_float(fre[k])));
                    __stcg(ws + int64_t(kBN + cc + k) * kBM + r, __float2int_rn(__uint_as_float(fim[k])));
                }
            }
            __threadfence();
            wbar();
            if (threadIdx.x == 0) {
                atomicAdd(&plan.counters[sg.tile], 1);
                volatile int *cnt = plan.counters + sg.tile;
                const long long t0 = clock64();
                bool ok = true;
                while (*cnt < 2) {
                    if (*status != 0 || clock64() - t0 > kWaitBudgetCycles) { ok = false; break; }
                }
                if (!ok) set_status(plan.status, kStatusTimeoutEpilogue);
                *epi_flag = ok ? 1 : 0;
            }
            wbar();
            if (*epi_flag == 1) {
                __threadfence();
                const int32_t *w = plan.ws + int64_t(plan.tile_slots[tl.part_off + (1 - part)]) * kWsSlotElems;
                // The partner's share (re and im, half x 128 int32 each) goes into the idle
                // operand stages in one pair of bulk copies; warps 4..7 take their transpose
                // buffers from the stages after it.
                const uint32_t bytes = uint32_t(half) * kBM * 4u;
                if (threadIdx.x == 0) {
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    mbar_arrive_expect_tx(xfer, 2u * bytes);
                    bulk_g2s(smem, w, bytes, xfer);
                    bulk_g2s(smem + bytes, w + int64_t(kBN) * kBM, bytes, xfer);
                }
                const long long t0 = clock64();
                bool got = false;
                while (!(got = mbar_try_wait(xfer, 0)) && clock64() - t0 < kWaitBudgetCycles) {}
                if (!got) set_status(plan.status, kStatusTimeoutEpilogue);
                const int32_t *sh = reinterpret_cast<const int32_t *>(smem);
                int2 *buf = share == 0 ? epi_stage
                                       : reinterpret_cast<int2 *>(smem + 2 * bytes) + (warp - 4) * 32 * 33;
                for (int cc = c_lo; cc < c_hi; cc += 32) {
                    uint32_t fre[32], fim[32];
                    tmem_ld_32x32b_x32(tmem + lane_base + mine0 + cc, fre);
                    tmem_ld_32x32b_x32(tmem + lane_base + 256 + mine0 + cc, fim);
                    int re[32], im[32];
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        re[k] = sh[(cc + k) * kBM + r];
                        im[k] = sh[(half + cc + k) * kBM + r];
                    }
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        re[k] += __float2int_rn(__uint_as_float(fre[k]));
                        im[k] += __float2int_rn(__uint_as_float(fim[k]));
                    }
                    store_block(jb, tl.chan, tl.i0 + quarter * 32, tl.j0 + mine0 + cc, re, im,
                                jt.accumulate | jb.accumulate, buf);
                }
                wbar();
                // Both parts have read each other's share: the second to finish resets the
                // counter for the next launch.
                if (threadIdx.x == 0 && atomicAdd(&plan.counters[sg.tile], 1) == 3) plan.counters[sg.tile] = 0;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (MC) {
        // Both CTAs are done with each other's barriers and shared memory before either exits;
        // after an abort, give multicast copies already in flight time to land.
        cluster_sync();
        if (*status != 0) {
            const long long t0 = clock64();
            while (clock64() - t0 < 4000000LL) {}
            cluster_sync();
        }
    }
    if (warp == 5) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

template <int EB>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_kernel(const __grid_constant__ JobTable jt, const __grid_constant__ PlanDev plan) {
    tc_body<EB, false>(jt, plan);
}

template <int EB>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kTcThreads, 1)
    tc_mc_kernel(const __grid_constant__ JobTable jt, const __grid_constant__ PlanDev plan) {
    tc_body<EB, true>(jt, plan);
}

int tc_smem_bytes() { return kTcSmem; }

const void *stage_kernel_fn(int elem_bytes, bool masked) {
    if (elem_bytes == 1)
        return masked ? reinterpret_cast<const void *>(stage_e4m3_kernel<true>)
                      : reinterpret_cast<const void *>(stage_e4m3_kernel<false>);
    return reinterpret_cast<const void *>(stage_kernel<2>);
}

const void *tc_kernel_fn(int elem_bytes, bool clustered) {
    if (clustered)
        return elem_bytes == 1 ? reinterpret_cast<const void *>(tc_mc_kernel<1>)
                               : reinterpret_cast<const void *>(tc_mc_kernel<2>);
    return elem_bytes == 1 ? reinterpret_cast<const void *>(tc_kernel<1>)
                           : reinterpret_cast<const void *>(tc_kernel<2>);
}

// Opt the correlation kernels into their dynamic shared memory (once per process/device).
cudaError_t tc_prepare() {
    static int done_dev[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done_dev[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(tc_mc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(tc_mc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) done_dev[dev] = 1;
    return cudaSuccess;
}

// Clusters of two tensor-core CTAs that can be resident at once (0 if the query fails).
int tc_max_clusters() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
    if (tc_prepare() != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * 256);
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = kTcSmem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, reinterpret_cast<const void *>(tc_mc_kernel<1>), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (dev >= 0 && dev < 64) cached[dev] = n;
    return n;
}

cudaError_t launch_tc(const JobTable &jt, const PlanDev &plan, int elem_bytes, cudaStream_t s,
                      bool clustered) {
    if (plan.n_cta <= 0 || plan.n_tiles <= 0) return cudaSuccess;
    if (clustered && (plan.n_cta & 1)) return cudaErrorInvalidValue;
    cudaError_t e = tc_prepare();
    if (e != cudaSuccess) return e;
    if (clustered) {
        if (elem_bytes == 1) tc_mc_kernel<1><<<plan.n_cta, kTcThreads, kTcSmem, s>>>(jt, plan);
        else tc_mc_kernel<2><<<plan.n_cta, kTcThreads, kTcSmem, s>>>(jt, plan);
    } else {
        // Programmatic dependent launch: the grid is set up while the staging kernel runs
        // and its CTAs start on SMs as the staging blocks leave them; only the producer
        // thread, which reads the planes, waits for the staging grid to complete.
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(plan.n_cta));
        cfg.blockDim = dim3(kTcThreads);
        cfg.dynamicSmemBytes = size_t(kTcSmem);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = elem_bytes == 1 ? cudaLaunchKernelEx(&cfg, tc_kernel<1>, jt, plan)
                            : cudaLaunchKernelEx(&cfg, tc_kernel<2>, jt, plan);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace xe
