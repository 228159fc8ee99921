// xe_stage.cu -- operand staging for the tensor-core correlation kernel.
//
// Packed 4+4-bit samples [T][N] (Denman et al. 2020, section 2.2: 4-bit real and imaginary
// parts) become the correlation kernel's operand planes [kb][re|im][n_pad][64 B]: every
// sample component as an exact FP8 e4m3 (or f16) code, laid out in the exact shared-memory
// image the MMA reads (64-byte swizzle), so the correlation kernel fetches each plane tile
// with one bulk copy.  The masking variant applies per-(sample, input) validity flags and
// the offset-binary encoding, and writes the validity planes of count jobs.
//
// Kernels:
//   stage_kernel<2>       f16 operands, one block per (job, channel, k-block, 256 inputs).
//   stage_e4m3_kernel     e4m3 operands, persistent: a three-deep cp.async ring of input
//                         tiles, register-only conversion (4x4 byte transposes and byte-
//                         permute table lookups, xe_codes.cuh), full-sector plane stores.
#include <cstdint>
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
    if (jt.checks && __syncthreads_or(tid == 0 && *reinterpret_cast<volatile int *>(jt.status) != 0)) return;
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
    // With descriptor checks on, a failed check stops the staging before it reads a job.
    if (jt.checks && __syncthreads_or(tid == 0 && *reinterpret_cast<volatile int *>(jt.status) != 0)) return;

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


const void *stage_kernel_fn(int elem_bytes, bool masked) {
    if (elem_bytes == 1)
        return masked ? reinterpret_cast<const void *>(stage_e4m3_kernel<true>)
                      : reinterpret_cast<const void *>(stage_e4m3_kernel<false>);
    return reinterpret_cast<const void *>(stage_kernel<2>);
}

}  // namespace xe
