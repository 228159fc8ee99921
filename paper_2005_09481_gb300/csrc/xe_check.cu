// xe_check.cu -- device-side checks of a launch's descriptors (option "checks").
//
// The correlation's launches are driven by host-built descriptors: the job table (operand
// planes, shapes, views) and the plan (tiles of the triangle, their k-ranges and workspace
// slots).  With checks on, one small block reads them on the device before the staging and
// correlation kernels of the launch, holds every index and range against what was
// allocated, and on the first violation writes kStatusCheck + its number into the stream's
// status word instead of trapping; the staging and correlation kernels then return at once,
// and the host reports XE_ECHECK.  The checks only read the descriptors, never through an
// index that has not been checked first.
#include <cstdint>
#include <cuda_runtime.h>

#include "xe_internal.h"

namespace xe {

namespace {

__device__ __forceinline__ void check_fail(int *status, int id) { atomicCAS(status, 0, kStatusCheck + id); }

// Tiles of one channel of an N-input job (256-wide tiles, rows of 128): the same count the
// host and the implicit-plan decode use.
__device__ __forceinline__ int64_t tiles_of(int N) {
    int64_t n = 0;
    for (int r = 0; r * kBM < N; ++r) {
        const int half = r & 1;
        const int js = r * kBM + half * kBM;
        n += half + (js < N ? (N - js + kBN - 1) / kBN : 0);
    }
    return n;
}

}  // namespace

__global__ void __launch_bounds__(256) check_launch_kernel(const __grid_constant__ JobTable jt,
                                                           const __grid_constant__ PlanDev pd,
                                                           const CheckLimits lim) {
    int *status = pd.status;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (jt.n_jobs < 1 || jt.n_jobs > kMaxJobs) {
        if (tid == 0) check_fail(status, 0);
        return;
    }
    // 1-5: the jobs.
    for (int k = tid; k < jt.n_jobs; k += nt) {
        const JobDev &jb = jt.jobs[k];
        if (jb.N < 1 || jb.N > XE_MAX_N || jb.n_pad < jb.N || jb.n_pad % kNPad != 0 || jb.C < 1 ||
            jb.kblocks < 1) {
            check_fail(status, 1);
            continue;
        }
        if (jb.plane_chan_bytes != int64_t(jb.kblocks) * 2 * jb.n_pad * kRowBytes) check_fail(status, 2);
        const uint8_t *end = lim.planes + lim.planes_bytes;
        if (jb.planes < lim.planes || jb.planes + int64_t(jb.C) * jb.plane_chan_bytes > end) check_fail(status, 3);
        if (jb.count_planes) {
            const int64_t cchan = int64_t((jb.kblocks + 1) >> 1) * 2 * jb.n_pad * kRowBytes;
            if (jb.count_planes < lim.planes || jb.count_planes + int64_t(jb.C) * cchan > end) check_fail(status, 3);
        }
        if (!jb.vis || jb.vis_chan_elems < int64_t(jb.N) * (jb.N + 1) / 2) check_fail(status, 4);
        if (jb.stage_block0 < 0 || jb.stage_block0 > jt.total_stage_blocks ||
            (k > 0 && jb.stage_block0 < jt.jobs[k - 1].stage_block0))
            check_fail(status, 5);
    }
    if (pd.implicit) {
        // 6: implicit plans: every job's tiles, in order, and nothing beyond them.
        if (tid == 0) {
            int64_t t = 0;
            for (int k = 0; k < jt.n_jobs; ++k) {
                const JobDev &jb = jt.jobs[k];
                if (jb.tile0 != t || jb.tiles_per_chan != tiles_of(jb.N)) check_fail(status, 6);
                t += int64_t(jb.tiles_per_chan) * jb.C;
            }
            if (pd.n_tiles != t || pd.n_cta < 1) check_fail(status, 6);
        }
        return;
    }
    // 7-12: explicit plans.  Array lengths first, then the entries.
    if (pd.n_cta < 1 || pd.n_cta + 1 > lim.n_seg_off || pd.n_tiles < 1 || pd.n_tiles > lim.n_tiles ||
        int64_t(pd.n_tiles) > lim.n_counters) {
        if (tid == 0) check_fail(status, 7);
        return;
    }
    if (tid == 0 && (pd.seg_off[0] != 0 || pd.seg_off[pd.n_cta] != lim.n_segs)) check_fail(status, 8);
    for (int b = tid; b < pd.n_cta; b += nt)
        if (pd.seg_off[b] > pd.seg_off[b + 1] || pd.seg_off[b + 1] > lim.n_segs) check_fail(status, 8);
    for (int t = tid; t < pd.n_tiles; t += nt) {
        const Tile tl = pd.tiles[t];
        if (tl.job < 0 || tl.job >= jt.n_jobs) {
            check_fail(status, 9);
            continue;
        }
        const JobDev &jb = jt.jobs[tl.job];
        if (tl.chan < 0 || tl.chan >= jb.C || tl.i0 < 0 || tl.i0 % kBM != 0 || tl.i0 >= jb.n_pad ||
            (tl.nj != kBN && tl.nj != kBN / 2) || tl.j0 < tl.i0 || tl.j0 % (kBN / 2) != 0 ||
            tl.j0 + tl.nj > jb.n_pad || tl.kblocks != jb.kblocks)
            check_fail(status, 10);
        if (tl.n_parts < 0 || tl.part_off < 0 || tl.part_off + tl.n_parts > lim.n_tile_slots) check_fail(status, 11);
        for (int u = 0; tl.n_parts > 0 && tl.part_off >= 0 && tl.part_off + tl.n_parts <= lim.n_tile_slots && u < tl.n_parts; ++u) {
            const int slot = pd.tile_slots[tl.part_off + u];
            if (slot < 0 || slot >= lim.ws_slots) check_fail(status, 11);
        }
    }
    for (int q = tid; q < lim.n_segs; q += nt) {
        const Seg sg = pd.segs[q];
        if (sg.tile < 0 || sg.tile >= pd.n_tiles) {
            check_fail(status, 12);
            continue;
        }
        const Tile tl = pd.tiles[sg.tile];
        if (sg.k_lo < 0 || sg.k_lo >= sg.k_hi || sg.k_hi > tl.kblocks || sg.slot < -1 || sg.slot >= lim.ws_slots)
            check_fail(status, 12);
    }
}

cudaError_t launch_check(const JobTable &jt, const PlanDev &pd, const CheckLimits &lim, cudaStream_t s) {
    check_launch_kernel<<<1, 256, 0, s>>>(jt, pd, lim);
    return cudaGetLastError();
}

const void *check_kernel_fn() { return reinterpret_cast<const void *>(check_launch_kernel); }

}  // namespace xe
