// xe_tc.cu -- the tensor-core X-engine's correlation kernel.
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
// The operand planes come from the staging kernels (xe_stage.cu).
//
// Kernel:
//   tc_kernel     persistent, at most one CTA per SM; each CTA follows its list of
//                 segments (a k-range of one triangle tile of one job) from the host plan:
//                 warp 4 streams planes into a 4-stage shared-memory ring with bulk copies,
//                 warp 5 issues tcgen05.mma (M=128, N=256/128, K=32 bytes) into two f32
//                 accumulators in tensor memory (Re: columns 0-255, Im: 256-511),
//                 warps 0-3 drain them (tcgen05.ld), convert to int32 and store the packed
//                 upper triangle.  A tile split into several segments is summed exactly
//                 through a workspace by the last segment to finish (arrival counter, no
//                 spinning on other CTAs), or, for two parts, by a symmetric exchange of
//                 column halves.  When a CTA's only segment is one part of such a pair,
//                 all eight warps (the producer, the MMA warp and warps 6-7 join after the
//                 mainloop) run its epilogue, two warps per tensor-memory lane quarter.  The
//                 launch may overlap the staging kernel (programmatic dependent launch):
//                 only the producer waits for it before reading planes.
#include <cstdint>
#include <cuda_runtime.h>

#include "xe_internal.h"
#include "xe_ptx.cuh"

namespace xe {

// ---- persistent tensor-core correlation kernel -----------------------------------------------

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ __forceinline__ void set_status(int *status, int code) { atomicCAS(status, 0, code); }

// Implicit plans: tile t of the launch as a whole-tile segment.  The tiles of a job are its
// channels' tiles in channel order, each channel's in the order the host planner enumerates
// 256-wide tiles: row blocks of 128 inputs, in each first a 128-wide half tile where the row
// block starts mid-way through a 256 column block, then the 256-wide tiles to its right.
__device__ __forceinline__ void implicit_tile(const JobTable &jt, int t, Seg &sg, Tile &tl) {
    int lo = 0, hi = jt.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jt.jobs[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    const JobDev &jb = jt.jobs[lo];
    const int u = t - jb.tile0;
    const int c = u / jb.tiles_per_chan;
    int v = u - c * jb.tiles_per_chan;
    int i0 = 0, j0 = 0, nj = kBN;
    for (int r = 0; r * kBM < jb.N; ++r) {
        const int half = r & 1;
        const int js = r * kBM + half * kBM;
        const int n = half + (js < jb.N ? (jb.N - js + kBN - 1) / kBN : 0);
        if (v < n) {
            i0 = r * kBM;
            if (half && v == 0) {
                j0 = i0;
                nj = kBM;
            } else {
                j0 = js + (v - half) * kBN;
            }
            break;
        }
        v -= n;
    }
    tl = Tile{lo, c, i0, j0, nj, jb.kblocks, 0, 0};
    sg = Seg{t, 0, jb.kblocks, -1};
}

// Segment q of this CTA (q in [q0, q1)) and its tile, from the plan arrays or implicitly.
__device__ __forceinline__ void fetch_segment(const JobTable &jt, const PlanDev &plan, int q, Seg &sg, Tile &tl) {
    if (plan.implicit) {
        implicit_tile(jt, int(blockIdx.x) + q * int(gridDim.x), sg, tl);
    } else {
        sg = plan.segs[q];
        tl = plan.tiles[sg.tile];
    }
}

// *p += v in L2 (a reduction: nothing is returned, so the thread does not wait).
__device__ __forceinline__ void red_add_s32(int32_t *p, int32_t v) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Store (or add) a 32 x 32 block of final visibilities held by one warp (lane = row
// i0 + lane, register k = column jbase + k).  The block is transposed through the warp's
// shared buffer so that each global access covers 32 consecutive baselines of one row
// (256 contiguous bytes); in accumulate mode the block is added by reductions in L2.
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
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const int i = i0 + r;
            if (i < jb.N && j >= i && j < jb.N) {
                const int64_t k = int64_t(i) * N - (int64_t(i) * (i - 1)) / 2 + (j - i);
                if (acc) red_add_s32(vis + k, stage[r * 33 + lane].x);
                else vis[k] = stage[r * 33 + lane].x;
            }
        }
    } else if (acc) {
        // Adding into the sums: reductions performed in L2, so no warp waits for the old
        // values (a load, add and store per element held each tile's epilogue, and with it
        // the next tile's MMAs, on the loads' latency).  Integer addition is exact whatever
        // the order.
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const int i = i0 + r;
            if (i < jb.N && j >= i && j < jb.N) {
                const int64_t k = int64_t(i) * N - (int64_t(i) * (i - 1)) / 2 + (j - i);
                const int2 v = stage[r * 33 + lane];
                red_add_s32(vis + 2 * k, v.x);
                red_add_s32(vis + 2 * k + 1, v.y);
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

template <int EB>
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
    // With descriptor checks on, a failed check (or an earlier timeout not yet reported)
    // stops the launch before it reads a descriptor; the whole CTA decides together.
    if (jt.checks && __syncthreads_or(threadIdx.x == 0 && *status != 0)) return;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
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
    const uint32_t tmem = *tmem_slot;

    // This CTA's work: segments [q0, q1) of the plan, each a k-range of one tile.
    const int q0 = plan.implicit ? 0 : plan.seg_off[blockIdx.x];
    const int q1 = plan.implicit ? (plan.n_tiles - int(blockIdx.x) + int(gridDim.x) - 1) / int(gridDim.x)
                                 : plan.seg_off[blockIdx.x + 1];
    // A CTA whose only segment is one part of an exchanged tile (plans whose split tiles
    // all have 2, 4 or 8 parts, one segment per CTA, all CTAs resident) finishes it with
    // eight warps: the producer and MMA warps are idle by then, and two more warps wait.
    const bool wide = !plan.implicit && plan.pair_exchange && q1 - q0 == 1 && plan.segs[q0].slot >= 0;
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
            for (int q = plan.inject_stall ? q1 : q0; ok && q < q1; ++q) {
                Seg sg;
                Tile tl;
                fetch_segment(jt, plan, q, sg, tl);
                const JobDev &jb = jt.jobs[tl.job];
                const uint8_t *pl = jb.planes + int64_t(tl.chan) * jb.plane_chan_bytes;
                const uint32_t bbytes = uint32_t(tl.nj) * kRowBytes;
                for (int64_t k = sg.k_lo; k < sg.k_hi; ++k) {
                    if (!mbar_wait(&empty[stage], ph ^ 1u, status)) {
                        set_status(plan.status, kStatusTimeoutProducer);
                        ok = false;
                        break;
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
                        bulk_prefetch_l2(fre + int64_t(tl.j0) * kRowBytes, bbytes);
                        bulk_prefetch_l2(fim + int64_t(tl.j0) * kRowBytes, bbytes);
                    }
                    bulk_g2s(st, pre + int64_t(tl.i0) * kRowBytes, kAPlane, &full[stage]);
                    bulk_g2s(st + kAPlane, pim + int64_t(tl.i0) * kRowBytes, kAPlane, &full[stage]);
                    bulk_g2s(st + 2 * kAPlane, pre + int64_t(tl.j0) * kRowBytes, bbytes, &full[stage]);
                    bulk_g2s(st + 2 * kAPlane + kBPlane, pim + int64_t(tl.j0) * kRowBytes, bbytes, &full[stage]);
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
                Seg sg;
                Tile tl;
                fetch_segment(jt, plan, q, sg, tl);
                // Count job: its two slots hold the validity of two consecutive sample
                // blocks, and only the Re accumulator is formed.
                const bool re_only = (jt.jobs[tl.job].mode & kModeCount) != 0;
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
                        mma_commit(&empty[stage]);
                        if (++stage == kStages) { stage = 0; ph ^= 1u; }
                    }
                };
                if (re_only) mainloop(std::true_type{});
                else mainloop(std::false_type{});
                if (ok) mma_commit(acc_full);
            }
            // Every MMA of this CTA is issued: a launch that depends on this grid
            // programmatically (the count launch after the visibilities') may set up its CTAs
            // on SMs that are free; its producer still waits for this grid to complete.
            asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
            if (!ok) {
                // Wait (bounded) for every MMA already issued before TMEM is released.
                mma_commit(drain);
                const long long t0 = clock64();
                while (!mbar_try_wait(drain, 0) && clock64() - t0 < kWaitBudgetCycles) {}
            }
        }
    } else if (warp < 4 && !wide) {
        // ---------------- epilogue: TMEM -> int32 -> packed triangle ----------------
        uint32_t acc_ph = 0;
        const int r = warp * 32 + lane;
        const uint32_t lane_base = uint32_t(warp * 32) << 16;
        for (int q = q0; q < q1; ++q) {
            Seg sg;
            Tile tl;
            fetch_segment(jt, plan, q, sg, tl);
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
            // Part u of the tile's s parts (s = 2, 4 or 8; the host keeps nj / s >= 32)
            // finalises the column slice [u nj / s, (u + 1) nj / s): it publishes every other
            // column of its sums at that column of its workspace slot, waits (bounded) for all
            // parts to have published, and adds the other parts' values of its slice.
            const int s = tl.n_parts;
            int part = 0;
            for (int u = 0; u < s; ++u)
                if (plan.tile_slots[tl.part_off + u] == sg.slot) part = u;
            const int wd = tl.nj / s;
            const int mine0 = part * wd;
            int32_t *ws = plan.ws + int64_t(sg.slot) * kWsSlotElems;
            for (int cc = 32 * share; cc < tl.nj; cc += 64) {
                if (cc >= mine0 && cc < mine0 + wd) continue;
                uint32_t fre[32], fim[32];
                tmem_ld_32x32b_x32(tmem + lane_base + cc, fre);
                tmem_ld_32x32b_x32(tmem + lane_base + 256 + cc, fim);
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
                while (*cnt < s) {
                    if (*status != 0 || clock64() - t0 > kWaitBudgetCycles) { ok = false; break; }
                }
                if (!ok) set_status(plan.status, kStatusTimeoutEpilogue);
                *epi_flag = ok ? 1 : 0;
            }
            wbar();
            if (*epi_flag == 1) {
                __threadfence();
                // My slice in shares of 32-column chunks: half each for slices of 64 columns
                // or more, else all of it to share 0.
                const int per = wd >= 64 ? wd / 2 : (share == 0 ? wd : 0);
                const int c_lo = mine0 + (wd >= 64 ? share * per : 0), c_hi = c_lo + per;
                // With two parts, the partner's values of my slice (re and im, wd x 128 int32
                // each) go into the idle operand stages in one pair of bulk copies; warps 4..7
                // take their transpose buffers from the stages after it.  With more parts the
                // chunks read the partners' slots from L2.
                const uint32_t bytes = uint32_t(wd) * kBM * 4u;
                const int32_t *w1 = plan.ws + int64_t(plan.tile_slots[tl.part_off + (1 - part)]) * kWsSlotElems;
                if (s == 2) {
                    if (threadIdx.x == 0) {
                        asm volatile("fence.proxy.async.global;" ::: "memory");
                        mbar_arrive_expect_tx(xfer, 2u * bytes);
                        bulk_g2s(smem, w1 + int64_t(mine0) * kBM, bytes, xfer);
                        bulk_g2s(smem + bytes, w1 + int64_t(kBN + mine0) * kBM, bytes, xfer);
                    }
                    const long long t0 = clock64();
                    bool got = false;
                    while (!(got = mbar_try_wait(xfer, 0)) && clock64() - t0 < kWaitBudgetCycles) {}
                    if (!got) set_status(plan.status, kStatusTimeoutEpilogue);
                }
                const int32_t *sh = reinterpret_cast<const int32_t *>(smem);
                // (After the largest two-part copy, re and im of 128 columns: 128 KB, so the
                // buffers end at 162 KB, inside the 192 KB of operand stages.)
                constexpr size_t kXferBytes = 2 * size_t(kBN / 2) * kBM * 4;
                static_assert(kXferBytes + 4 * 32 * 33 * sizeof(int2) <= size_t(kStages) * kStageBytes,
                              "transpose buffers of warps 4..7 must fit in the operand stages");
                int2 *buf = share == 0 ? epi_stage
                                       : reinterpret_cast<int2 *>(smem + kXferBytes) + (warp - 4) * 32 * 33;
                for (int cc = c_lo; cc < c_hi; cc += 32) {
                    uint32_t fre[32], fim[32];
                    tmem_ld_32x32b_x32(tmem + lane_base + cc, fre);
                    tmem_ld_32x32b_x32(tmem + lane_base + 256 + cc, fim);
                    int re[32], im[32];
                    if (s == 2) {
#pragma unroll
                        for (int k = 0; k < 32; ++k) {
                            re[k] = sh[(cc - mine0 + k) * kBM + r];
                            im[k] = sh[(wd + cc - mine0 + k) * kBM + r];
                        }
                    } else {
                        // The other parts' values of these 32 columns, from L2: three parts
                        // at a time, four columns at a time, all of those loads independent
                        // and in flight together (a loop over the parts that waited for each
                        // part's loads in turn took 16-33 us per slice).  The empty asm keeps
                        // the compiler from hoisting later loads above it, which bounds the
                        // registers held.
#pragma unroll
                        for (int k = 0; k < 32; ++k) re[k] = im[k] = 0;
                        for (int g0 = 0; g0 < s - 1; g0 += 3) {
                            int64_t base[3];
#pragma unroll
                            for (int v = 0; v < 3; ++v) {
                                const int pv = g0 + v, u = pv < part ? pv : pv + 1;
                                base[v] = pv < s - 1 ? int64_t(plan.tile_slots[tl.part_off + u]) * kWsSlotElems +
                                                           int64_t(cc) * kBM + r
                                                     : -1;
                            }
#pragma unroll
                            for (int k0 = 0; k0 < 32; k0 += 4) {
#pragma unroll
                                for (int k = k0; k < k0 + 4; ++k)
#pragma unroll
                                    for (int v = 0; v < 3; ++v)
                                        if (base[v] >= 0) {
                                            re[k] += __ldcg(plan.ws + base[v] + k * kBM);
                                            im[k] += __ldcg(plan.ws + base[v] + (kBN + k) * kBM);
                                        }
                                asm volatile("" ::: "memory");
                            }
                        }
                    }
                    tmem_ld_wait();
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        re[k] += __float2int_rn(__uint_as_float(fre[k]));
                        im[k] += __float2int_rn(__uint_as_float(fim[k]));
                    }
                    store_block(jb, tl.chan, tl.i0 + quarter * 32, tl.j0 + cc, re, im,
                                jt.accumulate | jb.accumulate, buf);
                }
                wbar();
                // Every part has read the others' values: the last to finish resets the
                // counter for the next launch.
                if (threadIdx.x == 0 && atomicAdd(&plan.counters[sg.tile], 1) == 2 * s - 1) plan.counters[sg.tile] = 0;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

template <int EB>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_kernel(const __grid_constant__ JobTable jt, const __grid_constant__ PlanDev plan) {
    tc_body<EB>(jt, plan);
}

int tc_smem_bytes() { return kTcSmem; }


const void *tc_kernel_fn(int elem_bytes) {
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
    if (dev >= 0 && dev < 64) done_dev[dev] = 1;
    return cudaSuccess;
}

cudaError_t launch_tc(const JobTable &jt, const PlanDev &plan, int elem_bytes, cudaStream_t s) {
    if (plan.n_cta <= 0 || plan.n_tiles <= 0) return cudaSuccess;
    cudaError_t e = tc_prepare();
    if (e != cudaSuccess) return e;
    // Programmatic dependent launch: the grid is set up while the staging kernel runs and its
    // CTAs start on SMs as the staging blocks leave them; only the producer thread, which
    // reads the planes, waits for the staging grid to complete.
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
    return cudaGetLastError();
}

}  // namespace xe
