// xe_api.cu -- host runtime behind the C ABI of include/xe.h: argument checks, the
// triangle-tile plans and their schedules (segment lists per persistent CTA), the
// autotuner that picks tile width and schedule per batch shape, per-stream scratch memory,
// the exact-window split of long integrations, CUDA-graph replay of batches, and timing.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <time.h>

#include <cuda_runtime.h>

#include "xe.h"
#include "xe_host.h"
#include "xe_internal.h"

namespace xe {

// ---- errors --------------------------------------------------------------------------

static thread_local char g_err[512] = "";

static int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int record_error(int code, const char *msg) { return fail(code, "%s", msg); }

// The error a nonzero device status word stands for.
static int status_error(int st) {
    if (st >= kStatusCheck && st < kStatusCheck + 16)
        return fail(XE_ECHECK, "device-side check %d of a launch's descriptors failed", st - kStatusCheck);
    return fail(XE_ETIMEOUT, "device wait timed out (status %d)", st);
}

#define XE_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(XE_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
    } while (0)

// ---- options -------------------------------------------------------------------------

struct Options {
    int operand_bytes = 1;                 // 1: e4m3 operands, 2: f16 operands
    int64_t exact_chunk_t = kExactChunkT;  // samples per f32 accumulation window
    int n_cta = 0;                         // 0: one CTA per SM
    int sched = -1;                        // -1: heuristic / autotuned; else a Sched
    int tile_n = 0;                        // 0: heuristic / autotuned; else 128 or 256
    int autotune = 0;                      // 1: time candidate plans on first sight of a shape
    int timing = 0;
    int inject_stall = 0;                  // test hook for the bounded-wait path (next call only)
    int64_t host_chunk_t = 8192;           // samples per pipelined chunk of xe_correlate_host
                                           // (0: one copy, then one correlation)
    int64_t host_async_chunk_t = 0;        // the same for xe_correlate_host_async, whose
                                           // calls overlap each other already
    int count_weight = 75;                 // cost of a count-job k-iteration, % of a data one
    int checks = 0;                        // 1: a device-side check of every correlation launch's
                                           // descriptors runs before it (XE_ECHECK on failure)
    int check_corrupt = 0;                 // test hook (checks on only): 1 = the plan claims no
                                           // tiles, 2 = job 0's plane stride is off by 64 bytes
    int count_launch = 1;                  // 1: count jobs in a launch of their own after the
                                           // data jobs' (masked calls with counts; measured
                                           // faster than one mixed launch); 0: one launch
    int part_overhead = 2;                 // modelled cost of one extra tile part, % of a
                                           // whole data tile (workspace fix-up)
    int implicit_plans = 1;                // 1: batches of the streaming server run without
                                           // host-built plans (whole tiles dealt round-robin,
                                           // decoded in the kernel); 0: host plans
};
static Options g_opt;

// XE_CHECKS=1 in the environment turns the descriptor checks on when the library loads.
static const bool g_env_checks = [] {
    const char *p = getenv("XE_CHECKS");
    if (p && *p && strcmp(p, "0") != 0) g_opt.checks = 1;
    return g_opt.checks != 0;
}();
static std::mutex g_mu;

// Host-side events of the runtime that can stall a caller (process-wide, under g_mu):
// plans built (and their host time), scratch regrowths and plan-cache trims (both
// synchronise the device), and launch records built (and their host time).
struct RuntimeCounters {
    int64_t plans_built = 0, plan_ns = 0, regrowths = 0, trims = 0, batches = 0, build_ns = 0;
};
static RuntimeCounters g_rc;

static int64_t host_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return int64_t(ts.tv_sec) * 1000000000LL + ts.tv_nsec;
}

// ---- plans ---------------------------------------------------------------------------

struct JobShape {
    int N;
    int64_t T;
    int C;
    int weight = 100;         // cost of one k-iteration of its tiles, percent of a data tile's
};

struct TuneCfg {
    int n_cta;
    int tile_n;
    int sched;
};

struct HostPlan {
    bool pair_exchange = false;   // every split tile has 2, 4 or 8 parts and every CTA 1 segment
    std::vector<Tile> tiles;
    std::vector<Seg> segs;
    std::vector<int> seg_off;     // n_cta + 1 entries
    std::vector<int> tile_slots;
    int n_cta = 0;
    int n_partial = 0;
    int64_t total_iters = 0;
};

static int n_pad_of(int N) { return (N + kNPad - 1) / kNPad * kNPad; }

static int64_t kblocks_of(int64_t T, int eb) {
    const int ks = samples_per_stage(eb);
    return (T + ks - 1) / ks;
}

// Triangle tiles of every job and channel: row blocks of 128 inputs; column tiles of width
// tile_n aligned to tile_n, plus a 128-wide half tile where a row block starts mid-way
// through a 256-aligned column block.  Together they cover every (i, j >= i) exactly once.
static void enumerate_tiles(const std::vector<JobShape> &jobs, int eb, int tile_n,
                            std::vector<Tile> &tiles) {
    tiles.clear();
    for (int q = 0; q < int(jobs.size()); ++q) {
        const JobShape &js = jobs[q];
        const int kb = int(kblocks_of(js.T, eb));
        for (int c = 0; c < js.C; ++c)
            for (int i0 = 0; i0 < js.N; i0 += kBM) {
                int j0 = i0;
                if (j0 % tile_n != 0) {
                    tiles.push_back(Tile{q, c, i0, j0, kBM, kb, 0, 0});
                    j0 += kBM;
                }
                for (; j0 < js.N; j0 += tile_n) tiles.push_back(Tile{q, c, i0, j0, tile_n, kb, 0, 0});
            }
    }
}

// The number of tiles enumerate_tiles makes for one channel of N inputs.
static int64_t count_tiles(int N, int tile_n) {
    int64_t n = 0;
    for (int i0 = 0; i0 < N; i0 += kBM) {
        int j0 = i0;
        if (j0 % tile_n != 0) {
            ++n;
            j0 += kBM;
        }
        if (j0 < N) n += (N - j0 + tile_n - 1) / tile_n;
    }
    return n;
}

// Equal contiguous ranges of the concatenated k-iterations of tiles [t_lo, t_hi), dealt to
// CTAs 0..G-1 (appended to their lists).
static void stream_k(const std::vector<Tile> &tiles, int t_lo, int t_hi, int G,
                     std::vector<std::vector<Seg>> &per) {
    int64_t W = 0;
    for (int t = t_lo; t < t_hi; ++t) W += tiles[size_t(t)].kblocks;
    if (W == 0) return;
    const int64_t g = std::min<int64_t>(G, W);
    int t = t_lo;
    int64_t tb = 0;   // first iteration of tile t in the concatenation
    for (int64_t b = 0; b < g; ++b) {
        const int64_t r0 = b * W / g, r1 = (b + 1) * W / g;
        while (t < t_hi && tb + tiles[size_t(t)].kblocks <= r0) { tb += tiles[size_t(t)].kblocks; ++t; }
        int tt = t;
        int64_t ttb = tb;
        while (tt < t_hi && ttb < r1) {
            const int64_t lo = std::max(r0, ttb) - ttb;
            const int64_t hi = std::min(r1, ttb + tiles[size_t(tt)].kblocks) - ttb;
            if (hi > lo) per[size_t(b)].push_back(Seg{tt, int(lo), int(hi), -1});
            ttb += tiles[size_t(tt)].kblocks;
            ++tt;
        }
    }
}

// The least-loaded CTA (the lowest index among equal loads) as a tournament tree over the
// CTAs: top() is the CTA a greedy schedule deals the next part to, add() charges it the part.
// The same choice as popping the smallest (load, CTA) pair from a heap, at a fixed cost of
// log2(G) comparisons per part.
template <typename L>
struct LeastLoaded {
    int G, n_leaf = 1;
    std::vector<L> load;
    std::vector<int> win;     // node i: the winning CTA of its subtree (leaves n_leaf + b; -1: none)
    explicit LeastLoaded(int g) : G(g), load(static_cast<size_t>(g), L(0)) {
        while (n_leaf < G) n_leaf <<= 1;
        win.assign(static_cast<size_t>(2 * n_leaf), -1);
        for (int b = 0; b < G; ++b) win[size_t(n_leaf + b)] = b;
        for (int i = n_leaf - 1; i >= 1; --i) win[size_t(i)] = better(win[size_t(2 * i)], win[size_t(2 * i + 1)]);
    }
    int better(int a, int b) const {
        if (a < 0) return b;
        if (b < 0) return a;
        const L la = load[size_t(a)], lb = load[size_t(b)];
        return (lb < la || (lb == la && b < a)) ? b : a;
    }
    int top() const { return win[1]; }
    void add(int b, L d) {
        load[size_t(b)] += d;
        for (int i = (n_leaf + b) >> 1; i >= 1; i >>= 1)
            win[size_t(i)] = better(win[size_t(2 * i)], win[size_t(2 * i + 1)]);
    }
};

// Weighted schedule: every tile is cut into the same number s of equal k-parts, and the
// parts are dealt in k-phase order (all first parts, then all second parts, ...; heavier
// jobs first within a phase) each to the CTA with the least weighted load so far, so that
// CTAs still read nearby k-blocks at the same time (shared in L2) while light count-job
// parts fill the gaps left by data-job parts.  A part costs kblocks/s * weight, plus a
// modelled fix-up cost when s > 1; the s in [1, 4] with the smallest modelled makespan wins.
// Fix-up cost of splitting a tile, in k-blocks of mainloop time (split, hybrid and weighted schedules).
constexpr double kPairFixKb = 8.0;     // two parts: the symmetric column-half exchange
constexpr double kPartFixKb = 20.0;    // each further part: summed by the last arriving part
constexpr double kExch4FixKb = 30.0;   // four parts exchanging column slices
constexpr double kExch8FixKb = 56.0;   // eight parts exchanging column slices

static void schedule_weighted(const HostPlan &p, int G, const std::vector<int> &weight,
                              std::vector<std::vector<Seg>> &per) {
    const int n = int(p.tiles.size());
    int min_kb = 1 << 30, max_kb = 0;
    for (const Tile &t : p.tiles) {
        min_kb = std::min(min_kb, t.kblocks);
        max_kb = std::max(max_kb, t.kblocks);
    }
    std::vector<int> order(static_cast<size_t>(n));
    for (int t = 0; t < n; ++t) order[size_t(t)] = t;
    auto heavier = [&](int a, int b) {
        return weight[size_t(p.tiles[size_t(a)].job)] > weight[size_t(p.tiles[size_t(b)].job)];
    };
    if (!std::is_sorted(order.begin(), order.end(), heavier)) std::stable_sort(order.begin(), order.end(), heavier);
    auto deal = [&](int s, std::vector<std::vector<Seg>> *out) {
        LeastLoaded<double> ll(G);
        // Fix-up cost charged to every part of a split tile: the option's share of the longest
        // tile, but never less than the measured absolute cost (short tiles).
        const double over = s > 1 ? std::max(g_opt.part_overhead / 100.0 * max_kb,
                                             s == 2 ? kPairFixKb : kPartFixKb * (s - 1))
                                  : 0.0;
        double makespan = 0;
        for (int k = 0; k < s; ++k)
            for (int t : order) {
                const Tile &tl = p.tiles[size_t(t)];
                const int lo = int(int64_t(k) * tl.kblocks / s), hi = int(int64_t(k + 1) * tl.kblocks / s);
                if (hi <= lo) continue;
                const int b = ll.top();
                ll.add(b, double(hi - lo) * weight[size_t(tl.job)] / 100.0 + over);
                makespan = std::max(makespan, ll.load[size_t(b)]);
                if (out) (*out)[size_t(b)].push_back(Seg{t, lo, hi, -1});
            }
        return makespan;
    };
    int best_s = 1;
    double best = 1e300;
    for (int s = 1; s <= std::min(4, std::max(1, min_kb)); ++s) {
        const double m = deal(s, nullptr);
        if (m < best * (1 - 1e-9)) {
            best = m;
            best_s = s;
        }
    }
    deal(best_s, &per);
}

// Parts per tile for tiles [t0, t1) dealt over G CTAs: up to the CTAs per tile (and the
// k-blocks of the shortest tile), chosen to minimise max k-blocks per part + fix-up.  With
// `exchange` (each part alone on its CTA), 2, 4 or 8 parts whose slices are at least 32
// columns wide exchange slices; otherwise the last arriving part sums them.
static int split_parts(const std::vector<Tile> &tiles, int t0, int t1, int G, bool exchange) {
    const int n = t1 - t0;
    int min_kb = 1 << 30, max_kb = 0, min_nj = kBN;
    for (int t = t0; t < t1; ++t) {
        min_kb = std::min(min_kb, tiles[size_t(t)].kblocks);
        max_kb = std::max(max_kb, tiles[size_t(t)].kblocks);
        min_nj = std::min(min_nj, tiles[size_t(t)].nj);
    }
    const int s_max = std::min(n < G ? std::max(1, G / n) : 1, std::max(1, min_kb));
    int s = 1;
    double best = double(max_kb);
    for (int c = 2; c <= s_max; ++c) {
        double fix = kPartFixKb * (c - 1);
        if (exchange && min_nj / c >= 32 && (c == 2 || c == 4 || c == 8))
            fix = c == 2 ? kPairFixKb : c == 4 ? kExch4FixKb : kExch8FixKb;
        const double cost = double(max_kb) / c + fix;
        if (cost < best) {
            best = cost;
            s = c;
        }
    }
    return s;
}

static void schedule(HostPlan &p, int G, int sched, const std::vector<int> &weight) {
    const int n = int(p.tiles.size());
    std::vector<std::vector<Seg>> per(static_cast<size_t>(G));
    if (sched == kSchedWeighted) {
        schedule_weighted(p, G, weight, per);
    } else if (sched == kSchedSplit) {
        // Parts per tile: up to the CTAs per tile, chosen by a cost model in k-blocks.  A
        // split shortens the mainloop but each part past the first costs a fix-up: two parts
        // swap column halves through the workspace (about kPairFixKb k-blocks of time), more
        // parts are summed by the last arriving part (about kPartFixKb each; measured on the
        // GB300, where 64 parts of a 64-k-block tile took ten times as long as two).
        const int s = split_parts(p.tiles, 0, n, G, true);
        int64_t item = 0;
        const int64_t n_items = int64_t(n) * s;
        const int64_t g = std::min<int64_t>(G, n_items);
        for (int t = 0; t < n; ++t)
            for (int k = 0; k < s; ++k, ++item) {
                const int kb = p.tiles[size_t(t)].kblocks;
                const int lo = int(int64_t(k) * kb / s), hi = int(int64_t(k + 1) * kb / s);
                if (hi > lo) per[size_t(item % g)].push_back(Seg{t, lo, hi, -1});
            }
    } else if (sched == kSchedHybrid) {
        // Whole tiles in full waves; the last partial wave's tiles split by the same cost
        // model as the split schedule over the CTAs it leaves (whole when it leaves fewer
        // than two per tile).  An equal stream-K share of that wave over every CTA cut small
        // tails into many parts, and their fix-up outweighed the balance.
        const int full = (n / G) * G;
        for (int t = 0; t < full; ++t)
            per[size_t(t % G)].push_back(Seg{t, 0, p.tiles[size_t(t)].kblocks, -1});
        const int m = n - full;
        if (m > 0) {
            const int s = split_parts(p.tiles, full, n, G, false);
            int64_t item = 0;
            for (int t = full; t < n; ++t)
                for (int k = 0; k < s; ++k, ++item) {
                    const int kb = p.tiles[size_t(t)].kblocks;
                    const int lo = int(int64_t(k) * kb / s), hi = int(int64_t(k + 1) * kb / s);
                    if (hi > lo) per[size_t(item % G)].push_back(Seg{t, lo, hi, -1});
                }
        }
    } else if (sched == kSchedLPT) {
        // Longest tile first to the least-loaded CTA; every CTA then walks its tiles in tile
        // order.  (Batches whose jobs arrive longest first are already in order.)
        std::vector<int> order(static_cast<size_t>(n));
        for (int t = 0; t < n; ++t) order[size_t(t)] = t;
        auto longer = [&](int a, int b) { return p.tiles[size_t(a)].kblocks > p.tiles[size_t(b)].kblocks; };
        if (!std::is_sorted(order.begin(), order.end(), longer)) std::stable_sort(order.begin(), order.end(), longer);
        LeastLoaded<int64_t> ll(G);
        std::vector<int> cta_of(static_cast<size_t>(n)), count(static_cast<size_t>(G), 0);
        for (int t : order) {
            const int b = ll.top();
            cta_of[size_t(t)] = b;
            ++count[size_t(b)];
            ll.add(b, p.tiles[size_t(t)].kblocks);
        }
        for (int b = 0; b < G; ++b) per[size_t(b)].reserve(size_t(count[size_t(b)]));
        for (int t = 0; t < n; ++t)
            per[size_t(cta_of[size_t(t)])].push_back(Seg{t, 0, p.tiles[size_t(t)].kblocks, -1});
    } else {
        stream_k(p.tiles, 0, n, G, per);
    }
    // Drop trailing CTAs without work; build the CSR lists.
    int used = G;
    while (used > 1 && per[size_t(used - 1)].empty()) --used;
    p.n_cta = used;
    p.segs.clear();
    p.seg_off.assign(size_t(used) + 1, 0);
    for (int b = 0; b < used; ++b) {
        p.seg_off[size_t(b)] = int(p.segs.size());
        for (const Seg &s : per[size_t(b)]) p.segs.push_back(s);
    }
    p.seg_off[size_t(used)] = int(p.segs.size());
}

// Mark partial segments, give each a workspace slot, and list the slots of every tile.
// Returns false if the segments do not partition every tile's k-range exactly.
static bool finalize_parts(HostPlan &p) {
    const int n = int(p.tiles.size());
    const int ns = int(p.segs.size());
    // The segments of every tile, in segment order (a counting sort by tile), then each
    // tile's list by k_lo.
    std::vector<int> first(static_cast<size_t>(n) + 1, 0), qs(static_cast<size_t>(ns));
    for (const Seg &s : p.segs)
        if (s.tile >= 0) ++first[size_t(s.tile) + 1];
    for (int t = 0; t < n; ++t) first[size_t(t) + 1] += first[size_t(t)];
    {
        std::vector<int> fill(first.begin(), first.end() - 1);
        for (int q = 0; q < ns; ++q)
            if (p.segs[size_t(q)].tile >= 0) qs[size_t(fill[size_t(p.segs[size_t(q)].tile)]++)] = q;
    }
    p.tile_slots.clear();
    p.n_partial = 0;
    p.total_iters = 0;
    for (int t = 0; t < n; ++t) {
        Tile &tl = p.tiles[size_t(t)];
        int *q0 = qs.data() + first[size_t(t)], *q1 = qs.data() + first[size_t(t) + 1];
        if (q1 - q0 > 1)
            std::sort(q0, q1, [&](int a, int b) { return p.segs[size_t(a)].k_lo < p.segs[size_t(b)].k_lo; });
        int k = 0;
        for (const int *q = q0; q != q1; ++q) {
            if (p.segs[size_t(*q)].k_lo != k) return false;
            k = p.segs[size_t(*q)].k_hi;
        }
        if (k != tl.kblocks) return false;
        p.total_iters += tl.kblocks;
        tl.n_parts = 0;
        tl.part_off = int(p.tile_slots.size());
        if (q1 - q0 > 1) {
            for (const int *q = q0; q != q1; ++q) {
                p.segs[size_t(*q)].slot = p.n_partial;
                p.tile_slots.push_back(p.n_partial);
                ++p.n_partial;
            }
            tl.n_parts = int(q1 - q0);
        }
    }
    return true;
}

// The default plan when nothing is tuned: 256-wide tiles; with fewer tiles than CTAs and
// equal tile lengths, split every tile into the same number of k-parts so that concurrently
// running CTAs read the same k-blocks (shared in L2); many equal tiles: whole tiles in full
// waves, the last wave stream-K; uneven tiles: whole tiles, longest first.
static TuneCfg heuristic(const std::vector<JobShape> &jobs, int eb, int n_sm) {
    // 128-wide tiles when every job fits one 128-input row block (one 128 x 128 tile instead
    // of a 128 x 256 one that is half padding) with at most 256 k-blocks, or has at most 256
    // inputs and at most 32 k-blocks (where the launch, fill and epilogue outweigh the MMAs):
    // measured on the GB300, N=64 T=1024 25 us against 33, N=128 T=8192 43 against 50,
    // N=256 T=1024 27 against 35, N=200 T=2048 35 against 37.  Longer integrations keep
    // 256-wide tiles: their k-blocks cost less per output element and they split into eight
    // exchanging parts (a 128-wide tile into at most four).
    bool small = true;
    for (const JobShape &j : jobs) {
        const int64_t kb = kblocks_of(j.T, eb);
        small = small && ((j.N <= kBM && kb <= 256) || (j.N <= kBN && kb <= 32));
    }
    TuneCfg c{g_opt.n_cta > 0 ? g_opt.n_cta : n_sm, g_opt.tile_n > 0 ? g_opt.tile_n : small ? kBN / 2 : kBN,
              g_opt.sched};
    if (c.sched < 0) {
        // Decided from the job shapes alone (every job has at least one tile, all of them
        // with the job's k-block count), without enumerating the tiles.
        bool weighted = false, uniform = true;
        int64_t n_tiles = 0;
        const int64_t kb0 = kblocks_of(jobs[0].T, eb);
        for (const JobShape &j : jobs) {
            weighted = weighted || j.weight != 100;
            uniform = uniform && kblocks_of(j.T, eb) == kb0;
            n_tiles += count_tiles(j.N, c.tile_n) * j.C;
        }
        // Fewer tiles than CTAs: split them (whole tiles longest first left most CTAs idle:
        // 2.2x slower on a 32768 + 4096 + 2048-sample batch); otherwise whole tiles, longest
        // first when the k-block counts differ.
        if (weighted) c.sched = kSchedWeighted;
        else if (n_tiles < c.n_cta) c.sched = kSchedSplit;
        else if (!uniform) c.sched = kSchedLPT;
        else c.sched = kSchedHybrid;
    }
    return c;
}

static bool build_plan(const std::vector<JobShape> &jobs, int eb, const TuneCfg &cfg, HostPlan &p) {
    enumerate_tiles(jobs, eb, cfg.tile_n, p.tiles);
    if (p.tiles.empty()) return false;
    const int G = std::max(1, cfg.n_cta);
    std::vector<int> weight;
    for (const JobShape &j : jobs) weight.push_back(std::max(1, j.weight));
    schedule(p, G, cfg.sched, weight);
    if (!finalize_parts(p)) return false;
    // The exchange of column slices waits for the other parts, so it is used only when each
    // part is the only work of its CTA (all of them resident at once) and every split tile
    // has 2, 4 or 8 parts of at least 32 columns.
    bool pe = true;
    for (const Tile &t : p.tiles)
        pe = pe && (t.n_parts == 0 || ((t.n_parts == 2 || t.n_parts == 4 || t.n_parts == 8) &&
                                       t.nj % t.n_parts == 0 && t.nj / t.n_parts >= 32));
    for (int b = 0; b < p.n_cta && pe; ++b) pe = p.seg_off[size_t(b) + 1] - p.seg_off[size_t(b)] == 1;
    p.pair_exchange = pe;
    return true;
}

struct DevPlan {
    HostPlan host;
    void *blob = nullptr;         // tiles | segs | seg_off | tile_slots
    bool own_blob = false;        // blob was allocated alone (the arena was full), not carved
    cudaEvent_t ready = nullptr;  // the upload has landed (recorded on upload_stream)
    cudaStream_t upload_stream = nullptr;
    const Tile *d_tiles = nullptr;
    const Seg *d_segs = nullptr;
    const int *d_seg_off = nullptr;
    const int *d_tile_slots = nullptr;
};

struct Scratch {
    uint8_t *planes = nullptr;
    size_t planes_bytes = 0;
    int32_t *ws = nullptr;
    size_t ws_bytes = 0;
    int *counters = nullptr;
    size_t counters_bytes = 0;
    int *status = nullptr;
    uint8_t *beam_wt = nullptr;   // beam weights as MMA operand tiles
    size_t beam_wt_bytes = 0;
    int32_t *corner_partial = nullptr;   // per-block pre-sums of the corner turn
    size_t corner_partial_bytes = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

// One slot of the host-buffer entry points: its own device input and output buffers, so that
// the device -> host copy of one slot's result overlaps the next slot's copies and compute.
struct HostIO {
    std::vector<cudaEvent_t> landed; // one per chunk in flight: its copy has completed
    cudaEvent_t computed = nullptr;  // the slot's correlation has completed
    cudaEvent_t delivered = nullptr; // the slot's result is in host memory
    bool in_flight = false;
    uint8_t *d_in = nullptr;
    size_t in_bytes = 0;
    int32_t *d_vis = nullptr;
    size_t vis_bytes = 0;
};

// Streams shared by the slots: host -> device copies, compute, device -> host copies.
struct HostStreams {
    cudaStream_t copy = nullptr;
    cudaStream_t compute = nullptr;
    cudaStream_t d2h = nullptr;
};

constexpr int kHostSlots = XE_HOST_SLOTS + 1;   // the last one serves xe_correlate_host

struct LaunchRec {
    int kind;                     // 0 stage, 1 tensor-core correlation, 2 int8 anchor,
                                  // 3 descriptor check of a correlation launch (option "checks")
    int eb;
    bool masked;                  // kind 0: the masking variant of the staging kernel
    JobTable jt;
    PlanDev pd;
    CheckLimits lim;              // kind 1 and 3: the lengths of the plan's device arrays
};

struct GraphRec {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> nodes;
};

struct Device {
    int id = -1;
    int n_sm = 0;
    std::string name;             // device name with blanks as '_' (the tuning cache's key)
    HostIO io[kHostSlots];
    HostStreams hs;
    std::map<std::vector<int64_t>, DevPlan *> plans;
    std::map<std::vector<int64_t>, TuneCfg> tuned;
    std::map<cudaStream_t, Scratch *> scratch;
    std::map<std::vector<int64_t>, GraphRec *> graphs;
    uint8_t *arena = nullptr;     // device memory the plan blobs are carved from
    size_t arena_used = 0;
};

static std::map<int, Device *> g_devs;
static thread_local TuneCfg g_last_cfg{0, 0, -1};

static int get_device(Device **out) {
    int dev = 0;
    const cudaError_t ge = cudaGetDevice(&dev);
    if (ge == cudaErrorNoDevice || ge == cudaErrorInsufficientDriver) {
        cudaGetLastError();
        return fail(XE_ENODEV, "no usable CUDA device: %s", cudaGetErrorString(ge));
    }
    XE_CUDA(ge);
    auto it = g_devs.find(dev);
    if (it != g_devs.end()) {
        *out = it->second;
        return XE_OK;
    }
    cudaDeviceProp prop;
    XE_CUDA(cudaGetDeviceProperties(&prop, dev));
    if (!(prop.major == 10 && prop.minor == 3))
        return fail(XE_ENODEV, "device %d (%s) is sm_%d%d; libxe is built for sm_103a only", dev,
                    prop.name, prop.major, prop.minor);
    Device *d = new Device;
    d->id = dev;
    d->n_sm = prop.multiProcessorCount;
    d->name = prop.name;
    for (char &ch : d->name)
        if (ch == ' ' || ch == '\t') ch = '_';
    g_devs[dev] = d;
    *out = d;
    return XE_OK;
}

static std::vector<int64_t> shape_key(const std::vector<JobShape> &jobs, int eb) {
    std::vector<int64_t> key{eb};
    for (const JobShape &j : jobs) {
        key.push_back(j.N);
        key.push_back(j.T);
        key.push_back(j.C);
        key.push_back(j.weight);
    }
    return key;
}

// ---- autotuning cache ------------------------------------------------------------------
//
// Tuned plan configurations are keyed by the batch shape with T bucketed: the number of
// 64-sample blocks of each job, rounded up to a power of two (a plan is built for the exact
// shape; only its CTA count, tile width and schedule are reused within a bucket).  With a
// cache file set (xe_tune_cache, or XE_TUNE_CACHE in the environment), entries for this GPU
// (name, SM count) are read from it and every newly tuned configuration is appended to it, so
// a later process reuses it without timing candidates.  One line per entry:
//   xe-tune 1 <gpu> <n_sm> <eb> <n_jobs> {<N> <T bucket> <C> <weight>}*n_jobs <n_cta> <tile_n> <sched>

static int64_t t_bucket(int64_t T) {
    const int64_t kb = (T + 63) / 64;
    int64_t b = 1;
    while (b < kb) b <<= 1;
    return b;
}

static std::vector<int64_t> tune_key(const std::vector<JobShape> &jobs, int eb) {
    std::vector<int64_t> key{eb};
    for (const JobShape &j : jobs) {
        key.push_back(j.N);
        key.push_back(t_bucket(j.T));
        key.push_back(j.C);
        key.push_back(j.weight);
    }
    return key;
}

struct TuneStats {
    int64_t timed = 0;            // candidate plans the autotuner timed in this process
    int64_t from_file = 0;        // tuned shapes taken from the cache file
};
static TuneStats g_tune_stats;
static std::string g_tune_path;
static bool g_tune_env_read = false;
// Entries read from (or written to) the cache file: (gpu, n_sm, key) -> configuration.
static std::map<std::pair<std::string, std::vector<int64_t>>, TuneCfg> g_tune_file;

static std::string gpu_id(const std::string &name, int n_sm) { return name + "/" + std::to_string(n_sm); }

static bool valid_cfg(const TuneCfg &c) {
    return c.n_cta >= 1 && c.n_cta <= 4096 && (c.tile_n == 128 || c.tile_n == 256) && c.sched >= 0 &&
           c.sched < kNumSched;
}

// Read every well-formed entry of `path` into g_tune_file; a missing file is empty.
static int load_tune_file(const std::string &path) {
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return XE_OK;
    char line[8192];
    while (fgets(line, sizeof line, f)) {
        char tag[16], gpu[256];
        int ver = 0, n_sm = 0, eb = 0, n_jobs = 0, used = 0;
        const char *q = line;
        if (sscanf(q, "%15s %d %255s %d %d %d%n", tag, &ver, gpu, &n_sm, &eb, &n_jobs, &used) != 6) continue;
        if (strcmp(tag, "xe-tune") != 0 || ver != 1 || n_jobs < 1 || n_jobs > kMaxJobs) continue;
        q += used;
        std::vector<int64_t> key{eb};
        bool ok = true;
        for (int k = 0; k < n_jobs && ok; ++k) {
            long long v[4];
            if (sscanf(q, "%lld %lld %lld %lld%n", &v[0], &v[1], &v[2], &v[3], &used) != 4) ok = false;
            else {
                q += used;
                for (long long x : v) key.push_back(x);
            }
        }
        TuneCfg c{0, 0, -1};
        if (!ok || sscanf(q, "%d %d %d", &c.n_cta, &c.tile_n, &c.sched) != 3 || !valid_cfg(c)) continue;
        g_tune_file[{gpu_id(gpu, n_sm), key}] = c;
    }
    fclose(f);
    return XE_OK;
}

static void read_tune_env() {
    if (g_tune_env_read) return;
    g_tune_env_read = true;
    const char *p = getenv("XE_TUNE_CACHE");
    if (p && *p && g_tune_path.empty()) {
        g_tune_path = p;
        load_tune_file(g_tune_path);
    }
}

// Record a tuned configuration in memory and, with a cache file set, append it there.
static int store_tune(const std::string &gpu, int n_sm, const std::vector<int64_t> &key, const TuneCfg &c) {
    g_tune_file[{gpu_id(gpu, n_sm), key}] = c;
    if (g_tune_path.empty()) return XE_OK;
    std::string line = "xe-tune 1 " + gpu + " " + std::to_string(n_sm) + " " + std::to_string(key[0]) + " " +
                       std::to_string((key.size() - 1) / 4);
    for (size_t k = 1; k < key.size(); ++k) line += " " + std::to_string(key[k]);
    line += " " + std::to_string(c.n_cta) + " " + std::to_string(c.tile_n) + " " + std::to_string(c.sched) + "\n";
    FILE *f = fopen(g_tune_path.c_str(), "a");
    if (!f) return fail(XE_EINVAL, "cannot append to the tuning cache %s", g_tune_path.c_str());
    const bool ok = fputs(line.c_str(), f) >= 0;
    fclose(f);
    return ok ? XE_OK : fail(XE_EINVAL, "cannot write the tuning cache %s", g_tune_path.c_str());
}

// The tuned configuration of a batch shape on device d: tuned in this process, else read
// from the cache file (then kept in the device's table).
static const TuneCfg *find_tuned(Device *d, const std::vector<int64_t> &key) {
    auto it = d->tuned.find(key);
    if (it != d->tuned.end()) return &it->second;
    read_tune_env();
    auto f = g_tune_file.find({gpu_id(d->name, d->n_sm), key});
    if (f == g_tune_file.end()) return nullptr;
    ++g_tune_stats.from_file;
    return &(d->tuned[key] = f->second);
}

constexpr size_t kMaxCachedPlans = 4096;   // a plan blob holds a few KB to a few MB
constexpr size_t kPlanArenaBytes = size_t(64) << 20;

// Bounded plan cache: a stream of ever-new batch shapes (e.g. merged stream frames) would
// otherwise keep one device blob per shape forever.  Called before a batch builds its launch
// records (none of which may hold a plan yet); plans of launches already queued may still be
// read, so the cache (and the graphs that point into it) is dropped only once the device is
// idle.  Half of the arena is kept free for the plans of the batch that follows.
static int trim_plan_cache(Device *d) {
    if (d->plans.size() < kMaxCachedPlans && d->arena_used <= kPlanArenaBytes / 2) return XE_OK;
    ++g_rc.trims;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(XE_ECUDA, "sync before dropping plans: %s", cudaGetErrorString(e));
    for (auto &kv : d->plans) {
        if (kv.second->own_blob) cudaFree(kv.second->blob);
        if (kv.second->ready) cudaEventDestroy(kv.second->ready);
        delete kv.second;
    }
    d->plans.clear();
    d->arena_used = 0;
    for (auto &kv : d->graphs) {
        cudaGraphExecDestroy(kv.second->exec);
        cudaGraphDestroy(kv.second->graph);
        delete kv.second;
    }
    d->graphs.clear();
    return XE_OK;
}

// The device plan of a batch shape and configuration, for launches on stream s.  A new plan
// is carved from the device's plan arena (one allocation per device, on first use) and
// uploaded with a copy ordered on s, so building a plan neither allocates nor waits for the
// device; launches on another stream wait for the upload's event.
static int get_plan(Device *d, const std::vector<JobShape> &jobs, int eb, const TuneCfg &cfg, cudaStream_t s,
                    DevPlan **out) {
    std::vector<int64_t> key = shape_key(jobs, eb);
    key.push_back(cfg.n_cta);
    key.push_back(cfg.tile_n);
    key.push_back(cfg.sched);
    auto it = d->plans.find(key);
    if (it != d->plans.end()) {
        DevPlan *p = it->second;
        if (p->upload_stream != s) XE_CUDA(cudaStreamWaitEvent(s, p->ready, 0));
        *out = p;
        return XE_OK;
    }
    const int64_t t_plan = host_ns();
    DevPlan *p = new DevPlan;
    if (!build_plan(jobs, eb, cfg, p->host)) {
        delete p;
        return fail(XE_EINVAL, "internal: plan does not cover the triangle");
    }
    const HostPlan &h = p->host;
    const size_t b_t = h.tiles.size() * sizeof(Tile), b_s = h.segs.size() * sizeof(Seg);
    const size_t b_o = h.seg_off.size() * sizeof(int), b_l = (h.tile_slots.size() + 1) * sizeof(int);
    const size_t o_s = (b_t + 255) / 256 * 256, o_o = o_s + (b_s + 255) / 256 * 256,
                 o_l = o_o + (b_o + 255) / 256 * 256, total = o_l + b_l;
    const size_t carve = (total + 255) / 256 * 256;
    if (!d->arena && cudaMalloc(reinterpret_cast<void **>(&d->arena), kPlanArenaBytes) != cudaSuccess) {
        cudaGetLastError();
        d->arena = nullptr;
    }
    if (d->arena && d->arena_used + carve <= kPlanArenaBytes) {
        p->blob = d->arena + d->arena_used;
        d->arena_used += carve;
    } else if (cudaMalloc(&p->blob, total) == cudaSuccess) {
        p->own_blob = true;
    } else {
        cudaGetLastError();
        delete p;
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        return fail(XE_ENOMEM, "cannot allocate %zu bytes for a plan (%zu of %zu bytes free, %zu plans cached)",
                    total, fr, tot, d->plans.size());
    }
    std::vector<uint8_t> host(total, 0);
    memcpy(host.data(), h.tiles.data(), b_t);
    memcpy(host.data() + o_s, h.segs.data(), b_s);
    memcpy(host.data() + o_o, h.seg_off.data(), b_o);
    if (!h.tile_slots.empty()) memcpy(host.data() + o_l, h.tile_slots.data(), b_l - sizeof(int));
    // From pageable memory the copy returns once the bytes are staged (the vector may go) and
    // lands in stream order on s, before any launch enqueued on s after it.
    cudaError_t e = cudaEventCreateWithFlags(&p->ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->blob, host.data(), total, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(p->ready, s);
    if (e != cudaSuccess) {
        if (p->own_blob) cudaFree(p->blob);
        if (p->ready) cudaEventDestroy(p->ready);
        delete p;
        return fail(XE_ECUDA, "plan upload failed: %s", cudaGetErrorString(e));
    }
    p->upload_stream = s;
    ++g_rc.plans_built;
    g_rc.plan_ns += host_ns() - t_plan;
    uint8_t *base = static_cast<uint8_t *>(p->blob);
    p->d_tiles = reinterpret_cast<const Tile *>(base);
    p->d_segs = reinterpret_cast<const Seg *>(base + o_s);
    p->d_seg_off = reinterpret_cast<const int *>(base + o_o);
    p->d_tile_slots = reinterpret_cast<const int *>(base + o_l);
    d->plans[key] = p;
    *out = p;
    return XE_OK;
}

static int grow(void **ptr, size_t *have, size_t need, bool zero, bool headroom = true) {
    if (*have >= need && *ptr) return XE_OK;
    if (*ptr) {
        ++g_rc.regrowths;
        cudaError_t e = cudaDeviceSynchronize();  // nothing may still use the old buffer
        if (e != cudaSuccess) return fail(XE_ECUDA, "sync before regrow: %s", cudaGetErrorString(e));
        cudaFree(*ptr);
        *ptr = nullptr;
        *have = 0;
    }
    // Regrowing synchronises the device, so leave room for batches half as large again
    // (a stream's batches grow a few jobs at a time while its load ramps up).
    size_t sz = headroom ? need + need / 2 + 256 : need;
    if (cudaMalloc(ptr, sz) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        return fail(XE_ENOMEM, "cannot allocate %zu bytes of scratch (%zu of %zu bytes free)", sz, fr, tot);
    }
    if (zero) {
        // cudaMemset runs on the legacy stream, which does not order work on non-blocking
        // streams: finish it before any kernel reads the buffer.
        XE_CUDA(cudaMemset(*ptr, 0, sz));
        XE_CUDA(cudaStreamSynchronize(0));
    }
    *have = sz;
    return XE_OK;
}

static int get_scratch(Device *d, cudaStream_t s, Scratch **out) {
    auto it = d->scratch.find(s);
    if (it != d->scratch.end()) {
        *out = it->second;
        return XE_OK;
    }
    Scratch *sc = new Scratch;
    if (cudaMalloc(&sc->status, sizeof(int)) != cudaSuccess) {
        delete sc;
        return fail(XE_ENOMEM, "cannot allocate the status word");
    }
    XE_CUDA(cudaMemset(sc->status, 0, sizeof(int)));
    XE_CUDA(cudaStreamSynchronize(0));          // (see grow)
    for (auto &e : sc->ev) XE_CUDA(cudaEventCreate(&e));
    d->scratch[s] = sc;
    *out = sc;
    return XE_OK;
}

static thread_local cudaEvent_t g_last_ev[4] = {nullptr, nullptr, nullptr, nullptr};
static thread_local const int *g_job_acc = nullptr;   // per-job accumulate flags (stream server)
// Per-job masking of a masked batch (null for plain batches).
static thread_local const xe_masked_job *g_job_mask = nullptr;
// Per-job input views of a view call (null: every input is a plain [C][T][N] array).
static thread_local const xe_view *g_job_view = nullptr;

static void set_view(JobDev &jd, const xe_job &j, const xe_view *v) {
    if (v) {
        jd.s_c = v->chan_stride;
        jd.s_t = v->time_stride;
        jd.s_seg = v->seg_stride;
        jd.seg = int(v->seg_inputs);
    } else {
        jd.s_c = j.T * int64_t(j.N);
        jd.s_t = j.N;
        jd.s_seg = 0;
        jd.seg = j.N;
    }
}

static int check_job(const uint8_t *in, int N, int64_t T, int C, const int32_t *vis) {
    if (!in || !vis) return fail(XE_EINVAL, "null input or output pointer");
    if (N < 1 || N > XE_MAX_N) return fail(XE_EINVAL, "N=%d outside [1, %d]", N, XE_MAX_N);
    if (T < 1) return fail(XE_EINVAL, "T=%lld < 1", (long long)T);
    if (T > XE_MAX_T) return fail(XE_EOVERFLOW, "T=%lld > %lld: int32 visibilities could overflow",
                                  (long long)T, (long long)XE_MAX_T);
    if (C < 1) return fail(XE_EINVAL, "n_chan=%d < 1", C);
    if (reinterpret_cast<uintptr_t>(vis) & 7) return fail(XE_EINVAL, "vis must be 8-byte aligned");
    return XE_OK;
}

// Build the launch sequence for a batch (allocating scratch and plans as needed), without
// enqueuing anything.  `forced` overrides the plan configuration (autotuner candidates).
static int build_launches(Device *d, Scratch *sc, const xe_job *jobs, int n_jobs, int algo,
                          int accumulate, const TuneCfg *forced, cudaStream_t s, std::vector<LaunchRec> &out) {
    out.clear();
    if (algo == XE_ALGO_IMMA) {
        for (int g0 = 0; g0 < n_jobs; g0 += kMaxJobs) {
            const int ng = std::min(n_jobs - g0, kMaxJobs);
            LaunchRec r{};
            r.kind = 2;
            r.eb = 1;
            JobTable &jt = r.jt;
            jt.n_jobs = ng;
            jt.accumulate = accumulate ? 1 : 0;
            int64_t blocks = 0;
            for (int q = 0; q < ng; ++q) {
                const xe_job &j = jobs[g0 + q];
                JobDev &jd = jt.jobs[q];
                jd.in = j.in;
                jd.vis = j.vis;
                jd.T = j.T;
                jd.T_in = j.T;
                set_view(jd, j, nullptr);
                jd.N = j.N;
                jd.C = j.n_chan;
                jd.vis_chan_elems = int64_t(j.N) * (j.N + 1);
                jd.stage_block0 = blocks;
                blocks += imma_blocks(j.N, j.n_chan);
            }
            jt.total_stage_blocks = blocks;
            out.push_back(r);
        }
        return XE_OK;
    }
    const int eb = g_opt.operand_bytes;
    if (g_job_mask && eb != 1) return fail(XE_EINVAL, "masked correlation needs 1-byte operands");
    const int64_t wt = g_opt.exact_chunk_t / samples_per_stage(eb) * samples_per_stage(eb);
    // A masked group holds at most half the job slots: each job may add its count job.
    const size_t group = g_job_mask ? size_t(kMaxJobs / 2) : size_t(kMaxJobs);
    int64_t max_T = 0;
    for (int q = 0; q < n_jobs; ++q) max_T = std::max(max_T, jobs[q].T);
    const int64_t n_win = (max_T + wt - 1) / wt;
    size_t max_planes = 0, max_ws = 0, max_counters = 0;
    const size_t first_rec = out.size();
    for (int64_t w = 0; w < n_win; ++w) {
        std::vector<int> act;
        for (int q = 0; q < n_jobs; ++q)
            if (jobs[q].T > w * wt) act.push_back(q);
        for (size_t g0 = 0; g0 < act.size(); g0 += group) {
            const int ng = int(std::min(act.size() - g0, group));
            std::vector<JobShape> shapes;
            LaunchRec st{};
            st.jt.status = sc->status;
            st.jt.checks = g_opt.checks;
            st.kind = 0;
            st.eb = eb;
            JobTable &jt = st.jt;
            jt.n_jobs = ng;
            jt.accumulate = (w > 0 || accumulate) ? 1 : 0;
            size_t plane_off = 0;
            int64_t blocks = 0;
            for (int k = 0; k < ng; ++k) {
                const xe_job &j = jobs[act[g0 + size_t(k)]];
                const int64_t Tw = std::min(j.T - w * wt, wt);
                jt.jobs[k].accumulate = g_job_acc ? g_job_acc[act[g0 + size_t(k)]] : 0;
                shapes.push_back(JobShape{j.N, Tw, j.n_chan});
                JobDev &jd = jt.jobs[k];
                jd.in = j.in;
                jd.vis = j.vis;
                jd.T = Tw;
                jd.t0 = w * wt;
                jd.T_in = j.T;
                set_view(jd, j, g_job_view ? &g_job_view[act[g0 + size_t(k)]] : nullptr);
                jd.N = j.N;
                jd.n_pad = n_pad_of(j.N);
                jd.C = j.n_chan;
                jd.kblocks = int(kblocks_of(Tw, eb));
                jd.plane_chan_bytes = int64_t(jd.kblocks) * 2 * jd.n_pad * kRowBytes;
                jd.vis_chan_elems = int64_t(j.N) * (j.N + 1);
                jd.stage_block0 = blocks;
                if (g_job_mask) {
                    const xe_masked_job &mj = g_job_mask[act[g0 + size_t(k)]];
                    jd.mode = kModeMasked | (mj.encoding == XE_ENC_OFFSET ? kModeOffsetBinary : 0);
                    jd.flags = mj.flags;
                    st.masked = true;
                }
                blocks += int64_t(j.n_chan) * jd.kblocks * (jd.n_pad / 256);
                plane_off += size_t(jd.plane_chan_bytes) * size_t(j.n_chan);
            }
            // Count jobs after every data job, with no staging blocks of their own (their
            // planes are written by their masked job's staging): their stage_block0 is the
            // total, so the staging kernel's job search never lands on them.
            std::vector<int> count_of(size_t(ng), -1);
            for (int k = 0; k < ng && g_job_mask; ++k) {
                const int q = act[g0 + size_t(k)];
                if (!g_job_mask[q].counts) continue;
                const int idx = jt.n_jobs++;
                JobDev &cj = jt.jobs[idx];
                cj = jt.jobs[k];
                cj.in = nullptr;
                cj.flags = nullptr;
                cj.count_planes = nullptr;
                cj.mode = kModeCount;
                // The epilogue writes (or adds) n_ij into the caller's counts directly.
                cj.accumulate = g_job_mask[q].accumulate ? 1 : 0;
                cj.vis = g_job_mask[q].counts;
                cj.vis_chan_elems = int64_t(cj.N) * (cj.N + 1) / 2;
                cj.stage_block0 = blocks;
                // One count k-iteration covers two sample blocks (the validity of block kb is
                // in slot kb % 2 of iteration kb / 2): half the k-iterations, full stages.
                cj.kblocks = (jt.jobs[k].kblocks + 1) / 2;
                cj.plane_chan_bytes = int64_t(cj.kblocks) * 2 * cj.n_pad * kRowBytes;
                count_of[size_t(k)] = idx;
                shapes.push_back(shapes[size_t(k)]);
                shapes.back().T = int64_t(cj.kblocks) * samples_per_stage(eb);
                shapes.back().weight = g_opt.count_weight;
                plane_off += size_t(cj.plane_chan_bytes) * size_t(cj.C);
            }
            jt.total_stage_blocks = blocks;
            // The staging kernel decodes its items in 32-bit arithmetic.  (Unreachable in
            // practice: 2^31 items would stage 64 TB of planes.)
            if (blocks > 0x7fffffffLL) return fail(XE_EINVAL, "batch too large for one staging grid");
            // Plane offsets within the scratch; the base is bound once every group is known
            // (the scratch is sized for the largest group: growing it per group would free
            // the buffer earlier groups' records already point into).
            max_planes = std::max(max_planes, plane_off);
            size_t off = 0;
            for (int k = 0; k < jt.n_jobs; ++k) {
                jt.jobs[k].planes = reinterpret_cast<const uint8_t *>(off);
                off += size_t(jt.jobs[k].plane_chan_bytes) * size_t(jt.jobs[k].C);
            }
            for (int k = 0; k < ng; ++k)
                if (count_of[size_t(k)] >= 0)
                    jt.jobs[k].count_planes = const_cast<uint8_t *>(jt.jobs[count_of[size_t(k)]].planes);
            // Batches of the streaming server (per-job accumulate flags, default tiling): no host
            // plan.  Their shapes change from pass to pass as frames merge, and a new plan costs
            // milliseconds of host time; whole tiles dealt round-robin over the CTAs need none.
            if (!forced && g_job_acc && !g_job_mask && g_opt.implicit_plans && g_opt.sched < 0 &&
                (g_opt.tile_n == 0 || g_opt.tile_n == kBN)) {
                int tiles = 0;
                for (int k = 0; k < jt.n_jobs; ++k) {
                    JobDev &jd = jt.jobs[k];
                    jd.tile0 = tiles;
                    jd.tiles_per_chan = int(count_tiles(jd.N, kBN));
                    tiles += jd.tiles_per_chan * jd.C;
                }
                LaunchRec tc = st;
                tc.kind = 1;
                PlanDev &pd = tc.pd;
                pd = PlanDev{};
                pd.implicit = 1;
                pd.n_tiles = tiles;
                pd.n_cta = std::min(tiles, g_opt.n_cta > 0 ? g_opt.n_cta : d->n_sm);
                pd.status = sc->status;
                pd.inject_stall = g_opt.inject_stall;
                out.push_back(st);
                out.push_back(tc);
                continue;
            }
            // The correlation launch(es) of the group: one for data and count jobs together,
            // or (option "count_launch") the data jobs, then the count jobs in a launch of their
            // own after it (both read the planes this group's staging wrote).
            auto make_tc = [&](const JobTable &jtab, const std::vector<JobShape> &shp, LaunchRec &tc) -> int {
                TuneCfg cfg;
                if (forced) {
                    cfg = *forced;
                } else {
                    const TuneCfg *t = find_tuned(d, tune_key(shp, eb));
                    cfg = t ? *t : heuristic(shp, eb, d->n_sm);
                }
                g_last_cfg = cfg;
                DevPlan *p = nullptr;
                const int rc = get_plan(d, shp, eb, cfg, s, &p);
                if (rc) return rc;
                const size_t ws_need =
                    size_t(std::max(1, p->host.n_partial)) * size_t(kWsSlotElems) * sizeof(int32_t);
                max_ws = std::max(max_ws, ws_need);
                max_counters = std::max(max_counters, p->host.tiles.size() * sizeof(int));
                tc = st;
                tc.jt = jtab;
                tc.kind = 1;
                PlanDev &pd = tc.pd;
                pd.tiles = p->d_tiles;
                pd.segs = p->d_segs;
                pd.seg_off = p->d_seg_off;
                pd.tile_slots = p->d_tile_slots;
                pd.n_tiles = int(p->host.tiles.size());
                pd.n_cta = p->host.n_cta;
                pd.ws = nullptr;          // bound below
                pd.counters = nullptr;
                pd.status = sc->status;
                pd.inject_stall = g_opt.inject_stall;
                tc.lim = CheckLimits{};
                tc.lim.n_tiles = int(p->host.tiles.size());
                tc.lim.n_segs = int(p->host.segs.size());
                tc.lim.n_seg_off = int(p->host.seg_off.size());
                tc.lim.n_tile_slots = int(p->host.tile_slots.size());
                // All CTAs of the launch must be resident together for the exchange's wait.
                pd.pair_exchange = p->host.pair_exchange && p->host.n_cta <= d->n_sm ? 1 : 0;
                return XE_OK;
            };
            out.push_back(st);
            if (g_opt.count_launch && jt.n_jobs > ng) {
                LaunchRec data_rec, count_rec;
                JobTable jd_tab = jt, jc_tab = jt;
                jd_tab.n_jobs = ng;
                jc_tab.n_jobs = jt.n_jobs - ng;
                for (int k = 0; k < jc_tab.n_jobs; ++k) jc_tab.jobs[k] = jt.jobs[ng + k];
                std::vector<JobShape> sd(shapes.begin(), shapes.begin() + ng), sc_(shapes.begin() + ng, shapes.end());
                for (JobShape &x : sc_) x.weight = 100;
                int rc = make_tc(jd_tab, sd, data_rec);
                if (rc) return rc;
                rc = make_tc(jc_tab, sc_, count_rec);
                if (rc) return rc;
                out.push_back(data_rec);
                out.push_back(count_rec);
            } else {
                LaunchRec tc;
                const int rc = make_tc(jt, shapes, tc);
                if (rc) return rc;
                out.push_back(tc);
            }
        }
    }
    // Size the scratch for the largest group, then bind it into every record.
    {
        int rc = grow(reinterpret_cast<void **>(&sc->planes), &sc->planes_bytes, std::max<size_t>(max_planes, 1), false);
        if (rc) return rc;
        rc = grow(reinterpret_cast<void **>(&sc->ws), &sc->ws_bytes, std::max<size_t>(max_ws, 1), false);
        if (rc) return rc;
        rc = grow(reinterpret_cast<void **>(&sc->counters), &sc->counters_bytes, std::max<size_t>(max_counters, 4), true);
        if (rc) return rc;
        for (size_t r = first_rec; r < out.size(); ++r) {
            LaunchRec &rec = out[r];
            if (rec.kind != 0 && rec.kind != 1) continue;
            for (int k = 0; k < rec.jt.n_jobs; ++k) {
                JobDev &jd = rec.jt.jobs[k];
                jd.planes = sc->planes + reinterpret_cast<uintptr_t>(jd.planes);
                if (jd.count_planes) jd.count_planes = sc->planes + reinterpret_cast<uintptr_t>(jd.count_planes);
            }
            if (rec.kind == 1) {
                rec.pd.ws = sc->ws;
                rec.pd.counters = sc->counters;
                rec.lim.planes = sc->planes;
                rec.lim.planes_bytes = int64_t(sc->planes_bytes);
                rec.lim.ws_slots = int64_t(sc->ws_bytes / (size_t(kWsSlotElems) * sizeof(int32_t)));
                rec.lim.n_counters = int64_t(sc->counters_bytes / sizeof(int));
            }
        }
    }
    if (g_opt.checks) {
        // Each group's checks run before its staging (which writes through the job table):
        // one check record per correlation launch of the group, then the group's records.
        std::vector<LaunchRec> grouped(out.begin(), out.begin() + std::ptrdiff_t(first_rec));
        for (size_t r = first_rec; r < out.size();) {
            size_t e = r + 1;
            while (e < out.size() && out[e].kind != 0) ++e;
            for (size_t k = r; k < e; ++k) {
                if (out[k].kind != 1) continue;
                if (g_opt.check_corrupt == 1) out[k].pd.n_tiles = 0;
                if (g_opt.check_corrupt == 2) out[k].jt.jobs[0].plane_chan_bytes += 64;
                LaunchRec c = out[k];
                c.kind = 3;
                grouped.push_back(c);
            }
            for (size_t k = r; k < e; ++k) grouped.push_back(out[k]);
            r = e;
        }
        out.swap(grouped);
    }
    return XE_OK;
}

static cudaError_t enqueue(const LaunchRec &r, cudaStream_t s) {
    if (r.kind == 0) return launch_stage(r.jt, r.eb, s, r.masked);
    if (r.kind == 1) return launch_tc(r.jt, r.pd, r.eb, s);
    if (r.kind == 3) return launch_check(r.jt, r.pd, r.lim, s);
    return launch_imma(r.jt, s);
}

static cudaKernelNodeParams node_params(const LaunchRec &r, void **args) {
    cudaKernelNodeParams p{};
    args[0] = const_cast<JobTable *>(&r.jt);
    args[1] = const_cast<PlanDev *>(&r.pd);
    args[2] = const_cast<CheckLimits *>(&r.lim);
    p.kernelParams = args;
    p.extra = nullptr;
    if (r.kind == 0) {
        p.func = const_cast<void *>(stage_kernel_fn(r.eb, r.masked));
        p.gridDim = dim3(stage_grid(r.jt, r.eb, r.masked));
        p.blockDim = dim3(256);
        p.sharedMemBytes = unsigned(stage_smem_bytes(r.eb, r.masked));
    } else if (r.kind == 1) {
        p.func = const_cast<void *>(tc_kernel_fn(r.eb));
        p.gridDim = dim3(unsigned(r.pd.n_cta));
        p.blockDim = dim3(kTcThreads);
        p.sharedMemBytes = unsigned(tc_smem_bytes());
    } else if (r.kind == 3) {
        p.func = const_cast<void *>(check_kernel_fn());
        p.gridDim = dim3(1);
        p.blockDim = dim3(256);
        p.sharedMemBytes = 0;
    } else {
        p.func = const_cast<void *>(imma_kernel_fn());
        p.gridDim = dim3(unsigned(r.jt.total_stage_blocks));
        p.blockDim = dim3(128);
        p.sharedMemBytes = 0;
    }
    return p;
}

// Time one launch sequence (median of `reps` runs after one warm-up) on stream s.
static float time_launches(const std::vector<LaunchRec> &recs, cudaStream_t s, Scratch *sc, int reps) {
    std::vector<float> t;
    for (int k = 0; k < reps + 1; ++k) {
        cudaEventRecord(sc->ev[0], s);
        for (const LaunchRec &r : recs) enqueue(r, s);
        cudaEventRecord(sc->ev[2], s);
        cudaEventSynchronize(sc->ev[2]);
        float ms = 0;
        cudaEventElapsedTime(&ms, sc->ev[0], sc->ev[2]);
        if (k > 0) t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    return t.empty() ? 1e30f : t[t.size() / 2];
}

// Pick tile width and schedule for a batch shape by timing the candidates (each candidate
// overwrites the batch's own outputs, so only non-accumulating calls tune).
static int autotune(Device *d, Scratch *sc, const xe_job *jobs, int n_jobs, cudaStream_t s) {
    const int eb = g_opt.operand_bytes;
    if (n_jobs > kMaxJobs || n_jobs < 1) return XE_OK;
    std::vector<JobShape> shapes;
    for (int q = 0; q < n_jobs; ++q) {
        if (jobs[q].T > g_opt.exact_chunk_t) return XE_OK;  // windowed: keep the heuristic
        shapes.push_back(JobShape{jobs[q].N, jobs[q].T, jobs[q].n_chan});
    }
    for (JobShape &j : shapes) j.T = std::min<int64_t>(j.T, g_opt.exact_chunk_t);
    const std::vector<int64_t> key = tune_key(shapes, eb);
    if (find_tuned(d, key)) return XE_OK;
    const int n_cta = g_opt.n_cta > 0 ? g_opt.n_cta : d->n_sm;
    TuneCfg best = heuristic(shapes, eb, d->n_sm);
    float best_ms = 1e30f;
    const int widths[2] = {256, 128};
    for (int wi = 0; wi < 2; ++wi) {
        if (g_opt.tile_n > 0 && widths[wi] != g_opt.tile_n) continue;
        for (int si = 0; si < kNumSched; ++si) {
            if (g_opt.sched >= 0 && si != g_opt.sched) continue;
            TuneCfg c{n_cta, widths[wi], si};
            std::vector<LaunchRec> recs;
            int rc = build_launches(d, sc, jobs, n_jobs, XE_ALGO_TC, 0, &c, s, recs);
            if (rc) return rc;
            const float ms = time_launches(recs, s, sc, 3);
            ++g_tune_stats.timed;
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
    }
    XE_CUDA(cudaGetLastError());
    d->tuned[key] = best;
    return store_tune(d->name, d->n_sm, key, best);
}

// Enqueue a batch of jobs (all validated) on stream s.
static int run_jobs(const xe_job *jobs, int n_jobs, int algo, cudaStream_t s, int accumulate = 0,
                    int use_graph = 0) {
    Device *d = nullptr;
    int rc = get_device(&d);
    if (rc) return rc;
    Scratch *sc = nullptr;
    rc = get_scratch(d, s, &sc);
    if (rc) return rc;
    rc = trim_plan_cache(d);
    if (rc) return rc;
    // Candidates overwrite the jobs' outputs, so calls that add into any output never tune.
    if (algo == XE_ALGO_TC && g_opt.autotune && !accumulate && !g_job_acc) {
        rc = autotune(d, sc, jobs, n_jobs, s);
        if (rc) return rc;
    }
    std::vector<LaunchRec> recs;
    const int64_t t_build = host_ns();
    rc = build_launches(d, sc, jobs, n_jobs, algo, accumulate, nullptr, s, recs);
    ++g_rc.batches;
    g_rc.build_ns += host_ns() - t_build;
    g_opt.inject_stall = 0;
    if (rc) return rc;
    const bool timing = g_opt.timing != 0;
    if (timing) XE_CUDA(cudaEventRecord(sc->ev[0], s));

    if (use_graph && algo == XE_ALGO_TC && !g_job_mask) {
        // One CUDA graph per (stream, batch shape, launch geometry); the kernel arguments
        // (pointers) are refreshed in place on every replay.
        std::vector<int64_t> key{reinterpret_cast<int64_t>(s), accumulate};
        for (int q = 0; q < n_jobs; ++q) {
            key.push_back(jobs[q].N);
            key.push_back(jobs[q].T);
            key.push_back(jobs[q].n_chan);
        }
        for (const LaunchRec &r : recs) {
            key.push_back(r.kind);
            key.push_back(r.kind == 1 ? int64_t(r.pd.n_cta) : r.jt.total_stage_blocks);
            key.push_back(reinterpret_cast<int64_t>(r.kind == 1 ? static_cast<const void *>(r.pd.segs)
                                                                : nullptr));
        }
        GraphRec *g = nullptr;
        auto it = d->graphs.find(key);
        if (it == d->graphs.end()) {
            XE_CUDA(tc_prepare());
            XE_CUDA(stage_prepare());
            g = new GraphRec;
            XE_CUDA(cudaGraphCreate(&g->graph, 0));
            cudaGraphNode_t prev = nullptr;
            for (const LaunchRec &r : recs) {
                void *args[3];
                cudaKernelNodeParams kp = node_params(r, args);
                cudaGraphNode_t node;
                XE_CUDA(cudaGraphAddKernelNode(&node, g->graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
                g->nodes.push_back(node);
                prev = node;
            }
            XE_CUDA(cudaGraphInstantiate(&g->exec, g->graph, 0));
            d->graphs[key] = g;
        } else {
            g = it->second;
            for (size_t k = 0; k < recs.size(); ++k) {
                void *args[3];
                cudaKernelNodeParams kp = node_params(recs[k], args);
                XE_CUDA(cudaGraphExecKernelNodeSetParams(g->exec, g->nodes[k], &kp));
            }
        }
        if (timing) XE_CUDA(cudaEventRecord(sc->ev[1], s));
        XE_CUDA(cudaGraphLaunch(g->exec, s));
        if (timing) XE_CUDA(cudaEventRecord(sc->ev[2], s));
    } else {
        bool marked = false;
        for (const LaunchRec &r : recs) {
            if (timing && !marked && r.kind != 0 && r.kind != 3) {
                XE_CUDA(cudaEventRecord(sc->ev[1], s));   // staging done (or none)
                marked = true;
            }
            XE_CUDA(enqueue(r, s));
        }
        if (timing && !marked) XE_CUDA(cudaEventRecord(sc->ev[1], s));
        // Counts are written by the correlation kernel itself: nothing follows it.
        if (timing) XE_CUDA(cudaEventRecord(sc->ev[2], s));
    }
    if (timing) {
        XE_CUDA(cudaEventRecord(sc->ev[3], s));
        for (int k = 0; k < 4; ++k) g_last_ev[k] = sc->ev[k];
    }
    return XE_OK;
}

int run_jobs_accumulate(const xe_job *jobs, int n_jobs, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    return run_jobs(jobs, n_jobs, XE_ALGO_TC, s, 1);
}

int release_stream_scratch(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    Device *d = nullptr;
    int rc = get_device(&d);
    if (rc) return rc;
    auto it = d->scratch.find(s);
    if (it == d->scratch.end()) return XE_OK;
    XE_CUDA(cudaStreamSynchronize(s));
    Scratch *sc = it->second;
    d->scratch.erase(it);
    cudaFree(sc->planes);
    cudaFree(sc->ws);
    cudaFree(sc->counters);
    cudaFree(sc->status);
    cudaFree(sc->beam_wt);
    cudaFree(sc->corner_partial);
    for (cudaEvent_t e : sc->ev)
        if (e) cudaEventDestroy(e);
    delete sc;
    return XE_OK;
}

int reserve_stream_scratch(cudaStream_t s, int max_jobs, int N, int64_t max_T) {
    if (max_jobs < 1 || N < 1 || N > XE_MAX_N || max_T < 1) return XE_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    Device *d = nullptr;
    int rc = get_device(&d);
    if (rc) return rc;
    Scratch *sc = nullptr;
    rc = get_scratch(d, s, &sc);
    if (rc) return rc;
    // The bounds build_launches meets for such batches: one launch group holds at most
    // kMaxJobs jobs, each staged over one exact window at most; 128-wide tiles are the most
    // numerous; the schedules give at most two partial segments per CTA (whole tiles for
    // uneven lengths).
    const int eb = g_opt.operand_bytes;
    const int64_t wt = g_opt.exact_chunk_t / samples_per_stage(eb) * samples_per_stage(eb);
    const size_t jobs = size_t(std::min(max_jobs, kMaxJobs));
    const size_t planes = jobs * size_t(kblocks_of(std::min(max_T, wt), eb)) * 2 * size_t(n_pad_of(N)) * kRowBytes;
    const size_t counters = jobs * size_t(count_tiles(N, 128)) * sizeof(int);
    const size_t ws = size_t(2 * d->n_sm) * size_t(kWsSlotElems) * sizeof(int32_t);
    rc = grow(reinterpret_cast<void **>(&sc->planes), &sc->planes_bytes, planes, false, false);
    if (rc) return rc;
    rc = grow(reinterpret_cast<void **>(&sc->ws), &sc->ws_bytes, ws, false, false);
    if (rc) return rc;
    return grow(reinterpret_cast<void **>(&sc->counters), &sc->counters_bytes, counters, true, false);
}

int64_t option_exact_chunk_t() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_opt.exact_chunk_t;
}

int take_inject_stall() {
    std::lock_guard<std::mutex> lk(g_mu);
    const int v = g_opt.inject_stall;
    g_opt.inject_stall = 0;
    return v;
}

int run_jobs_mixed(const xe_job *jobs, const int *accumulate, int n_jobs, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_job_acc = accumulate;
    const int rc = run_jobs(jobs, n_jobs, XE_ALGO_TC, s, 0);
    g_job_acc = nullptr;
    return rc;
}

static int plan_from_args(const int *N, const int64_t *T, const int *n_chan, int n_jobs, int n_cta,
                          int sched, int tile_n, HostPlan &p) {
    if (!N || !T || !n_chan || n_jobs < 1 || n_cta < 1) return fail(XE_EINVAL, "bad plan query");
    if (sched < -1 || sched >= kNumSched) return fail(XE_EINVAL, "bad schedule");
    if (tile_n != 0 && tile_n != 128 && tile_n != 256) return fail(XE_EINVAL, "bad tile width");
    std::vector<JobShape> shapes;
    for (int q = 0; q < n_jobs; ++q) {
        if (N[q] < 1 || T[q] < 1 || n_chan[q] < 1) return fail(XE_EINVAL, "bad job %d", q);
        shapes.push_back(JobShape{N[q], T[q], n_chan[q]});
    }
    TuneCfg c = heuristic(shapes, g_opt.operand_bytes, n_cta);
    c.n_cta = n_cta;
    if (sched >= 0) c.sched = sched;
    if (tile_n > 0) c.tile_n = tile_n;
    if (!build_plan(shapes, g_opt.operand_bytes, c, p))
        return fail(XE_EINVAL, "plan does not cover the triangle");
    return XE_OK;
}

}  // namespace xe

using namespace xe;

extern "C" {

const char *xe_strerror(int code) {
    switch (code) {
        case XE_OK: return "ok";
        case XE_EINVAL: return "invalid argument";
        case XE_EOVERFLOW: return "integration too long for exact int32 visibilities";
        case XE_ENOMEM: return "out of memory";
        case XE_EBUDGET: return "HBM budget exceeded";
        case XE_EAGAIN: return "try again";
        case XE_ETIMEOUT: return "a bounded wait timed out";
        case XE_ECUDA: return "CUDA error";
        case XE_ENODEV: return "no usable sm_103 device";
        case XE_ECLOSED: return "stream closed";
        case XE_ECHECK: return "a device-side check of a launch's descriptors failed";
        default: return "unknown error";
    }
}

const char *xe_last_error(void) { return g_err; }

int xe_version(void) { return 100; }

double xe_cmac(int64_t N, int64_t T, int64_t C) {
    return double(C) * double(T) * double(N) * double(N + 1) / 2.0;
}

int xe_set_option(const char *key, int64_t value) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!key) return fail(XE_EINVAL, "null option key");
    if (!strcmp(key, "operand_bytes")) {
        if (value != 1 && value != 2) return fail(XE_EINVAL, "operand_bytes must be 1 or 2");
        g_opt.operand_bytes = int(value);
    } else if (!strcmp(key, "exact_chunk_t")) {
        if (value < 64 || value > kExactChunkT)
            return fail(XE_EINVAL, "exact_chunk_t must lie in [64, %lld]", (long long)kExactChunkT);
        g_opt.exact_chunk_t = value;
    } else if (!strcmp(key, "n_cta")) {
        if (value < 0 || value > 4096) return fail(XE_EINVAL, "n_cta must lie in [0, 4096]");
        g_opt.n_cta = int(value);
    } else if (!strcmp(key, "sched")) {
        if (value < -1 || value >= kNumSched)
            return fail(XE_EINVAL, "sched must lie in [-1, %d]", kNumSched - 1);
        g_opt.sched = int(value);
    } else if (!strcmp(key, "tile_n")) {
        if (value != 0 && value != 128 && value != 256)
            return fail(XE_EINVAL, "tile_n must be 0, 128 or 256");
        g_opt.tile_n = int(value);
    } else if (!strcmp(key, "autotune")) {
        g_opt.autotune = value ? 1 : 0;
    } else if (!strcmp(key, "timing")) {
        g_opt.timing = value ? 1 : 0;
    } else if (!strcmp(key, "inject_stall")) {
        g_opt.inject_stall = value ? 1 : 0;
    } else if (!strcmp(key, "host_chunk_t") || !strcmp(key, "host_async_chunk_t")) {
        if (value != 0 && (value < 64 || value > XE_MAX_T || value % 64 != 0))
            return fail(XE_EINVAL, "%s must be 0 or a multiple of 64 in [64, %lld]", key, (long long)XE_MAX_T);
        (key[5] == 'c' ? g_opt.host_chunk_t : g_opt.host_async_chunk_t) = value;
    } else if (!strcmp(key, "count_weight")) {
        if (value < 1 || value > 100) return fail(XE_EINVAL, "count_weight must lie in [1, 100]");
        g_opt.count_weight = int(value);
    } else if (!strcmp(key, "implicit_plans")) {
        g_opt.implicit_plans = value ? 1 : 0;
    } else if (!strcmp(key, "count_launch")) {
        g_opt.count_launch = value ? 1 : 0;
    } else if (!strcmp(key, "checks")) {
        g_opt.checks = value ? 1 : 0;
        if (!g_opt.checks) g_opt.check_corrupt = 0;
    } else if (!strcmp(key, "check_corrupt")) {
        if (value < 0 || value > 2) return fail(XE_EINVAL, "check_corrupt must lie in [0, 2]");
        if (value && !g_opt.checks) return fail(XE_EINVAL, "check_corrupt needs option \"checks\" on");
        g_opt.check_corrupt = int(value);
    } else if (!strcmp(key, "part_overhead")) {
        if (value < 0 || value > 100) return fail(XE_EINVAL, "part_overhead must lie in [0, 100]");
        g_opt.part_overhead = int(value);
    } else {
        return fail(XE_EINVAL, "unknown option '%s'", key);
    }
    return XE_OK;
}

int xe_set_timing(int enable) { return xe_set_option("timing", enable); }

int xe_last_timing(float *stage_ms, float *correlate_ms) {
    return xe_last_timing_counts(stage_ms, correlate_ms, nullptr);
}

int xe_last_timing_counts(float *stage_ms, float *correlate_ms, float *count_ms) {
    if (!g_last_ev[0]) return XE_EAGAIN;
    cudaError_t e = cudaEventSynchronize(g_last_ev[3]);
    if (e != cudaSuccess) return fail(XE_ECUDA, "event sync: %s", cudaGetErrorString(e));
    float a = 0, b = 0, c = 0;
    cudaEventElapsedTime(&a, g_last_ev[0], g_last_ev[1]);
    cudaEventElapsedTime(&b, g_last_ev[1], g_last_ev[2]);
    cudaEventElapsedTime(&c, g_last_ev[2], g_last_ev[3]);
    if (stage_ms) *stage_ms = a;
    if (correlate_ms) *correlate_ms = b;
    if (count_ms) *count_ms = c;
    return XE_OK;
}

int xe_last_config(int *n_cta, int *tile_n, int *sched) {
    if (n_cta) *n_cta = g_last_cfg.n_cta;
    if (tile_n) *tile_n = g_last_cfg.tile_n;
    if (sched) *sched = g_last_cfg.sched;
    return g_last_cfg.sched < 0 ? XE_EAGAIN : XE_OK;
}

static int tune_shapes(const int *N, const int64_t *T, const int *n_chan, int n_jobs, int eb,
                       std::vector<int64_t> *key) {
    if (!N || !T || !n_chan || n_jobs < 1 || n_jobs > kMaxJobs) return fail(XE_EINVAL, "bad batch shape");
    if (eb != 1 && eb != 2) return fail(XE_EINVAL, "operand bytes must be 1 or 2");
    std::vector<JobShape> shapes;
    for (int q = 0; q < n_jobs; ++q) {
        if (N[q] < 1 || N[q] > XE_MAX_N || T[q] < 1 || n_chan[q] < 1) return fail(XE_EINVAL, "bad job %d", q);
        shapes.push_back(JobShape{N[q], std::min<int64_t>(T[q], kExactChunkT), n_chan[q]});
    }
    *key = tune_key(shapes, eb);
    return XE_OK;
}

static int check_gpu_name(const char *gpu, int n_sm) {
    if (!gpu || !*gpu || strlen(gpu) > 200 || n_sm < 1) return fail(XE_EINVAL, "bad GPU name or SM count");
    for (const char *c = gpu; *c; ++c)
        if (*c == ' ' || *c == '\t' || *c == '\n') return fail(XE_EINVAL, "GPU name must not contain blanks");
    return XE_OK;
}

int xe_tune_cache(const char *path) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_tune_env_read = true;                    // an explicit choice overrides XE_TUNE_CACHE
    g_tune_path = path ? path : "";
    if (g_tune_path.empty()) return XE_OK;
    return load_tune_file(g_tune_path);
}

int xe_tune_store(const char *gpu, int n_sm, const int *N, const int64_t *T, const int *n_chan, int n_jobs,
                  int operand_bytes, int n_cta, int tile_n, int sched) {
    int rc = check_gpu_name(gpu, n_sm);
    if (rc) return rc;
    std::vector<int64_t> key;
    rc = tune_shapes(N, T, n_chan, n_jobs, operand_bytes, &key);
    if (rc) return rc;
    const TuneCfg c{n_cta, tile_n, sched};
    if (!valid_cfg(c)) return fail(XE_EINVAL, "bad plan configuration");
    std::lock_guard<std::mutex> lk(g_mu);
    read_tune_env();
    return store_tune(gpu, n_sm, key, c);
}

int xe_tune_lookup(const char *gpu, int n_sm, const int *N, const int64_t *T, const int *n_chan, int n_jobs,
                   int operand_bytes, int *n_cta, int *tile_n, int *sched) {
    int rc = check_gpu_name(gpu, n_sm);
    if (rc) return rc;
    std::vector<int64_t> key;
    rc = tune_shapes(N, T, n_chan, n_jobs, operand_bytes, &key);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    read_tune_env();
    auto it = g_tune_file.find({gpu_id(gpu, n_sm), key});
    if (it == g_tune_file.end()) return fail(XE_EAGAIN, "no tuned configuration for this shape");
    if (n_cta) *n_cta = it->second.n_cta;
    if (tile_n) *tile_n = it->second.tile_n;
    if (sched) *sched = it->second.sched;
    return XE_OK;
}

int xe_runtime_counters(int64_t *out, int n) {
    if (!out || n < 1) return fail(XE_EINVAL, "bad counter query");
    std::lock_guard<std::mutex> lk(g_mu);
    const int64_t v[6] = {g_rc.batches, g_rc.build_ns, g_rc.plans_built, g_rc.plan_ns, g_rc.regrowths, g_rc.trims};
    for (int k = 0; k < n && k < 6; ++k) out[k] = v[k];
    return n < 6 ? n : 6;
}

int xe_tune_stats(int64_t *timed_candidates, int64_t *from_cache) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (timed_candidates) *timed_candidates = g_tune_stats.timed;
    if (from_cache) *from_cache = g_tune_stats.from_file;
    return XE_OK;
}

int xe_correlate_async(const uint8_t *in, int N, int64_t T, int n_chan, int32_t *vis, int algo,
                       void *stream) {
    int rc = check_job(in, N, T, n_chan, vis);
    if (rc) return rc;
    if (algo != XE_ALGO_AUTO && algo != XE_ALGO_TC && algo != XE_ALGO_IMMA)
        return fail(XE_EINVAL, "unknown algo %d", algo);
    xe_job j{in, vis, N, n_chan, T};
    std::lock_guard<std::mutex> lk(g_mu);
    return run_jobs(&j, 1, algo == XE_ALGO_AUTO ? XE_ALGO_TC : algo,
                    reinterpret_cast<cudaStream_t>(stream));
}

int xe_correlate(const uint8_t *in, int N, int64_t T, int n_chan, int32_t *vis) {
    return xe_correlate_async(in, N, T, n_chan, vis, XE_ALGO_AUTO, nullptr);
}

// Enqueue one host-buffer correlation into slot `slot` (the caller holds g_mu): copies of the
// input on the copy stream, chunk by chunk; the correlation on the compute stream, each chunk
// as soon as its bytes have landed (the first chunk overwrites, later ones add: int32 sums of
// exact partial sums are exact); the copy of the result on the device -> host stream.
static int host_enqueue(Device *d, int slot, const uint8_t *host_in, int N, int64_t T, int n_chan,
                        int32_t *host_vis, int algo) {
    HostIO &io = d->io[slot];
    HostStreams &hs = d->hs;
    if (io.in_flight) return fail(XE_EAGAIN, "host slot %d is still in flight: call xe_host_wait first", slot);
    if (!hs.copy) {
        XE_CUDA(cudaStreamCreateWithFlags(&hs.copy, cudaStreamNonBlocking));
        XE_CUDA(cudaStreamCreateWithFlags(&hs.compute, cudaStreamNonBlocking));
        XE_CUDA(cudaStreamCreateWithFlags(&hs.d2h, cudaStreamNonBlocking));
    }
    if (!io.computed) {
        XE_CUDA(cudaEventCreateWithFlags(&io.computed, cudaEventDisableTiming));
        XE_CUDA(cudaEventCreateWithFlags(&io.delivered, cudaEventDisableTiming));
    }
    const size_t in_bytes = size_t(n_chan) * size_t(T) * size_t(N);
    const size_t vis_bytes = size_t(n_chan) * size_t(N) * size_t(N + 1) * sizeof(int32_t);
    int rc = grow(reinterpret_cast<void **>(&io.d_in), &io.in_bytes, in_bytes, false);
    if (rc) return rc;
    rc = grow(reinterpret_cast<void **>(&io.d_vis), &io.vis_bytes, vis_bytes, false);
    if (rc) return rc;
    const int64_t chunk = slot == kHostSlots - 1 ? g_opt.host_chunk_t : g_opt.host_async_chunk_t;
    const int64_t n_chunks = (algo == XE_ALGO_IMMA || chunk == 0 || chunk >= T) ? 1 : (T + chunk - 1) / chunk;
    const int64_t step = n_chunks == 1 ? T : chunk;
    while (int64_t(io.landed.size()) < std::min<int64_t>(n_chunks, 64)) {
        cudaEvent_t e;
        XE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        io.landed.push_back(e);
    }
    const size_t row = size_t(N);
    for (int64_t k = 0; k < n_chunks; ++k) {
        const int64_t t0 = k * step, t1 = std::min(T, t0 + step);
        cudaEvent_t ev = io.landed[size_t(k % int64_t(io.landed.size()))];
        if (k >= int64_t(io.landed.size())) XE_CUDA(cudaEventSynchronize(ev));   // event reuse
        for (int c = 0; c < n_chan; ++c) {
            const size_t off = (size_t(c) * size_t(T) + size_t(t0)) * row;
            XE_CUDA(cudaMemcpyAsync(io.d_in + off, host_in + off, size_t(t1 - t0) * row, cudaMemcpyHostToDevice,
                                    hs.copy));
        }
        XE_CUDA(cudaEventRecord(ev, hs.copy));
        XE_CUDA(cudaStreamWaitEvent(hs.compute, ev, 0));
        if (n_chunks == 1) {
            xe_job j{io.d_in, io.d_vis, N, n_chan, T};
            rc = run_jobs(&j, 1, algo == XE_ALGO_AUTO ? XE_ALGO_TC : algo, hs.compute);
        } else {
            const xe_view view{T * int64_t(N), int64_t(N), int64_t(N), 0};
            xe_job j{io.d_in + size_t(t0) * row, io.d_vis, N, n_chan, t1 - t0};
            g_job_view = &view;
            rc = run_jobs(&j, 1, XE_ALGO_TC, hs.compute, k > 0 ? 1 : 0);
            g_job_view = nullptr;
        }
        if (rc) return rc;
    }
    XE_CUDA(cudaEventRecord(io.computed, hs.compute));
    XE_CUDA(cudaStreamWaitEvent(hs.d2h, io.computed, 0));
    XE_CUDA(cudaMemcpyAsync(host_vis, io.d_vis, vis_bytes, cudaMemcpyDeviceToHost, hs.d2h));
    XE_CUDA(cudaEventRecord(io.delivered, hs.d2h));
    io.in_flight = true;
    return XE_OK;
}

// Wait for slot `slot`'s result (the caller holds g_mu); reports a device-side timeout.
static int host_finish(Device *d, int slot) {
    HostIO &io = d->io[slot];
    if (!io.in_flight) return XE_OK;
    io.in_flight = false;
    XE_CUDA(cudaEventSynchronize(io.delivered));
    auto it = d->scratch.find(d->hs.compute);
    if (it != d->scratch.end()) {
        int st = 0;
        XE_CUDA(cudaMemcpy(&st, it->second->status, sizeof(int), cudaMemcpyDeviceToHost));
        if (st != 0) {
            XE_CUDA(cudaMemset(it->second->status, 0, sizeof(int)));
            if (it->second->counters) XE_CUDA(cudaMemset(it->second->counters, 0, it->second->counters_bytes));
            XE_CUDA(cudaStreamSynchronize(0));
            return status_error(st);
        }
    }
    return XE_OK;
}

static int check_host_call(const uint8_t *host_in, int N, int64_t T, int n_chan, const int32_t *host_vis, int algo) {
    int rc = check_job(host_in, N, T, n_chan, host_vis);
    if (rc) return rc;
    if (algo != XE_ALGO_AUTO && algo != XE_ALGO_TC && algo != XE_ALGO_IMMA)
        return fail(XE_EINVAL, "unknown algo %d", algo);
    return XE_OK;
}

int xe_correlate_host(const uint8_t *host_in, int N, int64_t T, int n_chan, int32_t *host_vis,
                      int algo) {
    int rc = check_host_call(host_in, N, T, n_chan, host_vis, algo);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    Device *d = nullptr;
    rc = get_device(&d);
    if (rc) return rc;
    rc = host_enqueue(d, kHostSlots - 1, host_in, N, T, n_chan, host_vis, algo);
    const int rc2 = host_finish(d, kHostSlots - 1);
    return rc ? rc : rc2;
}

int xe_correlate_host_async(const uint8_t *host_in, int N, int64_t T, int n_chan, int32_t *host_vis, int slot) {
    int rc = check_host_call(host_in, N, T, n_chan, host_vis, XE_ALGO_TC);
    if (rc) return rc;
    if (slot < 0 || slot >= XE_HOST_SLOTS) return fail(XE_EINVAL, "slot %d outside [0, %d)", slot, XE_HOST_SLOTS);
    std::lock_guard<std::mutex> lk(g_mu);
    Device *d = nullptr;
    rc = get_device(&d);
    if (rc) return rc;
    return host_enqueue(d, slot, host_in, N, T, n_chan, host_vis, XE_ALGO_TC);
}

int xe_host_wait(int slot) {
    if (slot < 0 || slot >= XE_HOST_SLOTS) return fail(XE_EINVAL, "slot %d outside [0, %d)", slot, XE_HOST_SLOTS);
    std::lock_guard<std::mutex> lk(g_mu);
    Device *d = nullptr;
    int rc = get_device(&d);
    if (rc) return rc;
    return host_finish(d, slot);
}

int xe_correlate_batch(const xe_job *jobs, int n_jobs, int use_graph, void *stream) {
    if (!jobs || n_jobs < 1) return fail(XE_EINVAL, "empty batch");
    for (int q = 0; q < n_jobs; ++q) {
        int rc = check_job(jobs[q].in, jobs[q].N, jobs[q].T, jobs[q].n_chan, jobs[q].vis);
        if (rc) return rc;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    return run_jobs(jobs, n_jobs, XE_ALGO_TC, reinterpret_cast<cudaStream_t>(stream), 0, use_graph);
}

int xe_correlate_accumulate(const xe_job *jobs, int n_jobs, void *stream) {
    if (!jobs || n_jobs < 1) return fail(XE_EINVAL, "empty batch");
    for (int q = 0; q < n_jobs; ++q) {
        int rc = check_job(jobs[q].in, jobs[q].N, jobs[q].T, jobs[q].n_chan, jobs[q].vis);
        if (rc) return rc;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    return run_jobs(jobs, n_jobs, XE_ALGO_TC, reinterpret_cast<cudaStream_t>(stream), 1, 0);
}

int xe_correlate_masked_batch(const xe_masked_job *jobs, int n_jobs, void *stream) {
    if (!jobs || n_jobs < 1) return fail(XE_EINVAL, "empty batch");
    std::vector<xe_job> plain(static_cast<size_t>(n_jobs));
    std::vector<int> acc(static_cast<size_t>(n_jobs));
    for (int q = 0; q < n_jobs; ++q) {
        const xe_masked_job &m = jobs[q];
        int rc = check_job(m.in, m.N, m.T, m.n_chan, m.vis);
        if (rc) return rc;
        if (m.encoding != XE_ENC_TWOS && m.encoding != XE_ENC_OFFSET)
            return fail(XE_EINVAL, "job %d: unknown encoding %d", q, m.encoding);
        if (m.counts && (reinterpret_cast<uintptr_t>(m.counts) & 3))
            return fail(XE_EINVAL, "job %d: counts must be 4-byte aligned", q);
        plain[size_t(q)] = xe_job{m.in, m.vis, m.N, m.n_chan, m.T};
        acc[size_t(q)] = m.accumulate ? 1 : 0;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_job_mask = jobs;
    g_job_acc = acc.data();
    const int rc = run_jobs(plain.data(), n_jobs, XE_ALGO_TC, reinterpret_cast<cudaStream_t>(stream), 0, 0);
    g_job_acc = nullptr;
    g_job_mask = nullptr;
    return rc;
}

int xe_beamform(const uint8_t *in, int N, int64_t T, int n_chan, const int8_t *weights, int n_beams,
                int32_t *beams, void *stream) {
    if (!in || !weights || !beams) return fail(XE_EINVAL, "null input, weight or beam pointer");
    if (N < 1 || N > XE_MAX_N) return fail(XE_EINVAL, "N=%d outside [1, %d]", N, XE_MAX_N);
    if (T < 1) return fail(XE_EINVAL, "T=%lld < 1", (long long)T);
    if (n_chan < 1) return fail(XE_EINVAL, "n_chan=%d < 1", n_chan);
    if (n_beams < 1 || n_beams > kBeamMaxBeams)
        return fail(XE_EINVAL, "n_beams=%d outside [1, %d]", n_beams, kBeamMaxBeams);
    if (reinterpret_cast<uintptr_t>(beams) & 3) return fail(XE_EINVAL, "beams must be 4-byte aligned");
    if (int64_t(n_chan) * ((T + kBeamRows - 1) / kBeamRows) > 0x7fffffffLL)
        return fail(XE_EINVAL, "too many sample tiles");
    std::lock_guard<std::mutex> lk(g_mu);
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Device *d = nullptr;
    int rc = get_device(&d);
    if (rc) return rc;
    Scratch *sc = nullptr;
    rc = get_scratch(d, s, &sc);
    if (rc) return rc;
    // Beams in groups of at most kBeamMaxPerLaunch (4 MMA columns each); every group is one
    // weight preparation and one launch over all inputs (exact in one f32 accumulation).
    const int group = std::min(n_beams, kBeamMaxPerLaunch);
    rc = grow(reinterpret_cast<void **>(&sc->beam_wt), &sc->beam_wt_bytes, beam_wt_bytes(group, N), false);
    if (rc) return rc;
    const bool timing = g_opt.timing != 0;
    const int n_chunks = (N + kBeamChunk - 1) / kBeamChunk;
    for (int b0 = 0; b0 < n_beams; b0 += group) {
        const int nb = std::min(group, n_beams - b0);
        const int ncols = beam_ncols(nb);
        if (timing && b0 == 0) XE_CUDA(cudaEventRecord(sc->ev[0], s));
        XE_CUDA(launch_beam_weights(weights, b0, nb, N, ncols, sc->beam_wt, s));
        if (timing && b0 == 0) XE_CUDA(cudaEventRecord(sc->ev[1], s));
        BeamDev bd{};
        bd.in = in;
        bd.wt = sc->beam_wt;
        bd.y = beams;
        bd.status = sc->status;
        bd.T = T;
        bd.N = N;
        bd.C = n_chan;
        bd.B_total = n_beams;
        bd.b0 = b0;
        bd.B = nb;
        bd.ncols = ncols;
        bd.k_lo = 0;
        bd.k_hi = n_chunks;
        XE_CUDA(launch_beam(bd, s));
    }
    if (timing) {
        XE_CUDA(cudaEventRecord(sc->ev[2], s));
        XE_CUDA(cudaEventRecord(sc->ev[3], s));
        for (int k = 0; k < 4; ++k) g_last_ev[k] = sc->ev[k];
    }
    return XE_OK;
}

int xe_corner_turn(const uint8_t *bundles, int n_cyl, int n_freq, int n_in, int64_t T, uint8_t *frames,
                   int32_t *presums, void *stream) {
    if (!bundles || !frames) return fail(XE_EINVAL, "null bundle or frame pointer");
    if (n_cyl < 1 || n_freq < 1 || n_in < 1 || T < 1 || int64_t(n_cyl) * n_in > XE_MAX_N)
        return fail(XE_EINVAL, "bad bundle shape");
    if (T > XE_MAX_T) return fail(XE_EOVERFLOW, "T=%lld > %lld: pre-sums could overflow int32", (long long)T,
                                  (long long)XE_MAX_T);
    if (presums && (reinterpret_cast<uintptr_t>(presums) & 3)) return fail(XE_EINVAL, "presums must be 4-byte aligned");
    std::lock_guard<std::mutex> lk(g_mu);
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Device *d = nullptr;
    int rc = get_device(&d);
    if (rc) return rc;
    Scratch *sc = nullptr;
    rc = get_scratch(d, s, &sc);
    if (rc) return rc;
    if (presums) {
        rc = grow(reinterpret_cast<void **>(&sc->corner_partial), &sc->corner_partial_bytes,
                  size_t(corner_partial_elems(n_cyl, n_freq, n_in, T)) * sizeof(int32_t), false);
        if (rc) return rc;
    }
    const bool timing = g_opt.timing != 0;
    if (timing) XE_CUDA(cudaEventRecord(sc->ev[0], s));
    if (timing) XE_CUDA(cudaEventRecord(sc->ev[1], s));
    XE_CUDA(launch_corner_turn(bundles, n_cyl, n_freq, n_in, T, frames, sc->corner_partial, presums, s));
    if (timing) {
        XE_CUDA(cudaEventRecord(sc->ev[2], s));
        XE_CUDA(cudaEventRecord(sc->ev[3], s));
        for (int k = 0; k < 4; ++k) g_last_ev[k] = sc->ev[k];
    }
    return XE_OK;
}

int xe_bundle_view(int n_cyl, int n_freq, int n_in, int64_t T, xe_view *view) {
    if (!view) return fail(XE_EINVAL, "null view");
    if (n_cyl < 1 || n_freq < 1 || n_in < 1 || T < 1 || int64_t(n_cyl) * n_in > XE_MAX_N)
        return fail(XE_EINVAL, "bad bundle shape");
    view->chan_stride = n_in;
    view->time_stride = int64_t(n_freq) * n_in;
    view->seg_inputs = n_in;
    view->seg_stride = T * n_freq * int64_t(n_in);
    return XE_OK;
}

int xe_correlate_view(const uint8_t *in, const xe_view *view, int N, int64_t T, int n_chan, int32_t *vis,
                      void *stream) {
    int rc = check_job(in, N, T, n_chan, vis);
    if (rc) return rc;
    if (!view) return fail(XE_EINVAL, "null view");
    if (view->seg_inputs < 1 || view->seg_inputs > XE_MAX_N || view->chan_stride < 0 || view->time_stride < 0 ||
        view->seg_stride < 0)
        return fail(XE_EINVAL, "bad view: seg_inputs must lie in [1, %d] and strides be >= 0", XE_MAX_N);
    xe_job j{in, vis, N, n_chan, T};
    std::lock_guard<std::mutex> lk(g_mu);
    g_job_view = view;
    rc = run_jobs(&j, 1, XE_ALGO_TC, reinterpret_cast<cudaStream_t>(stream));
    g_job_view = nullptr;
    return rc;
}

int xe_correlate_masked(const uint8_t *in, const uint8_t *flags, int N, int64_t T, int n_chan,
                        int encoding, int32_t *vis, int32_t *counts, int accumulate, void *stream) {
    xe_masked_job j{in, flags, vis, counts, N, n_chan, T, encoding, accumulate};
    return xe_correlate_masked_batch(&j, 1, stream);
}

int xe_plan_stats(const int *N, const int64_t *T, const int *n_chan, int n_jobs, int n_cta,
                  int64_t *n_tiles, int64_t *n_iters, int64_t *n_split_tiles) {
    std::lock_guard<std::mutex> lk(g_mu);      // the planner reads the options
    HostPlan p;
    int rc = plan_from_args(N, T, n_chan, n_jobs, n_cta, -1, 0, p);
    if (rc) return rc;
    int64_t split = 0;
    for (const Tile &t : p.tiles) split += t.n_parts > 0 ? 1 : 0;
    if (n_tiles) *n_tiles = int64_t(p.tiles.size());
    if (n_iters) *n_iters = p.total_iters;
    if (n_split_tiles) *n_split_tiles = split;
    return XE_OK;
}

int64_t xe_plan_dump(const int *N, const int64_t *T, const int *n_chan, int n_jobs, int n_cta,
                     int sched, int tile_n, int32_t *out, int64_t cap) {
    std::lock_guard<std::mutex> lk(g_mu);      // the planner reads the options
    HostPlan p;
    int rc = plan_from_args(N, T, n_chan, n_jobs, n_cta, sched, tile_n, p);
    if (rc) return rc;
    const int64_t need = 4 + 6 * int64_t(p.tiles.size()) + 5 * int64_t(p.segs.size());
    if (!out || cap < need) return need;
    int64_t k = 0;
    out[k++] = int32_t(p.tiles.size());
    out[k++] = int32_t(p.segs.size());
    out[k++] = p.n_cta;
    out[k++] = p.n_partial;
    for (const Tile &t : p.tiles) {
        out[k++] = t.job;
        out[k++] = t.chan;
        out[k++] = t.i0;
        out[k++] = t.j0;
        out[k++] = t.nj;
        out[k++] = t.kblocks;
    }
    for (int b = 0; b < p.n_cta; ++b)
        for (int q = p.seg_off[size_t(b)]; q < p.seg_off[size_t(b) + 1]; ++q) {
            const Seg &s = p.segs[size_t(q)];
            out[k++] = b;
            out[k++] = s.tile;
            out[k++] = s.k_lo;
            out[k++] = s.k_hi;
            out[k++] = s.slot;
        }
    return need;
}

// Read and clear the device status word of the scratch bound to `stream` (synchronises it).
int xe_device_status(void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    Device *d = nullptr;
    int rc = get_device(&d);
    if (rc) return rc;
    auto it = d->scratch.find(reinterpret_cast<cudaStream_t>(stream));
    if (it == d->scratch.end()) return XE_OK;
    int st = 0;
    XE_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    XE_CUDA(cudaMemcpy(&st, it->second->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        XE_CUDA(cudaMemset(it->second->status, 0, sizeof(int)));
        if (it->second->counters)
            XE_CUDA(cudaMemset(it->second->counters, 0, it->second->counters_bytes));
        XE_CUDA(cudaStreamSynchronize(0));
        return status_error(st);
    }
    return XE_OK;
}

int xe_release_stream(void *stream) { return release_stream_scratch(reinterpret_cast<cudaStream_t>(stream)); }

uint32_t xe_debug_operand_code(int v, int elem_bytes) { return operand_code(v, elem_bytes); }

int xe_device_info(int *n_sm) {
    std::lock_guard<std::mutex> lk(g_mu);
    Device *d = nullptr;
    int rc = get_device(&d);
    if (rc) return rc;
    if (n_sm) *n_sm = d->n_sm;
    return XE_OK;
}

}  // extern "C"
