// xe_api.cu -- host runtime behind the C ABI of include/xe.h: argument checks, the
// triangle-tile plan of the persistent stream-K scheduler, per-stream scratch memory,
// the exact-chunk split of long integrations, CUDA-graph replay of batches, and timing.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "xe.h"
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
    int timing = 0;
};
static Options g_opt;
static std::mutex g_mu;

// ---- plans ---------------------------------------------------------------------------

struct JobShape {
    int N;
    int64_t T;
    int C;
};

struct HostPlan {
    std::vector<Tile> tiles;
    int64_t total_iters = 0;
    int n_cta = 0;
    int64_t n_split = 0;
};

static int n_pad_of(int N) { return (N + kNPad - 1) / kNPad * kNPad; }

static int64_t kblocks_of(int64_t T, int eb) {
    const int ks = samples_per_stage(eb);
    return (T + ks - 1) / ks;
}

// Triangle tiles of one job: row blocks of 128 inputs; for each, column tiles of 256 inputs
// aligned to 256, except a 128-wide half tile when the row block starts in the middle of a
// 256-aligned column block.  Together they cover every (i, j >= i) exactly once.
static void build_tiles(const std::vector<JobShape> &jobs, int eb, int n_sm, HostPlan &p) {
    p.tiles.clear();
    int64_t it = 0;
    for (int q = 0; q < int(jobs.size()); ++q) {
        const JobShape &js = jobs[q];
        const int kb = int(kblocks_of(js.T, eb));
        for (int c = 0; c < js.C; ++c) {
            for (int i0 = 0; i0 < js.N; i0 += kBM) {
                int j0 = i0;
                if (j0 % kBN != 0) {
                    p.tiles.push_back(Tile{q, c, i0, j0, kBM, kb, it});
                    it += kb;
                    j0 += kBM;
                }
                for (; j0 < js.N; j0 += kBN) {
                    p.tiles.push_back(Tile{q, c, i0, j0, kBN, kb, it});
                    it += kb;
                }
            }
        }
    }
    p.total_iters = it;
    int64_t g = n_sm;
    if (g > it) g = it;
    if (g < 1) g = 1;
    p.n_cta = int(g);
    // Tiles whose iterations are split across CTA ranges.
    p.n_split = 0;
    for (const Tile &t : p.tiles) {
        const int64_t b0 = ((t.iter_begin + 1) * g - 1) / it;
        const int64_t b1 = ((t.iter_begin + t.kblocks) * g - 1) / it;
        p.n_split += (b0 != b1) ? 1 : 0;
    }
}

struct DevPlan {
    HostPlan host;
    Tile *d_tiles = nullptr;
};

struct Scratch {
    uint8_t *planes = nullptr;
    size_t planes_bytes = 0;
    int32_t *ws = nullptr;
    size_t ws_bytes = 0;
    int *counters = nullptr;
    size_t n_counters = 0;
    int *status = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
};

struct HostIO {
    cudaStream_t stream = nullptr;
    uint8_t *d_in = nullptr;
    size_t in_bytes = 0;
    int32_t *d_vis = nullptr;
    size_t vis_bytes = 0;
};

struct Device {
    int id = -1;
    int n_sm = 0;
    HostIO io;
    std::map<std::vector<int64_t>, DevPlan *> plans;
    std::map<cudaStream_t, Scratch *> scratch;
};

static std::map<int, Device *> g_devs;

static int get_device(Device **out) {
    int dev = 0;
    XE_CUDA(cudaGetDevice(&dev));
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
    g_devs[dev] = d;
    *out = d;
    return XE_OK;
}

static int get_plan(Device *d, const std::vector<JobShape> &jobs, int eb, DevPlan **out) {
    const int n_sm = g_opt.n_cta > 0 ? g_opt.n_cta : d->n_sm;
    std::vector<int64_t> key{eb, n_sm};
    for (const JobShape &j : jobs) {
        key.push_back(j.N);
        key.push_back(j.T);
        key.push_back(j.C);
    }
    auto it = d->plans.find(key);
    if (it != d->plans.end()) {
        *out = it->second;
        return XE_OK;
    }
    DevPlan *p = new DevPlan;
    build_tiles(jobs, eb, n_sm, p->host);
    if (p->host.tiles.size() > size_t(0x7fffffff)) {
        delete p;
        return fail(XE_EINVAL, "too many tiles");
    }
    const size_t bytes = p->host.tiles.size() * sizeof(Tile);
    if (cudaMalloc(&p->d_tiles, bytes) != cudaSuccess) {
        delete p;
        return fail(XE_ENOMEM, "cannot allocate %zu bytes for the tile plan", bytes);
    }
    cudaError_t e = cudaMemcpy(p->d_tiles, p->host.tiles.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->d_tiles);
        delete p;
        return fail(XE_ECUDA, "plan upload failed: %s", cudaGetErrorString(e));
    }
    d->plans[key] = p;
    *out = p;
    return XE_OK;
}

static int grow(void **ptr, size_t *have, size_t need, bool zero) {
    if (*have >= need && *ptr) return XE_OK;
    if (*ptr) {
        cudaError_t e = cudaDeviceSynchronize();  // nothing may still use the old buffer
        if (e != cudaSuccess) return fail(XE_ECUDA, "sync before regrow: %s", cudaGetErrorString(e));
        cudaFree(*ptr);
        *ptr = nullptr;
        *have = 0;
    }
    size_t sz = need + need / 8;
    if (cudaMalloc(ptr, sz) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(XE_ENOMEM, "cannot allocate %zu bytes of scratch", sz);
    }
    if (zero) XE_CUDA(cudaMemset(*ptr, 0, sz));
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
    for (auto &e : sc->ev) XE_CUDA(cudaEventCreate(&e));
    d->scratch[s] = sc;
    *out = sc;
    return XE_OK;
}

static thread_local cudaEvent_t g_last_ev[3] = {nullptr, nullptr, nullptr};

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

// Enqueue a batch of jobs (all validated) on stream s with the given algorithm.
static int run_jobs(const xe_job *jobs, int n_jobs, int algo, cudaStream_t s, int accumulate = 0) {
    Device *d = nullptr;
    int rc = get_device(&d);
    if (rc) return rc;
    Scratch *sc = nullptr;
    rc = get_scratch(d, s, &sc);
    if (rc) return rc;
    const bool timing = g_opt.timing != 0;
    if (timing) XE_CUDA(cudaEventRecord(sc->ev[0], s));

    if (algo == XE_ALGO_IMMA) {
        for (int g0 = 0; g0 < n_jobs; g0 += kMaxJobs) {
            const int ng = n_jobs - g0 < kMaxJobs ? n_jobs - g0 : kMaxJobs;
            JobTable jt{};
            jt.n_jobs = ng;
            jt.accumulate = accumulate ? 1 : 0;
            int64_t blocks = 0;
            for (int q = 0; q < ng; ++q) {
                const xe_job &j = jobs[g0 + q];
                JobDev &jd = jt.jobs[q];
                jd.in = j.in;
                jd.vis = j.vis;
                jd.T = j.T;
                jd.t0 = 0;
                jd.T_in = j.T;
                jd.N = j.N;
                jd.C = j.n_chan;
                jd.vis_chan_elems = int64_t(j.N) * (j.N + 1);
                jd.stage_block0 = blocks;
                blocks += imma_blocks(j.N, j.n_chan);
            }
            jt.total_stage_blocks = blocks;
            XE_CUDA(launch_imma(jt, s));
        }
        if (timing) {
            XE_CUDA(cudaEventRecord(sc->ev[1], s));
            XE_CUDA(cudaEventRecord(sc->ev[2], s));
        }
    } else {
        const int eb = g_opt.operand_bytes;
        const int64_t wt = g_opt.exact_chunk_t / samples_per_stage(eb) * samples_per_stage(eb);
        int64_t max_T = 0;
        for (int q = 0; q < n_jobs; ++q) max_T = jobs[q].T > max_T ? jobs[q].T : max_T;
        const int64_t n_win = (max_T + wt - 1) / wt;
        bool stage_marked = false;
        for (int64_t w = 0; w < n_win; ++w) {
            // Jobs that still have samples in window w, in groups of kMaxJobs.
            std::vector<int> act;
            for (int q = 0; q < n_jobs; ++q)
                if (jobs[q].T > w * wt) act.push_back(q);
            for (size_t g0 = 0; g0 < act.size(); g0 += kMaxJobs) {
                const int ng = int(act.size() - g0 < size_t(kMaxJobs) ? act.size() - g0 : kMaxJobs);
                std::vector<JobShape> shapes;
                JobTable jt{};
                jt.n_jobs = ng;
                jt.accumulate = (w > 0 || accumulate) ? 1 : 0;
                size_t plane_off = 0;
                int64_t blocks = 0;
                for (int k = 0; k < ng; ++k) {
                    const xe_job &j = jobs[act[g0 + k]];
                    const int64_t Tw = (j.T - w * wt) < wt ? (j.T - w * wt) : wt;
                    shapes.push_back(JobShape{j.N, Tw, j.n_chan});
                    JobDev &jd = jt.jobs[k];
                    jd.in = j.in;
                    jd.vis = j.vis;
                    jd.T = Tw;
                    jd.t0 = w * wt;
                    jd.T_in = j.T;
                    jd.N = j.N;
                    jd.n_pad = n_pad_of(j.N);
                    jd.C = j.n_chan;
                    jd.kblocks = int(kblocks_of(Tw, eb));
                    jd.plane_chan_bytes = int64_t(jd.kblocks) * 2 * jd.n_pad * kRowBytes;
                    jd.vis_chan_elems = int64_t(j.N) * (j.N + 1);
                    jd.stage_block0 = blocks;
                    blocks += int64_t(j.n_chan) * jd.kblocks * (jd.n_pad / 256);
                    plane_off += size_t(jd.plane_chan_bytes) * j.n_chan;
                }
                jt.total_stage_blocks = blocks;
                rc = grow(reinterpret_cast<void **>(&sc->planes), &sc->planes_bytes, plane_off, false);
                if (rc) return rc;
                size_t off = 0;
                for (int k = 0; k < ng; ++k) {
                    jt.jobs[k].planes = sc->planes + off;
                    off += size_t(jt.jobs[k].plane_chan_bytes) * jt.jobs[k].C;
                }
                DevPlan *p = nullptr;
                rc = get_plan(d, shapes, eb, &p);
                if (rc) return rc;
                const size_t ws_need = size_t(2) * p->host.n_cta * kWsSlotElems * sizeof(int32_t);
                rc = grow(reinterpret_cast<void **>(&sc->ws), &sc->ws_bytes, ws_need, false);
                if (rc) return rc;
                size_t cnt_have = sc->n_counters * sizeof(int);
                rc = grow(reinterpret_cast<void **>(&sc->counters), &cnt_have,
                          p->host.tiles.size() * sizeof(int), true);
                if (rc) return rc;
                sc->n_counters = cnt_have / sizeof(int);

                PlanDev pd{};
                pd.tiles = p->d_tiles;
                pd.n_tiles = int(p->host.tiles.size());
                pd.n_cta = p->host.n_cta;
                pd.total_iters = p->host.total_iters;
                pd.ws = sc->ws;
                pd.counters = sc->counters;
                pd.status = sc->status;
                XE_CUDA(launch_stage(jt, eb, s));
                if (timing && !stage_marked) {
                    XE_CUDA(cudaEventRecord(sc->ev[1], s));
                    stage_marked = true;
                }
                XE_CUDA(launch_tc(jt, pd, eb, s));
            }
        }
        if (timing) XE_CUDA(cudaEventRecord(sc->ev[2], s));
    }
    if (timing) {
        for (int k = 0; k < 3; ++k) g_last_ev[k] = sc->ev[k];
    }
    return XE_OK;
}

int run_jobs_accumulate(const xe_job *jobs, int n_jobs, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g_mu);
    return run_jobs(jobs, n_jobs, XE_ALGO_TC, s, 1);
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
    } else if (!strcmp(key, "timing")) {
        g_opt.timing = value ? 1 : 0;
    } else {
        return fail(XE_EINVAL, "unknown option '%s'", key);
    }
    return XE_OK;
}

int xe_set_timing(int enable) { return xe_set_option("timing", enable); }

int xe_last_timing(float *stage_ms, float *correlate_ms) {
    if (!g_last_ev[0]) return XE_EAGAIN;
    cudaError_t e = cudaEventSynchronize(g_last_ev[2]);
    if (e != cudaSuccess) return fail(XE_ECUDA, "event sync: %s", cudaGetErrorString(e));
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, g_last_ev[0], g_last_ev[1]);
    cudaEventElapsedTime(&b, g_last_ev[1], g_last_ev[2]);
    if (stage_ms) *stage_ms = a;
    if (correlate_ms) *correlate_ms = b;
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

int xe_correlate_host(const uint8_t *host_in, int N, int64_t T, int n_chan, int32_t *host_vis,
                      int algo) {
    int rc = check_job(host_in, N, T, n_chan, host_vis);
    if (rc) return rc;
    if (algo != XE_ALGO_AUTO && algo != XE_ALGO_TC && algo != XE_ALGO_IMMA)
        return fail(XE_EINVAL, "unknown algo %d", algo);
    std::lock_guard<std::mutex> lk(g_mu);
    Device *d = nullptr;
    rc = get_device(&d);
    if (rc) return rc;
    HostIO &io = d->io;
    if (!io.stream) XE_CUDA(cudaStreamCreateWithFlags(&io.stream, cudaStreamNonBlocking));
    const size_t in_bytes = size_t(n_chan) * size_t(T) * size_t(N);
    const size_t vis_bytes = size_t(n_chan) * size_t(N) * size_t(N + 1) * sizeof(int32_t);
    rc = grow(reinterpret_cast<void **>(&io.d_in), &io.in_bytes, in_bytes, false);
    if (rc) return rc;
    rc = grow(reinterpret_cast<void **>(&io.d_vis), &io.vis_bytes, vis_bytes, false);
    if (rc) return rc;
    XE_CUDA(cudaMemcpyAsync(io.d_in, host_in, in_bytes, cudaMemcpyHostToDevice, io.stream));
    xe_job j{io.d_in, io.d_vis, N, n_chan, T};
    rc = run_jobs(&j, 1, algo == XE_ALGO_AUTO ? XE_ALGO_TC : algo, io.stream);
    if (rc) return rc;
    XE_CUDA(cudaMemcpyAsync(host_vis, io.d_vis, vis_bytes, cudaMemcpyDeviceToHost, io.stream));
    XE_CUDA(cudaStreamSynchronize(io.stream));
    return XE_OK;
}

int xe_correlate_batch(const xe_job *jobs, int n_jobs, int use_graph, void *stream) {
    (void)use_graph;
    if (!jobs || n_jobs < 1) return fail(XE_EINVAL, "empty batch");
    for (int q = 0; q < n_jobs; ++q) {
        int rc = check_job(jobs[q].in, jobs[q].N, jobs[q].T, jobs[q].n_chan, jobs[q].vis);
        if (rc) return rc;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    return run_jobs(jobs, n_jobs, XE_ALGO_TC, reinterpret_cast<cudaStream_t>(stream));
}

int xe_plan_stats(const int *N, const int64_t *T, const int *n_chan, int n_jobs, int n_cta,
                  int64_t *n_tiles, int64_t *n_iters, int64_t *n_split_tiles) {
    if (!N || !T || !n_chan || n_jobs < 1 || n_cta < 1) return fail(XE_EINVAL, "bad plan query");
    std::vector<JobShape> shapes;
    for (int q = 0; q < n_jobs; ++q) {
        if (N[q] < 1 || T[q] < 1 || n_chan[q] < 1) return fail(XE_EINVAL, "bad job %d", q);
        shapes.push_back(JobShape{N[q], T[q], n_chan[q]});
    }
    HostPlan p;
    build_tiles(shapes, g_opt.operand_bytes, n_cta, p);
    if (n_tiles) *n_tiles = int64_t(p.tiles.size());
    if (n_iters) *n_iters = p.total_iters;
    if (n_split_tiles) *n_split_tiles = p.n_split;
    return XE_OK;
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
            XE_CUDA(cudaMemset(it->second->counters, 0, it->second->n_counters * sizeof(int)));
        return fail(XE_ETIMEOUT, "device wait timed out (status %d)", st);
    }
    return XE_OK;
}

uint32_t xe_debug_operand_code(int v, int elem_bytes) { return operand_code(v, elem_bytes); }

}  // extern "C"
