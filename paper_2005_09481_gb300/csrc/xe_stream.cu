// xe_stream.cu -- the streaming X-engine server: frames in, integrated visibilities out.
//
// The CHIME X-engine integrates visibilities on the GPU and exports them at a fixed cadence
// (Denman et al. 2020, sections 2.1 and 3.1: per-block GPU processing, time integration,
// export of correlated visibilities, Table tab:data-flow).  Here each admitted channel owns
// two device-resident int32 accumulators (one filling, one being exported) and a ring of
// device frame slots.  Producers push frames (host or device memory).  One scheduler thread
// gathers, every pass, the next in-order ready frame of every channel and correlates all of
// them in batched persistent launches that ADD into the accumulators (continuous batching:
// frames that arrive while a batch runs join the next one).  When a channel's integration is
// complete, the channel switches to its other accumulator and the finished one is copied to
// a pinned host buffer on a separate copy stream (overlapping the next batches), cleared,
// and handed to xe_stream_poll with its arrival and ready times (frame-to-visibility latency).
//
// Admission is by HBM budget: a channel is admitted only if its accumulators, frame ring and
// share of staging memory fit the stream's budget.  Lost frames (sequence gaps) are counted
// and mark their integration incomplete; nothing shifts integration boundaries.
//
// Checkpoints: xe_stream_snapshot copies a channel's open integration (its sums so far and
// the frame count they cover) to the host; xe_stream_restore loads such a copy into a newly
// admitted channel of another stream, which then continues the integration from the next
// frame.  The paper's nodes are diskless and keep no such state; this is for a server that
// is restarted or moves a channel between GPUs.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <time.h>

#include <cuda_runtime.h>

#include "xe.h"
#include "xe_host.h"
#include "xe_internal.h"

namespace xe {
namespace {

int64_t now_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return int64_t(ts.tv_sec) * 1000000000LL + ts.tv_nsec;
}

enum SlotState { kFree = 0, kCopying = 1, kReady = 2, kQueued = 3 };

struct Slot {
    uint8_t *dev = nullptr;
    cudaEvent_t copy_ev = nullptr;   // the frame's bytes have landed in the slot
    int pass_ev = -1;                // index of the event of the pass that read the slot
    int state = kFree;
};

struct Entry {          // one frame of a channel, in sequence order
    int64_t seq;
    int slot;           // -1: the frame was lost
    int64_t t_arrival;
};

struct Chan {
    bool admitted = false;
    int32_t *acc[2] = {nullptr, nullptr};
    cudaEvent_t acc_free_ev[2] = {nullptr, nullptr};  // export of that accumulator done
    bool acc_wait[2] = {false, false};                // compute must wait on acc_free_ev
    bool fresh[2] = {true, true};                     // next frame overwrites (no stale sums)
    int cur = 0;                                      // accumulator being filled
    uint8_t *ring_base = nullptr;                     // ring slots, contiguous: slot k at
                                                      // ring_base + k * frame_bytes
    int next_slot = 0;                                // slots are filled round-robin
    std::vector<Slot> ring;
    std::deque<Entry> fifo;
    int n_copying = 0;
    int64_t expected_push = 0;     // next sequence number a push may carry
    int64_t integ_index = 0;
    int64_t frames_in_integ = 0;
    int64_t samples_in_integ = 0;
    int64_t t_first = 0, t_last = 0;
    bool lost = false;
    std::vector<int> bufs;         // result buffers owned by this channel (indices)
};

struct ResultBuf {
    int32_t *host = nullptr;
    int chan = -1;
    bool busy = false;             // between export and xe_stream_release
};

struct Pending {
    xe_result r;
    cudaEvent_t ev;
};

struct PassEvent {
    cudaEvent_t ev = nullptr;
    int refs = 0;
};

// A checkpoint request, filled in by the scheduler thread between passes.
struct SnapReq {
    int chan = -1;
    int state = 0;            // 0 asked, 1 served (copy enqueued), 2 channel gone
    bool zero = false;        // the open integration holds no sums yet
    xe_snapshot info{};
};

}  // namespace
}  // namespace xe

struct xe_stream {
    xe_stream_cfg cfg{};
    int dev = 0;
    int64_t B = 0;
    size_t frame_bytes = 0, acc_bytes = 0, per_chan_bytes = 0;
    int64_t frames_per_integ = 0;
    cudaStream_t copy_s = nullptr, comp_s = nullptr, d2h_s = nullptr;
    std::vector<xe::Chan> chans;
    std::vector<xe::ResultBuf> bufs;
    std::deque<xe::Pending> pending;
    std::deque<xe_result> ready;
    std::vector<cudaEvent_t> spare_events;
    std::vector<xe::PassEvent> pass_events;
    std::vector<int> queued_slots;   // (chan << 8 | slot) of slots read by launched passes
    std::mutex mu;
    std::condition_variable cv_work, cv_ready;
    std::thread sched;
    std::atomic<bool> stop{false};
    bool closed = false;
    int64_t used_bytes = 0;
    int64_t n_admitted = 0, n_frames = 0, n_integ = 0, n_dropped = 0;
    int last_error = XE_OK;
    std::string last_msg;            // detail of last_error (from the scheduler thread)

    int64_t hold_since = 0;          // first pass that held back a partial batch
    bool flush_req = false;
    int64_t n_launch_groups = 0, n_launch_passes = 0, n_held = 0, launch_ns = 0;
    int64_t n_rejected = 0;          // admissions refused for the HBM budget

    // Checkpoints: one request at a time (snap_mu), served by the scheduler thread.
    std::mutex snap_mu;
    xe::SnapReq *snap = nullptr;
    std::condition_variable cv_snap;
    int32_t *snap_host = nullptr;    // pinned copy of one accumulator
    cudaEvent_t snap_ev = nullptr;   // the copy into snap_host has landed
};

namespace xe {
namespace {

constexpr int kBufsPerChan = 2;
constexpr int kMaxGroups = 4;                 // launch groups (jobs of one channel) per pass
constexpr int kMaxMerge = 4;                  // consecutive frames merged into one job
constexpr int64_t kHoldNs = 1500000;          // longest wait for a fuller batch

cudaEvent_t take_event(xe_stream *s) {
    if (!s->spare_events.empty()) {
        cudaEvent_t e = s->spare_events.back();
        s->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

int take_pass_event(xe_stream *s) {
    for (int k = 0; k < int(s->pass_events.size()); ++k)
        if (s->pass_events[size_t(k)].refs == 0) return k;
    PassEvent pe;
    cudaEventCreateWithFlags(&pe.ev, cudaEventDisableTiming);
    s->pass_events.push_back(pe);
    return int(s->pass_events.size()) - 1;
}

bool has_free_buf(xe_stream *s, int c) {
    for (int k : s->chans[size_t(c)].bufs)
        if (!s->bufs[size_t(k)].busy) return true;
    return false;
}

struct Export {
    int chan;
    int acc_idx;
    int buf;
    xe_result r;
};

// Close channel c's integration (s->mu held): pick a result buffer, switch the channel to its
// other accumulator, and describe the export to enqueue after the pass's launches.
Export close_integration(xe_stream *s, int c) {
    Chan &ch = s->chans[size_t(c)];
    int b = -1;
    for (int k : ch.bufs)
        if (!s->bufs[size_t(k)].busy) { b = k; break; }
    s->bufs[size_t(b)].busy = true;   // a free buffer is guaranteed by the caller
    Export ex{};
    ex.chan = c;
    ex.acc_idx = ch.cur;
    ex.buf = b;
    ex.r.chan = c;
    ex.r.integ_index = ch.integ_index;
    ex.r.n_samples = ch.samples_in_integ;
    ex.r.complete = (!ch.lost && ch.samples_in_integ == s->cfg.integ_T) ? 1 : 0;
    ex.r.vis = s->bufs[size_t(b)].host;
    ex.r.t_first_arrival_ns = ch.t_first;
    ex.r.t_last_arrival_ns = ch.t_last;
    ex.r.handle = b;
    ch.cur ^= 1;
    ch.acc_wait[ch.cur] = true;
    ch.integ_index += 1;
    ch.frames_in_integ = 0;
    ch.samples_in_integ = 0;
    ch.lost = false;
    ch.t_first = ch.t_last = 0;
    return ex;
}

// One scheduler pass.  Returns true if it did any work.
bool pass(xe_stream *s) {
    std::vector<std::vector<xe_job>> groups(static_cast<size_t>(kMaxGroups));
    std::vector<std::vector<int>> group_acc(static_cast<size_t>(kMaxGroups));
    size_t n_jobs = 0;
    std::vector<int> used;             // (chan << 8 | slot) read by this pass
    std::vector<cudaEvent_t> waits;    // accumulator exports the launches must follow
    std::vector<Export> exports;
    bool work = false;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        // Frames whose copies landed; slots whose readers finished.
        for (size_t c = 0; c < s->chans.size(); ++c) {
            Chan &ch = s->chans[c];
            if (!ch.admitted || ch.n_copying == 0) continue;
            for (Slot &sl : ch.ring)
                if (sl.state == kCopying && cudaEventQuery(sl.copy_ev) == cudaSuccess) {
                    sl.state = kReady;
                    --ch.n_copying;
                }
        }
        for (size_t k = 0; k < s->queued_slots.size();) {
            const int code = s->queued_slots[k];
            Chan &ch = s->chans[size_t(code >> 8)];
            Slot &sl = ch.ring[size_t(code & 255)];
            PassEvent &pe = s->pass_events[size_t(sl.pass_ev)];
            if (cudaEventQuery(pe.ev) == cudaSuccess) {
                sl.state = kFree;
                pe.refs -= 1;
                sl.pass_ev = -1;
                s->queued_slots[k] = s->queued_slots.back();
                s->queued_slots.pop_back();
                work = true;
            } else {
                ++k;
            }
        }
        while (!s->pending.empty() && cudaEventQuery(s->pending.front().ev) == cudaSuccess) {
            Pending p = s->pending.front();
            s->pending.pop_front();
            p.r.t_ready_ns = now_ns();
            s->spare_events.push_back(p.ev);
            s->ready.push_back(p.r);
            s->n_integ += 1;
            s->cv_ready.notify_all();
            work = true;
        }
        // Batching: while frames are still being copied in and fewer than all waiting
        // channels are ready, hold the launch for up to kHoldNs so one launch carries them.
        int n_ready = 0, n_copying = 0;
        for (size_t c = 0; c < s->chans.size(); ++c) {
            const Chan &ch = s->chans[c];
            if (!ch.admitted || ch.fifo.empty()) continue;
            const Entry &e = ch.fifo.front();
            if (e.slot < 0 || ch.ring[size_t(e.slot)].state == kReady) ++n_ready;
            else ++n_copying;
        }
        const int64_t t_now = now_ns();
        if (n_ready == 0) {
            s->hold_since = 0;
        } else if (n_copying > 0) {
            if (s->hold_since == 0) s->hold_since = t_now;
            if (t_now - s->hold_since < kHoldNs && !s->flush_req) {
                ++s->n_held;
                return work;
            }
        }
        s->hold_since = 0;
        // Every channel's ready frames, in order: a run of consecutive frames that sit in
        // consecutive ring slots (slots are filled round-robin and contiguous) becomes ONE job
        // of up to kMaxMerge frames; the channel's g-th job goes to launch group g (jobs of
        // one channel never share a launch: they add into the same accumulator).  A channel
        // stops at its first closed integration in the pass.
        for (size_t c = 0; c < s->chans.size(); ++c) {
            Chan &ch = s->chans[c];
            if (!ch.admitted) continue;
            int g = 0, run_slot = -1, run_len = 0;
            auto emit = [&]() {
                if (run_len == 0) return;
                if (ch.acc_wait[ch.cur]) {
                    waits.push_back(ch.acc_free_ev[ch.cur]);
                    ch.acc_wait[ch.cur] = false;
                }
                groups[size_t(g)].push_back(xe_job{ch.ring[size_t(run_slot)].dev, ch.acc[ch.cur], s->cfg.N, 1,
                                                   int64_t(run_len) * s->cfg.frame_T});
                group_acc[size_t(g)].push_back(ch.fresh[ch.cur] ? 0 : 1);
                ch.fresh[ch.cur] = false;
                ++g;
                run_len = 0;
            };
            while (!ch.fifo.empty() && g < kMaxGroups) {
                const Entry e = ch.fifo.front();
                const bool closes = ch.frames_in_integ + 1 == s->frames_per_integ;
                if (closes && !has_free_buf(s, int(c))) break;       // consumer is behind
                if (e.slot < 0) {                                     // a lost frame
                    emit();
                    ch.fifo.pop_front();
                    if (ch.frames_in_integ == 0) ch.t_first = e.t_arrival;
                    ch.t_last = e.t_arrival;
                    ch.lost = true;
                    ch.frames_in_integ += 1;
                    if (closes) {
                        exports.push_back(close_integration(s, int(c)));
                        break;
                    }
                    continue;
                }
                Slot &sl = ch.ring[size_t(e.slot)];
                if (sl.state != kReady) break;
                if (run_len > 0 && (e.slot != run_slot + run_len || run_len == kMaxMerge)) {
                    emit();
                    if (g == kMaxGroups) break;
                }
                ch.fifo.pop_front();
                sl.state = kQueued;
                if (run_len == 0) run_slot = e.slot;
                ++run_len;
                used.push_back(int(c) << 8 | e.slot);
                if (ch.frames_in_integ == 0) ch.t_first = e.t_arrival;
                ch.t_last = e.t_arrival;
                ch.frames_in_integ += 1;
                ch.samples_in_integ += s->cfg.frame_T;
                if (closes) {
                    emit();
                    exports.push_back(close_integration(s, int(c)));
                    break;
                }
            }
            emit();
        }
        s->flush_req = false;
        n_jobs = 0;
        for (auto &gr : groups) n_jobs += gr.size();
    }
    if (n_jobs == 0 && exports.empty()) return work;

    // Launch outside the lock; pushes and polls proceed meanwhile.
    for (cudaEvent_t e : waits) cudaStreamWaitEvent(s->comp_s, e, 0);
    int rc = XE_OK;
    const int64_t t_l0 = now_ns();
    int n_groups = 0;
    for (size_t gi = 0; gi < groups.size(); ++gi)
        if (!groups[gi].empty() && rc == XE_OK) {
            // The jobs of a group are independent (different channels): listing them by
            // length (longest first, then channel order) makes the batch shape depend only
            // on how many jobs merged how many frames, so passes reuse cached plans instead
            // of planning every new arrangement of the same jobs.
            std::vector<size_t> order(groups[gi].size());
            for (size_t k = 0; k < order.size(); ++k) order[k] = k;
            std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
                return groups[gi][a].T > groups[gi][b].T;
            });
            std::vector<xe_job> jobs_sorted(order.size());
            std::vector<int> acc_sorted(order.size());
            for (size_t k = 0; k < order.size(); ++k) {
                jobs_sorted[k] = groups[gi][order[k]];
                acc_sorted[k] = group_acc[gi][order[k]];
            }
            rc = run_jobs_mixed(jobs_sorted.data(), acc_sorted.data(), int(jobs_sorted.size()), s->comp_s);
            ++n_groups;
        }
    const int64_t t_l1 = now_ns();
    cudaEvent_t done = nullptr;
    std::vector<Pending> pend;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (rc != XE_OK) {
            s->last_error = rc;
            s->last_msg = xe_last_error();
        }
        const int pe = take_pass_event(s);
        done = s->pass_events[size_t(pe)].ev;
        cudaEventRecord(done, s->comp_s);
        for (int code : used) {
            Slot &sl = s->chans[size_t(code >> 8)].ring[size_t(code & 255)];
            sl.pass_ev = pe;
            s->pass_events[size_t(pe)].refs += 1;
            s->queued_slots.push_back(code);
        }
        s->n_frames += int64_t(used.size());      // frames read (merged runs count each frame)
        s->n_launch_groups += n_groups;
        s->n_launch_passes += n_groups > 0 ? 1 : 0;
        s->launch_ns += t_l1 - t_l0;
        // Exports run on their own stream after this pass's launches.
        if (!exports.empty()) cudaStreamWaitEvent(s->d2h_s, done, 0);
        for (const Export &ex : exports) {
            Chan &ch = s->chans[size_t(ex.chan)];
            int32_t *acc = ch.acc[ex.acc_idx];
            // An integration whose frames were all lost never wrote its accumulator.
            if (ch.fresh[ex.acc_idx]) cudaMemsetAsync(acc, 0, s->acc_bytes, s->d2h_s);
            cudaMemcpyAsync(s->bufs[size_t(ex.buf)].host, acc, s->acc_bytes, cudaMemcpyDeviceToHost, s->d2h_s);
            Pending p{};
            p.r = ex.r;
            p.ev = take_event(s);
            cudaEventRecord(p.ev, s->d2h_s);
            cudaEventRecord(ch.acc_free_ev[ex.acc_idx], s->d2h_s);
            ch.fresh[ex.acc_idx] = true;        // its next frame overwrites it
            s->pending.push_back(p);
        }
    }
    return true;
}

// Serve a checkpoint request (between passes, so every frame the channel counts has its
// launches on the compute stream already): record the integration's bookkeeping and put the
// accumulator's copy on the compute stream, after those launches and before any later one.
void serve_snapshot(xe_stream *s) {
    std::lock_guard<std::mutex> lk(s->mu);
    SnapReq *q = s->snap;
    if (!q || q->state != 0) return;
    const Chan &ch = s->chans[size_t(q->chan)];
    if (!ch.admitted) {
        q->state = 2;
        s->cv_snap.notify_all();
        return;
    }
    q->info.integ_index = ch.integ_index;
    q->info.next_seq = ch.integ_index * s->frames_per_integ + ch.frames_in_integ;
    q->info.frames = ch.frames_in_integ;
    q->info.n_samples = ch.samples_in_integ;
    q->info.lost = ch.lost ? 1 : 0;
    q->info.t_first_arrival_ns = ch.t_first;
    q->zero = ch.fresh[ch.cur];
    if (!q->zero)
        cudaMemcpyAsync(s->snap_host, ch.acc[ch.cur], s->acc_bytes, cudaMemcpyDeviceToHost, s->comp_s);
    cudaEventRecord(s->snap_ev, s->comp_s);
    q->state = 1;
    s->cv_snap.notify_all();
}

void scheduler_main(xe_stream *s) {
    cudaSetDevice(s->dev);
    while (!s->stop.load()) {
        const bool worked = pass(s);
        serve_snapshot(s);
        if (!worked) {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait_for(lk, std::chrono::microseconds(200));
        }
    }
}

int sfail(int code, const char *msg) { return record_error(code, msg); }

// Queue one frame (s->mu held).  Returns XE_OK, XE_EAGAIN (ring full) or an error.
int push_locked(xe_stream *s, int chan, const uint8_t *frame, int64_t seq, int64_t t,
                cudaEvent_t *copy_ev) {
    if (chan < 0 || chan >= int(s->chans.size()) || !s->chans[size_t(chan)].admitted)
        return sfail(XE_EINVAL, "channel not admitted");
    if (!frame) return sfail(XE_EINVAL, "null frame");
    Chan &ch = s->chans[size_t(chan)];
    if (seq < ch.expected_push) return sfail(XE_EINVAL, "frame is older than the open integration or a duplicate");
    if (seq - ch.expected_push > 1000000) return sfail(XE_EINVAL, "sequence gap too large");
    int slot = -1;
    const int R = int(ch.ring.size());
    for (int k = 0; k < R; ++k) {
        const int idx = (ch.next_slot + k) % R;
        if (ch.ring[size_t(idx)].state == kFree) {
            slot = idx;
            ch.next_slot = (idx + 1) % R;
            break;
        }
    }
    if (slot < 0) return XE_EAGAIN;
    for (int64_t q = ch.expected_push; q < seq; ++q) {     // frames that never came
        ch.fifo.push_back(Entry{q, -1, t});
        s->n_dropped += 1;
    }
    Slot &sl = ch.ring[size_t(slot)];
    cudaError_t e = cudaMemcpyAsync(sl.dev, frame, s->frame_bytes,
                                    s->cfg.device_source ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    s->copy_s);
    if (e != cudaSuccess) return sfail(XE_ECUDA, cudaGetErrorString(e));
    cudaEventRecord(sl.copy_ev, s->copy_s);
    sl.state = kCopying;
    ch.n_copying += 1;
    ch.fifo.push_back(Entry{seq, slot, t});
    ch.expected_push = seq + 1;
    if (copy_ev) *copy_ev = sl.copy_ev;
    return XE_OK;
}

}  // namespace
}  // namespace xe

using namespace xe;

extern "C" {

int xe_stream_open(const xe_stream_cfg *cfg, xe_stream **out) {
    if (!cfg || !out) return sfail(XE_EINVAL, "null stream config or output");
    const xe_stream_cfg &c = *cfg;
    if (c.N < 1 || c.N > XE_MAX_N) return sfail(XE_EINVAL, "stream N out of range");
    if (c.frame_T < 1 || c.frame_T > kExactChunkT)
        return sfail(XE_EINVAL, "frame_T must lie in [1, 131072]");
    if (c.integ_T < c.frame_T || c.integ_T % c.frame_T != 0)
        return sfail(XE_EINVAL, "integ_T must be a positive multiple of frame_T");
    if (c.integ_T > XE_MAX_T) return sfail(XE_EOVERFLOW, "integ_T too long for int32 visibilities");
    if (c.max_chan < 1 || c.max_chan > 65536) return sfail(XE_EINVAL, "max_chan out of range");
    if (c.ring_frames < 2 || c.ring_frames > 64) return sfail(XE_EINVAL, "ring_frames must lie in [2, 64]");
    // One channel slot: two accumulators, the frame ring and a share of the staged planes
    // (up to `merge` frames of a channel are correlated as one job).
    const int64_t B = int64_t(c.N) * (c.N + 1) / 2;
    const size_t frame_bytes = size_t(c.frame_T) * size_t(c.N);
    const size_t acc_bytes = size_t(B) * 2 * sizeof(int32_t);
    const size_t n_pad = size_t((c.N + kNPad - 1) / kNPad * kNPad);
    const size_t merge = size_t(c.ring_frames < kMaxMerge ? c.ring_frames : kMaxMerge);
    const size_t stage_bytes = merge * 2 * n_pad * size_t((c.frame_T + 63) / 64 * 64);
    const size_t per_chan_bytes = 2 * acc_bytes + size_t(c.ring_frames) * frame_bytes + stage_bytes;
    if (c.hbm_budget < int64_t(per_chan_bytes)) return sfail(XE_EBUDGET, "the HBM budget does not fit one channel slot");
    int dev = 0;
    const cudaError_t ge = cudaGetDevice(&dev);
    if (ge == cudaErrorNoDevice || ge == cudaErrorInsufficientDriver)
        return sfail(XE_ENODEV, "no usable CUDA device (no device or no driver)");
    if (ge != cudaSuccess) return sfail(XE_ECUDA, "cudaGetDevice failed");
    xe_stream *s = new xe_stream;
    s->cfg = c;
    s->dev = dev;
    s->B = B;
    s->frame_bytes = frame_bytes;
    s->acc_bytes = acc_bytes;
    s->frames_per_integ = c.integ_T / c.frame_T;
    s->per_chan_bytes = per_chan_bytes;
    s->chans.resize(size_t(c.max_chan));
    if (cudaStreamCreateWithFlags(&s->copy_s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->comp_s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->d2h_s, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return sfail(XE_ECUDA, "stream creation failed");
    }
    // Size the correlation's scratch now for the largest batch the budget can admit (every
    // channel contributes at most one job of at most `merge` frames to a launch group), so
    // that no batch regrows it, which would synchronise the device, while frames stream in.
    // Best effort: if the memory is not there, batches grow the scratch as they need it.
    const int64_t fit = c.hbm_budget / int64_t(s->per_chan_bytes);
    const int max_jobs = int(std::min<int64_t>(std::min<int64_t>(c.max_chan, fit), kMaxJobs));
    if (reserve_stream_scratch(s->comp_s, max_jobs, c.N, int64_t(merge) * c.frame_T) != XE_OK)
        cudaGetLastError();
    s->sched = std::thread(scheduler_main, s);
    *out = s;
    return XE_OK;
}

int xe_stream_admit(xe_stream *s, int chan) {
    if (!s) return sfail(XE_EINVAL, "null stream");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->closed) return sfail(XE_ECLOSED, "stream closed");
    if (chan < 0 || chan >= int(s->chans.size())) return sfail(XE_EINVAL, "channel id out of range");
    Chan &ch = s->chans[size_t(chan)];
    if (ch.admitted) return XE_OK;
    if (s->used_bytes + int64_t(s->per_chan_bytes) > s->cfg.hbm_budget) {
        s->n_rejected += 1;
        return sfail(XE_EBUDGET, "HBM budget full");
    }
    if (int(s->cfg.ring_frames) > 255) return sfail(XE_EINVAL, "ring too large");
    cudaSetDevice(s->dev);
    for (int a = 0; a < 2; ++a) {
        if (cudaMalloc(&ch.acc[a], s->acc_bytes) != cudaSuccess) {
            cudaGetLastError();
            return sfail(XE_ENOMEM, "accumulator allocation failed");
        }
        cudaMemset(ch.acc[a], 0, s->acc_bytes);
        cudaEventCreateWithFlags(&ch.acc_free_ev[a], cudaEventDisableTiming);
        ch.acc_wait[a] = false;
        ch.fresh[a] = true;
    }
    ch.cur = 0;
    ch.ring.assign(size_t(s->cfg.ring_frames), Slot{});
    if (cudaMalloc(&ch.ring_base, s->frame_bytes * size_t(s->cfg.ring_frames)) != cudaSuccess) {
        cudaGetLastError();
        ch.ring_base = nullptr;
        return sfail(XE_ENOMEM, "frame ring allocation failed");
    }
    for (size_t k = 0; k < ch.ring.size(); ++k) {
        ch.ring[k].dev = ch.ring_base + k * s->frame_bytes;
        cudaEventCreateWithFlags(&ch.ring[k].copy_ev, cudaEventDisableTiming);
    }
    ch.next_slot = 0;
    if (ch.bufs.empty()) {
        for (int k = 0; k < kBufsPerChan; ++k) {
            ResultBuf rb;
            if (cudaHostAlloc(reinterpret_cast<void **>(&rb.host), s->acc_bytes, cudaHostAllocDefault) !=
                cudaSuccess) {
                cudaGetLastError();
                return sfail(XE_ENOMEM, "pinned result buffer allocation failed");
            }
            rb.chan = chan;
            ch.bufs.push_back(int(s->bufs.size()));
            s->bufs.push_back(rb);
        }
    }
    cudaDeviceSynchronize();
    ch.fifo.clear();
    ch.n_copying = 0;
    ch.expected_push = 0;
    ch.integ_index = ch.frames_in_integ = ch.samples_in_integ = 0;
    ch.lost = false;
    ch.admitted = true;
    s->used_bytes += int64_t(s->per_chan_bytes);
    s->n_admitted += 1;
    return XE_OK;
}

int xe_stream_evict(xe_stream *s, int chan) {
    if (!s) return sfail(XE_EINVAL, "null stream");
    std::lock_guard<std::mutex> lk(s->mu);
    if (chan < 0 || chan >= int(s->chans.size()) || !s->chans[size_t(chan)].admitted)
        return sfail(XE_EINVAL, "channel not admitted");
    Chan &ch = s->chans[size_t(chan)];
    cudaStreamSynchronize(s->copy_s);
    cudaStreamSynchronize(s->comp_s);
    cudaStreamSynchronize(s->d2h_s);
    for (size_t k = 0; k < s->queued_slots.size();) {
        if ((s->queued_slots[k] >> 8) == chan) {
            Slot &sl = ch.ring[size_t(s->queued_slots[k] & 255)];
            s->pass_events[size_t(sl.pass_ev)].refs -= 1;
            s->queued_slots[k] = s->queued_slots.back();
            s->queued_slots.pop_back();
        } else {
            ++k;
        }
    }
    for (Slot &sl : ch.ring) cudaEventDestroy(sl.copy_ev);
    cudaFree(ch.ring_base);
    ch.ring_base = nullptr;
    ch.ring.clear();
    ch.fifo.clear();
    for (int a = 0; a < 2; ++a) {
        cudaFree(ch.acc[a]);
        cudaEventDestroy(ch.acc_free_ev[a]);
        ch.acc[a] = nullptr;
        ch.acc_free_ev[a] = nullptr;
    }
    ch.admitted = false;
    s->used_bytes -= int64_t(s->per_chan_bytes);
    s->n_admitted -= 1;
    return XE_OK;
}

int xe_stream_push(xe_stream *s, int chan, const uint8_t *frame, int64_t seq, int64_t t_arrival_ns) {
    if (!s) return sfail(XE_EINVAL, "null stream");
    cudaEvent_t wait_ev = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->closed) return sfail(XE_ECLOSED, "stream closed");
        const int rc = push_locked(s, chan, frame, seq, t_arrival_ns > 0 ? t_arrival_ns : now_ns(), &wait_ev);
        if (rc != XE_OK) return rc;
    }
    // Host source: the caller's bytes are on the device before the call returns.
    if (!s->cfg.device_source) cudaEventSynchronize(wait_ev);
    s->cv_work.notify_one();
    return XE_OK;
}

int xe_stream_push_frames(xe_stream *s, int n, const int *chans, const uint8_t *const *frames,
                          const int64_t *seqs, int64_t t_arrival_ns, int *rc_out) {
    if (!s || n < 0 || (n > 0 && (!chans || !frames || !seqs))) return sfail(XE_EINVAL, "bad frame batch");
    cudaEvent_t last = nullptr;
    int n_ok = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->closed) return sfail(XE_ECLOSED, "stream closed");
        const int64_t t = t_arrival_ns > 0 ? t_arrival_ns : now_ns();
        for (int k = 0; k < n; ++k) {
            cudaEvent_t ev = nullptr;
            const int rc = push_locked(s, chans[k], frames[k], seqs[k], t, &ev);
            if (rc_out) rc_out[k] = rc;
            if (rc == XE_OK) {
                last = ev;
                ++n_ok;
            }
        }
    }
    if (!s->cfg.device_source && last) cudaStreamSynchronize(s->copy_s);
    s->cv_work.notify_one();
    return n_ok;
}

int xe_stream_flush(xe_stream *s) {
    if (!s) return sfail(XE_EINVAL, "null stream");
    // Wait (bounded) until every pushed frame has been launched.
    const int64_t deadline = now_ns() + 10000000000LL;
    while (now_ns() < deadline) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            bool any = false;
            for (const Chan &ch : s->chans)
                if (ch.admitted && !ch.fifo.empty()) { any = true; break; }
            if (!any) return XE_OK;
            s->flush_req = true;
        }
        s->cv_work.notify_one();
        std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
    return sfail(XE_ETIMEOUT, "flush: frames still waiting after 10 s");
}

int xe_stream_poll(xe_stream *s, xe_result *r, int timeout_ms) {
    if (!s || !r) return sfail(XE_EINVAL, "null stream or result");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->ready.empty() && timeout_ms > 0)
        s->cv_ready.wait_for(lk, std::chrono::milliseconds(timeout_ms), [s] { return !s->ready.empty(); });
    if (s->last_error != XE_OK) {
        const int e = s->last_error;
        s->last_error = XE_OK;
        const std::string msg = "a batched launch of the stream failed: " + s->last_msg;
        return sfail(e, msg.c_str());
    }
    if (s->ready.empty()) return XE_EAGAIN;
    *r = s->ready.front();
    s->ready.pop_front();
    return XE_OK;
}

int xe_stream_release(xe_stream *s, int64_t handle) {
    if (!s) return sfail(XE_EINVAL, "null stream");
    std::lock_guard<std::mutex> lk(s->mu);
    if (handle < 0 || handle >= int64_t(s->bufs.size()) || !s->bufs[size_t(handle)].busy)
        return sfail(XE_EINVAL, "unknown or already released result handle");
    s->bufs[size_t(handle)].busy = false;
    s->cv_work.notify_one();
    return XE_OK;
}

int xe_stream_stats(xe_stream *s, int64_t *admitted, int64_t *frames, int64_t *integrations,
                    int64_t *dropped) {
    if (!s) return sfail(XE_EINVAL, "null stream");
    std::lock_guard<std::mutex> lk(s->mu);
    if (admitted) *admitted = s->n_admitted;
    if (frames) *frames = s->n_frames;
    if (integrations) *integrations = s->n_integ;
    if (dropped) *dropped = s->n_dropped;
    return XE_OK;
}

int xe_stream_counters(xe_stream *s, int64_t *out, int n) {
    if (!s || !out || n < 1) return sfail(XE_EINVAL, "bad counter query");
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t v[9] = {s->n_admitted, s->n_frames, s->n_integ, s->n_dropped,
                          s->n_launch_passes, s->n_launch_groups, s->n_held, s->launch_ns,
                          s->n_rejected};
    for (int k = 0; k < n && k < 9; ++k) out[k] = v[k];
    return n < 9 ? n : 9;
}

int xe_stream_snapshot(xe_stream *s, int chan, int32_t *host_vis, xe_snapshot *info, int timeout_ms) {
    if (!s || !host_vis || !info) return sfail(XE_EINVAL, "null stream, buffer or snapshot");
    if (timeout_ms < 0) return sfail(XE_EINVAL, "negative timeout");
    std::lock_guard<std::mutex> one(s->snap_mu);
    SnapReq q;
    q.chan = chan;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->closed) return sfail(XE_ECLOSED, "stream closed");
        if (chan < 0 || chan >= int(s->chans.size()) || !s->chans[size_t(chan)].admitted)
            return sfail(XE_EINVAL, "channel not admitted");
        if (!s->snap_host) {
            cudaSetDevice(s->dev);
            if (cudaHostAlloc(reinterpret_cast<void **>(&s->snap_host), s->acc_bytes, cudaHostAllocDefault) !=
                cudaSuccess) {
                cudaGetLastError();
                s->snap_host = nullptr;
                return sfail(XE_ENOMEM, "pinned snapshot buffer allocation failed");
            }
            if (cudaEventCreateWithFlags(&s->snap_ev, cudaEventDisableTiming) != cudaSuccess)
                return sfail(XE_ECUDA, "event creation failed");
        }
        s->snap = &q;
        s->cv_work.notify_one();
        const bool served = s->cv_snap.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                                [&q] { return q.state != 0; });
        s->snap = nullptr;            // the scheduler touches q only under s->mu
        if (!served) return sfail(XE_ETIMEOUT, "snapshot: the scheduler did not serve the request in time");
        if (q.state == 2) return sfail(XE_EINVAL, "channel evicted");
    }
    const int64_t deadline = now_ns() + int64_t(timeout_ms) * 1000000LL;
    for (;;) {
        const cudaError_t e = cudaEventQuery(s->snap_ev);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return sfail(XE_ECUDA, cudaGetErrorString(e));
        if (now_ns() > deadline) return sfail(XE_ETIMEOUT, "snapshot: the copy did not land in time");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    if (q.zero)
        memset(host_vis, 0, s->acc_bytes);
    else
        memcpy(host_vis, s->snap_host, s->acc_bytes);
    *info = q.info;
    return XE_OK;
}

int xe_stream_restore(xe_stream *s, int chan, const int32_t *host_vis, const xe_snapshot *info) {
    if (!s || !info) return sfail(XE_EINVAL, "null stream or snapshot");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->closed) return sfail(XE_ECLOSED, "stream closed");
    if (chan < 0 || chan >= int(s->chans.size()) || !s->chans[size_t(chan)].admitted)
        return sfail(XE_EINVAL, "channel not admitted");
    Chan &ch = s->chans[size_t(chan)];
    if (ch.expected_push != 0 || !ch.fifo.empty() || ch.integ_index != 0 || ch.frames_in_integ != 0 ||
        !ch.fresh[ch.cur])
        return sfail(XE_EINVAL, "restore needs a channel that has taken no frame since it was admitted");
    const xe_snapshot &q = *info;
    const int64_t fpi = s->frames_per_integ, fT = s->cfg.frame_T;
    const bool ok = q.integ_index >= 0 && q.integ_index < (int64_t(1) << 40) && q.frames >= 0 &&
                    q.frames < fpi && q.n_samples >= 0 && q.n_samples % fT == 0 &&
                    q.n_samples <= q.frames * fT && (q.lost != 0 || q.n_samples == q.frames * fT) &&
                    q.next_seq == q.integ_index * fpi + q.frames;
    if (!ok) return sfail(XE_EINVAL, "inconsistent snapshot for this stream's frame and integration lengths");
    if (q.n_samples > 0) {
        if (!host_vis) return sfail(XE_EINVAL, "null visibilities for a snapshot with sums");
        cudaSetDevice(s->dev);
        // On the compute stream: every later launch that adds into this accumulator follows it.
        const cudaError_t e = cudaMemcpyAsync(ch.acc[ch.cur], host_vis, s->acc_bytes, cudaMemcpyHostToDevice, s->comp_s);
        if (e != cudaSuccess) return sfail(XE_ECUDA, cudaGetErrorString(e));
        ch.fresh[ch.cur] = false;
    }
    ch.integ_index = q.integ_index;
    ch.frames_in_integ = q.frames;
    ch.samples_in_integ = q.n_samples;
    ch.lost = q.lost != 0;
    ch.t_first = q.frames > 0 ? q.t_first_arrival_ns : 0;
    ch.t_last = ch.t_first;
    ch.expected_push = q.next_seq;
    return XE_OK;
}

void xe_stream_close(xe_stream *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->closed = true;
    }
    s->stop.store(true);
    s->cv_work.notify_all();
    if (s->sched.joinable()) s->sched.join();
    cudaSetDevice(s->dev);
    cudaStreamSynchronize(s->copy_s);
    cudaStreamSynchronize(s->comp_s);
    cudaStreamSynchronize(s->d2h_s);
    release_stream_scratch(s->comp_s);     // the correlation's scratch for this stream
    for (Chan &ch : s->chans) {
        for (Slot &sl : ch.ring) cudaEventDestroy(sl.copy_ev);
        if (ch.ring_base) cudaFree(ch.ring_base);
        ch.ring_base = nullptr;
        for (int a = 0; a < 2; ++a) {
            if (ch.acc[a]) cudaFree(ch.acc[a]);
            if (ch.acc_free_ev[a]) cudaEventDestroy(ch.acc_free_ev[a]);
        }
    }
    for (ResultBuf &rb : s->bufs) cudaFreeHost(rb.host);
    if (s->snap_host) cudaFreeHost(s->snap_host);
    if (s->snap_ev) cudaEventDestroy(s->snap_ev);
    for (Pending &p : s->pending) cudaEventDestroy(p.ev);
    for (cudaEvent_t e : s->spare_events) cudaEventDestroy(e);
    for (PassEvent &pe : s->pass_events) cudaEventDestroy(pe.ev);
    cudaStreamDestroy(s->copy_s);
    cudaStreamDestroy(s->comp_s);
    cudaStreamDestroy(s->d2h_s);
    delete s;
}

}  // extern "C"
