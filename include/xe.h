/*
 * xe.h -- C ABI of libxe, an exact X-engine correlator for GB300 (sm_103a).
 *
 * The operation (Denman et al. 2020, "A GPU Spatial Processing System for CHIME",
 * section 1 and section 2.2): for every frequency channel, correlate every receiver input
 * against every other, autocorrelations included:
 *
 *     V_ij = sum_{t < T} x_i(t) * conj(x_j(t)),   0 <= i <= j < N,
 *
 * over channelised complex voltages with 4 bits real + 4 bits imaginary per sample
 * (section 2.2, d = 8).  Channels are independent (section 2.3).  The sums are exact
 * integers: every call returns bit-identical results for the same input.
 *
 * Data formats (shared by every entry point):
 *   input   uint8  in[C][T][N]   one byte per sample; high nibble = real part, low
 *                                nibble = imaginary part, each two's complement (-8..7).
 *                                Per channel, time-major: all N inputs of one sample are
 *                                contiguous (the corner-turned order, section 2.3).
 *   output  int32  vis[C][B][2]  B = N(N+1)/2 baselines, row-major upper triangle
 *                                including the diagonal: baseline (i, j), i <= j, is at
 *                                k = i*N - i*(i-1)/2 + (j - i); {Re, Im} interleaved
 *                                (8 bytes per visibility, as in Table tab:data-flow).
 *
 * Ownership: unless an entry point says otherwise, `in` and `vis` are caller-owned
 * DEVICE pointers (e.g. torch tensors on cuda).  The library never frees them.  Work is
 * enqueued on the given stream (0 = the legacy default stream) and the call returns
 * without synchronising; the caller synchronises the stream before reading `vis`.
 * Scratch memory is owned by the library, cached per device, and reused across calls.
 *
 * Errors: every int-returning entry point returns XE_OK (0) or a negative XE_E* code.
 * A failed call enqueues nothing and leaves `vis` untouched.  xe_last_error() gives a
 * human-readable detail of the last failure on the calling thread.
 *
 * Exactness limit: |Re|, |Im| <= 128 * T must fit int32, so T <= XE_MAX_T.
 */
#ifndef XE_H
#define XE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XE_OK         0
#define XE_EINVAL    -1   /* bad argument: N < 1, T < 1, C < 1, null or misaligned pointer */
#define XE_EOVERFLOW -2   /* T > XE_MAX_T: the int32 result could overflow */
#define XE_ENOMEM    -3   /* device or host allocation failed */
#define XE_EBUDGET   -4   /* a stream request exceeds its HBM budget */
#define XE_EAGAIN    -5   /* nothing ready yet / not admitted now; try again */
#define XE_ETIMEOUT  -6   /* a bounded device or host wait gave up */
#define XE_ECUDA     -7   /* a CUDA runtime call failed (detail in xe_last_error) */
#define XE_ENODEV    -8   /* no usable sm_103 device */
#define XE_ECLOSED   -9   /* the stream was closed */
#define XE_ECHECK    -10  /* a device-side check of a launch's descriptors failed (option
                             "checks"); the launch wrote nothing */

#define XE_MAX_T 16777215LL   /* 128 * T < 2^31 */
#define XE_MAX_N 65536

/* Kernel families.  XE_ALGO_TC is the tcgen05 tensor-core path (FP8 e4m3 operands,
 * exact because every operand is an integer in [-8, 8] and every partial sum stays below
 * 2^24); XE_ALGO_IMMA is the legacy warp-level int8 mma.sync path (exact by construction,
 * int32 accumulate).  XE_ALGO_AUTO picks XE_ALGO_TC. */
#define XE_ALGO_AUTO 0
#define XE_ALGO_TC   1
#define XE_ALGO_IMMA 2

/* ---- library ------------------------------------------------------------------- */

/* Human-readable name of an XE_* code.  Never NULL; the string is static. */
const char *xe_strerror(int code);

/* Detail of the last failed call on this thread (static per-thread buffer). */
const char *xe_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
int xe_version(void);

/* Number of complex multiply-accumulates of one correlation: C * T * N(N+1)/2
 * (the cost metric eta / delta-nu of section 2.2). */
double xe_cmac(int64_t N, int64_t T, int64_t C);

/* ---- one-shot correlation (section 2.2 X stage) ------------------------------------ */

/* Correlate C channels of N inputs over T samples: in (device) -> vis (device), on the
 * current legacy default stream.  vis is overwritten, never accumulated into.
 * Returns XE_OK, XE_EINVAL, XE_EOVERFLOW, XE_ENOMEM, XE_ECUDA or XE_ENODEV. */
int xe_correlate(const uint8_t *in, int N, int64_t T, int n_chan, int32_t *vis);

/* As xe_correlate, enqueued on `stream` (a cudaStream_t passed as void*), with an
 * explicit kernel family (XE_ALGO_*). */
int xe_correlate_async(const uint8_t *in, int N, int64_t T, int n_chan, int32_t *vis,
                       int algo, void *stream);

/* As xe_correlate, but `host_in` and `host_vis` are HOST pointers (pinned memory gives the
 * full copy bandwidth).  The library copies the input to device memory it owns, correlates
 * and copies the visibilities back before returning (synchronous).  For callers that do
 * not manage device memory.  Returns as xe_correlate. */
int xe_correlate_host(const uint8_t *host_in, int N, int64_t T, int n_chan, int32_t *host_vis,
                      int algo);

/* Asynchronous host-buffer correlation for callers that feed a stream of host blocks.
 * Enqueues the copies and the correlation of host_in into slot `slot` (0 <= slot <
 * XE_HOST_SLOTS; each slot owns device buffers inside the library) and returns at once;
 * host_vis receives the visibilities, valid once xe_host_wait(slot) has returned XE_OK.
 * Both host buffers must stay untouched until then (pinned memory is required for the
 * copies to overlap).  Successive calls on different slots overlap: the device -> host copy
 * of one result runs while the next block is copied in and correlated.  Calling on a slot
 * that is still in flight returns XE_EAGAIN.  The input is copied in one piece and then
 * correlated (tensor-core path), or, with option "host_async_chunk_t", in chunks of that
 * many samples, each correlated as soon as it has landed.  Returns as xe_correlate_host
 * (XE_ETIMEOUT from xe_host_wait if a device wait gave up). */
#define XE_HOST_SLOTS 4
int xe_correlate_host_async(const uint8_t *host_in, int N, int64_t T, int n_chan, int32_t *host_vis, int slot);

/* Wait until slot `slot`'s visibilities are in its host_vis (blocking the calling thread).
 * Returns XE_OK (also for a slot with nothing in flight), XE_EINVAL for a slot outside
 * [0, XE_HOST_SLOTS), XE_ETIMEOUT if a kernel of the slot gave up on a bounded device wait
 * (its output is then invalid; the status is cleared), XE_ECUDA or XE_ENODEV. */
int xe_host_wait(int slot);

/* ---- batched correlation (one persistent launch over many jobs) ------------------- */

/* One job of a batch: n_chan channels of N inputs over T samples, with its own
 * device input and output pointers in the formats above. */
typedef struct xe_job {
    const uint8_t *in;
    int32_t *vis;
    int N;
    int n_chan;
    int64_t T;
} xe_job;

/* Correlate every job of the batch (jobs may differ in N and T) in ONE persistent
 * kernel launch whose work list covers all triangle tiles of all jobs; jobs[] is a
 * host array read during the call.  With use_graph != 0, the launch sequence is captured
 * into a CUDA graph keyed on the batch shape and replayed on later calls of the same
 * shape (pointers are refreshed in place).  Returns as xe_correlate_async. */
int xe_correlate_batch(const xe_job *jobs, int n_jobs, int use_graph, void *stream);

/* As xe_correlate_batch without graphs, but ADDS each job's visibilities into its vis
 * (vis += V): callers integrate consecutive blocks of samples into their own int32
 * accumulators (time integration, section 2.1).  The caller keeps |sum| < 2^31. */
int xe_correlate_accumulate(const xe_job *jobs, int n_jobs, void *stream);

/* ---- flag-masked correlation, offset-binary input --------------------------------- */

/* Flags and metadata travel with the voltages from the F-engine (section 2.2 and Table
 * tab:data-flow: 644 B per 4096 B of data), and RFI excision runs on the GPU before the
 * correlation (Table tab:computing).  The paper fixes no flag format; this library takes
 * one validity bit per (sample, input):
 *
 *   flags  uint8 [C][T][ceil(N/8)]  bit (n % 8) of byte (n / 8) of row (c, t) is 1 when
 *                                   sample t of input n in channel c is valid.
 *                                   Bits of inputs >= N in the last byte are ignored.
 *
 * The masked correlation sums only samples where both inputs are valid,
 *
 *     V_ij = sum_t f_i(t) f_j(t) x_i(t) conj(x_j(t)),
 *     n_ij = sum_t f_i(t) f_j(t)          (valid-sample count of every baseline),
 *
 * with counts int32 [C][B] in the same baseline order as vis.  flags == NULL means every
 * sample is valid.
 *
 * Sample encodings: XE_ENC_TWOS = two's-complement nibbles (the format of every other
 * entry point); XE_ENC_OFFSET = offset binary, nibble u encodes the value u - 8. */
#define XE_ENC_TWOS   0
#define XE_ENC_OFFSET 1

typedef struct xe_masked_job {
    const uint8_t *in;        /* device, [C][T][N] packed samples in `encoding` */
    const uint8_t *flags;     /* device, validity bits as above, or NULL (all valid) */
    int32_t *vis;             /* device, [C][B][2]; 8-byte aligned */
    int32_t *counts;          /* device, [C][B], 4-byte aligned; or NULL (not computed) */
    int N;
    int n_chan;
    int64_t T;
    int encoding;             /* XE_ENC_TWOS or XE_ENC_OFFSET */
    int accumulate;           /* 0: overwrite vis (and counts); 1: vis += V, counts += n */
} xe_masked_job;

/* Masked correlation of every job of the batch (tensor-core path; the counts are a 1-bit
 * tensor-core contraction of the flags).  jobs[] is a host array read during the call;
 * all pointers in it are caller-owned device memory.  Enqueued on `stream`, not
 * synchronised.  Returns XE_OK, XE_EINVAL (bad sizes, null in/vis, unknown encoding,
 * misaligned vis or counts), XE_EOVERFLOW, XE_ENOMEM, XE_ECUDA or XE_ENODEV. */
int xe_correlate_masked_batch(const xe_masked_job *jobs, int n_jobs, void *stream);

/* One masked job (see xe_masked_job for the arguments). */
int xe_correlate_masked(const uint8_t *in, const uint8_t *flags, int N, int64_t T, int n_chan,
                        int encoding, int32_t *vis, int32_t *counts, int accumulate, void *stream);

/* ---- host-side planning (no GPU needed; exposed for tests and tooling) ------------ */

/* Work plan the persistent scheduler would use for a batch: number of triangle tiles,
 * total k-iterations and the number of CTA segments that end in a partial (split) tile,
 * for `n_cta` persistent CTAs.  Pure host computation; returns XE_OK or XE_EINVAL. */
int xe_plan_stats(const int *N, const int64_t *T, const int *n_chan, int n_jobs, int n_cta,
                  int64_t *n_tiles, int64_t *n_iters, int64_t *n_split_tiles);

/* Dump the plan the scheduler builds for a batch, for a given CTA count, schedule
 * (-1 = the default choice; 0 stream-K, 1 equal k-split (parts per tile by a fix-up cost
 * model), 2 full waves + the last wave split the same way,
 * 3 longest-first, 4 k-aligned parts of about equal weighted cost, longest first; the
 * default for masked calls with counts, whose count jobs weigh less) and tile width
 * (0 = default, 128 or 256).  Writes into out[0..cap):
 * {n_tiles, n_segments, n_cta, n_partial}, then per tile {job, chan, i0, j0, nj, kblocks},
 * then per segment {cta, tile, k_lo, k_hi, slot}.  Returns the number of int32 values the
 * dump needs (nothing is written when cap is smaller), or a negative XE_* code.
 * Pure host computation. */
int64_t xe_plan_dump(const int *N, const int64_t *T, const int *n_chan, int n_jobs, int n_cta,
                     int sched, int tile_n, int32_t *out, int64_t cap);

/* The plan configuration (persistent CTAs, tile width, schedule) that the calling
 * thread's last correlation used: the autotuned one if option "autotune" was on when the
 * batch shape was first seen, else the default choice.  XE_EAGAIN if none yet. */
int xe_last_config(int *n_cta, int *tile_n, int *sched);

/* ---- corner turn and input views --------------------------------------------------- */

/* The F-engine delivers each GPU node bundles of four frequency channels, every bundle with
 * the inputs of one cylinder only; the node combines four bundles into full-array data
 * (section 2.1; section 2.3: the node completes the transpose; Table tab:computing:
 * "Re-Order and Pre-Sum").  The paper gives no byte layout; this library reads a bundle as
 *
 *   bundles  uint8 [n_cyl][T][n_freq][n_in]    (one cylinder per bundle, contiguous)
 *   frames   uint8 [n_freq][T][n_cyl * n_in]   full-array input n = cyl * n_in + i
 *   presums  int32 [n_freq][N][2]              sum over the T samples of {re, im} of x_n
 *
 * An input view describes where sample (c, t, n) of a correlation's input lives:
 *     byte  in + c * chan_stride + t * time_stride + (n / seg_inputs) * seg_stride
 *              + n % seg_inputs
 * A plain [C][T][N] input is chan_stride = T N, time_stride = N, seg_inputs = N.  Strides are
 * in bytes; when every stride and seg_inputs are multiples of 16 (and `in` 16-byte aligned)
 * the staging kernel loads 16 bytes at a time, otherwise it loads bytes. */
typedef struct xe_view {
    int64_t chan_stride;
    int64_t time_stride;
    int64_t seg_inputs;
    int64_t seg_stride;
} xe_view;

/* Fill *view with the view of n_freq channels of N = n_cyl * n_in inputs held as cylinder
 * bundles (layout above).  Returns XE_OK or XE_EINVAL. */
int xe_bundle_view(int n_cyl, int n_freq, int n_in, int64_t T, xe_view *view);

/* As xe_correlate_async (tensor-core path), reading the input through `view` (a host struct
 * read during the call).  With xe_bundle_view this correlates the bundles directly: the
 * corner turn happens inside the staging kernel's loads and no frame is materialised.
 * Returns as xe_correlate_async. */
int xe_correlate_view(const uint8_t *in, const xe_view *view, int N, int64_t T, int n_chan, int32_t *vis,
                      void *stream);

/* Materialise the corner turn: bundles -> frames (layouts above), and, if presums is not
 * NULL, the per-input pre-sums.  All pointers are caller-owned DEVICE memory.  Enqueued on
 * `stream`.  Returns XE_OK, XE_EINVAL, XE_EOVERFLOW (T > XE_MAX_T), XE_ENOMEM, XE_ECUDA or
 * XE_ENODEV. */
int xe_corner_turn(const uint8_t *bundles, int n_cyl, int n_freq, int n_in, int64_t T, uint8_t *frames,
                   int32_t *presums, void *stream);

/* ---- phased-array beams ------------------------------------------------------------ */

/* Besides the correlation, the X-engine nodes form phased-array beams for pulsar timing
 * (section 2.1: 10 beams; "Pulsar Beamforming" in Table tab:computing).  The paper gives
 * no formula or weight format; this library computes the weighted coherent sum
 *
 *     y_b(t) = sum_{i < N} w_{b,i} x_i(t),    b < n_beams,
 *
 * exactly in integers, with complex int8 weights:
 *
 *   weights  int8  [n_beams][N][2]      {re, im} of w_{b,i}, each in [-127, 127]
 *                                       (-128 is accepted and also exact)
 *   beams    int32 [C][T][n_beams][2]   {re, im} of y_b(t), time-major (all beams of one
 *                                       sample contiguous)
 *
 * in (the correlation's input format), weights and beams are caller-owned DEVICE pointers;
 * beams is overwritten.  1 <= n_beams <= 128.  Enqueued on `stream`, not synchronised.
 * Runs on the tcgen05 tensor cores: each weight component is split exactly as
 * w = 16 w_hi + w_lo (both in [-8, 8]), so every operand is exact in FP8 e4m3 and every f32
 * partial sum is an integer below 2^24 (<= 128 N).  Beams are formed in groups of at most
 * 64 per launch.  Returns XE_OK, XE_EINVAL (bad sizes, null or misaligned pointers),
 * XE_ENOMEM, XE_ECUDA or XE_ENODEV. */
int xe_beamform(const uint8_t *in, int N, int64_t T, int n_chan, const int8_t *weights, int n_beams,
                int32_t *beams, void *stream);

/* ---- streaming server (continuous integration of frames) --------------------------- */

typedef struct xe_stream_cfg {
    int N;                    /* inputs per channel */
    int64_t frame_T;          /* samples per frame (e.g. 8192) */
    int64_t integ_T;          /* samples per integration, a multiple of frame_T (e.g. 32768) */
    int max_chan;             /* channel slots to admit at most */
    int64_t hbm_budget;       /* bytes of device memory the stream may hold */
    int ring_frames;          /* frame slots in the device ring per channel (>= 2) */
    double sample_rate;       /* samples/s per channel the producer emits (390625 for CHIME) */
    int device_source;        /* 1: xe_stream_push takes device pointers; 0: host pointers */
} xe_stream_cfg;

typedef struct xe_stream xe_stream;

/* One completed integration returned by xe_stream_poll. */
typedef struct xe_result {
    int chan;                 /* channel slot */
    int64_t integ_index;      /* integration number within the channel (0, 1, ...) */
    int64_t n_samples;        /* samples accumulated (== integ_T unless frames were lost) */
    int complete;             /* 1 if every frame of the integration arrived */
    const int32_t *vis;       /* HOST pointer, [B][2] int32; valid until xe_stream_release */
    int64_t t_first_arrival_ns; /* arrival time of the integration's first frame */
    int64_t t_last_arrival_ns;  /* arrival time of its last frame */
    int64_t t_ready_ns;       /* time the visibilities were on the host */
    int64_t handle;           /* pass to xe_stream_release */
} xe_result;

/* Open a stream on the current device.  Validates the configuration, checks that at
 * least one channel slot fits the HBM budget, and allocates nothing per channel until
 * channels are admitted.  Returns XE_OK and *out, or XE_EINVAL / XE_EBUDGET / XE_ENOMEM. */
int xe_stream_open(const xe_stream_cfg *cfg, xe_stream **out);

/* Admit a channel slot if the HBM budget allows it.  A slot holds two int32 accumulators
 * (one filling while the other is exported), ring_frames frame buffers (one contiguous
 * ring, filled round-robin) and its share of the staging memory: up to min(4, ring_frames)
 * consecutive frames of a channel are correlated as one job when they are ready together,
 * so the share is that many frames' staged operands (2 bytes per sample and input).
 * Returns XE_OK, XE_EBUDGET when the budget is full, XE_EINVAL for a bad channel id. */
int xe_stream_admit(xe_stream *s, int chan);

/* Release a channel slot (its pending integration is dropped, its memory returned). */
int xe_stream_evict(xe_stream *s, int chan);

/* Push one frame (frame_T samples x N inputs, [T][N] packed bytes) of channel `chan`
 * with sequence number `seq` (frame index since the channel started) and arrival time
 * t_arrival_ns (CLOCK_MONOTONIC).  The bytes are copied before the call returns (host
 * source) or before the frame's slot is reused (device source).  Returns XE_OK,
 * XE_EAGAIN when the channel's ring is full, XE_EINVAL for an unknown channel or a frame
 * older than the open integration, XE_ECLOSED after close. */
int xe_stream_push(xe_stream *s, int chan, const uint8_t *frame, int64_t seq,
                   int64_t t_arrival_ns);

/* Push n frames at once (typically one frame of every channel that arrived together):
 * frame k is channel chans[k]'s frame with sequence number seqs[k], bytes at frames[k],
 * all with arrival time t_arrival_ns.  Per-frame results (XE_OK, XE_EAGAIN, XE_EINVAL) go to
 * rc_out[k] when rc_out is not NULL.  Host-source bytes are on the device before the call
 * returns.  Returns the number of frames accepted, or a negative XE_* code. */
int xe_stream_push_frames(xe_stream *s, int n, const int *chans, const uint8_t *const *frames,
                          const int64_t *seqs, int64_t t_arrival_ns, int *rc_out);

/* Flush what has been pushed so far: schedule every ready frame now. */
int xe_stream_flush(xe_stream *s);

/* Return the next completed integration, or XE_EAGAIN if none is ready yet.  Blocks for
 * at most timeout_ms milliseconds (0 = do not block). */
int xe_stream_poll(xe_stream *s, xe_result *r, int timeout_ms);

/* Hand a result buffer back to the stream. */
int xe_stream_release(xe_stream *s, int64_t handle);

/* Counters: admitted channels, frames processed, integrations completed, frames dropped. */
int xe_stream_stats(xe_stream *s, int64_t *admitted, int64_t *frames, int64_t *integrations,
                    int64_t *dropped);

/* Scheduler counters, written to out[0 .. min(n, 9)): admitted channels, frames processed,
 * integrations completed, frames dropped, scheduler passes that launched work, launch groups,
 * passes that held back to fill a batch, host nanoseconds spent enqueuing launches,
 * admissions refused for the HBM budget.  Returns the number of values written or a
 * negative XE_* code. */
int xe_stream_counters(xe_stream *s, int64_t *out, int n);

/* Checkpoint of one channel's open integration.  The paper's X-engine nodes are diskless
 * and keep no such state (section 3.1); this lets a server that restarts, or moves a channel
 * to another GPU, continue an integration instead of dropping it.  Frame sequence numbers
 * count from the channel's first frame, so integration k holds frames
 * [k * F, (k + 1) * F) with F = integ_T / frame_T. */
typedef struct xe_snapshot {
    int64_t integ_index;      /* integration the sums belong to */
    int64_t next_seq;         /* sequence number of the first frame not in the sums
                                 (= integ_index * F + frames) */
    int64_t frames;           /* frames of the integration covered, lost ones included (< F) */
    int64_t n_samples;        /* samples in the sums (frames that arrived x frame_T) */
    int lost;                 /* 1 if a frame of the integration was lost */
    int64_t t_first_arrival_ns; /* arrival time of the integration's first frame */
} xe_snapshot;

/* Copy channel `chan`'s open integration to host_vis (HOST memory, [B][2] int32, the
 * xe_result layout; zeros when no frame of it has been correlated yet) and its bookkeeping
 * to *info.  The sums cover the frames the scheduler has launched (frames pushed but still
 * queued are not in them and stay queued); integrations go on running.  Waits at most
 * timeout_ms for the scheduler and at most as long again for the copy.  Returns XE_OK,
 * XE_EINVAL (null pointers, channel not admitted or evicted meanwhile), XE_ETIMEOUT,
 * XE_ENOMEM, XE_ECUDA or XE_ECLOSED. */
int xe_stream_snapshot(xe_stream *s, int chan, int32_t *host_vis, xe_snapshot *info, int timeout_ms);

/* Load a snapshot into channel `chan`, which must have been admitted and have taken no frame
 * yet, on a stream with the same N, frame_T and integ_T.  The channel then expects frame
 * info->next_seq next and completes integration info->integ_index with the sums of
 * host_vis (HOST memory, [B][2] int32; may be NULL when info->n_samples == 0) added in.
 * Returns XE_OK, XE_EINVAL (channel not fresh, or info inconsistent with this stream's frame
 * and integration lengths), XE_ECUDA or XE_ECLOSED. */
int xe_stream_restore(xe_stream *s, int chan, const int32_t *host_vis, const xe_snapshot *info);

/* Close the stream: stops its threads, waits (bounded) for in-flight work and frees all
 * of its memory.  Results not yet released become invalid. */
void xe_stream_close(xe_stream *s);

/* ---- allocation-free correlation ------------------------------------------------------ */

/* Size of the fixed scratch array libxe.so compiles in for xe_correlate_noalloc (device
 * memory every GPU that loads the library holds until the process exits), and the most
 * triangle tiles one call may have. */
#define XE_NOALLOC_SCRATCH_BYTES (32u << 20)
#define XE_NOALLOC_MAX_TILES 4096

/* xe_correlate_noalloc: as xe_correlate_async with XE_ALGO_TC, for callers that cannot
 * call cudaMalloc (a real-time pipeline that forbids allocation once running, or a host
 * application whose own pool owns all device memory).  It allocates nothing: its scratch
 * (staged operands, tile table, status words) lives in one fixed 32 MiB device array
 * compiled into the library.  There is no counterpart in the paper; this is an interface
 * for constrained callers.
 *
 * in, vis: caller-owned device pointers, formats as above; enqueued on `stream`.
 * The integration runs in windows of as many 64-sample blocks as the array holds staged
 * operands for (2 * n_chan * ceil(N/256)*256 bytes per sample; e.g. 8128 samples for N=2048
 * and one channel), at most option "exact_chunk_t" samples each; every window after the
 * first adds into vis.  Operands are always FP8 e4m3 (option "operand_bytes" is not used
 * here; the result is the same exact integers).
 * Limits: T <= XE_MAX_T (else XE_EOVERFLOW); the staged operands of one 64-sample block,
 * 2 * n_chan * ceil(N/256)*256 * 64 bytes, must fit the array; at most
 * XE_NOALLOC_MAX_TILES triangle tiles.  Larger requests return XE_EINVAL with a message in
 * xe_last_error() and enqueue nothing.
 * The first call on a device (with that device current) looks up the array's device
 * address with cudaGetSymbolAddress and clears its status words; make that first call
 * before any stream capture.
 * Every call shares the one array, which keeps the previous call's contents: calls that
 * overlap on the GPU (other streams, unordered threads) race and give wrong results.
 * A device-side bounded wait that gives up leaves that call's visibilities invalid; this
 * call does not wait for its kernels, so it cannot return XE_ETIMEOUT itself: the timeout
 * is kept in the array (a later call latches it instead of erasing it) until
 * xe_noalloc_status reports it.
 * Returns XE_OK, XE_EINVAL, XE_EOVERFLOW, XE_ECUDA or XE_ENODEV. */
int xe_correlate_noalloc(const uint8_t *in, int N, int64_t T, int n_chan, int32_t *vis,
                         void *stream);

/* Synchronise `stream`, then read and clear the status words of xe_correlate_noalloc's
 * fixed array on the current device.  Returns XE_ETIMEOUT if any xe_correlate_noalloc call
 * since the last status query gave up on a bounded device wait (its visibilities are
 * invalid), else XE_OK; or XE_ECUDA / XE_ENODEV.  Allocates nothing. */
int xe_noalloc_status(void *stream);

/* ---- diagnostics -------------------------------------------------------------------- */

/* Measure a tensor-core ceiling on the current device: kind 0 = tcgen05 kind::f8f6f4
 * (e4m3, M=128 N=256 K=32, operands resident in shared memory), kind 1 = mma.sync
 * m16n8k32 s8, kind 2 = kind 0 while bulk copies stream 48 KB rounds into shared memory
 * as fast as they complete from a 1 MB source, kind 3 = the same from a 64 MB source
 * (*aux receives that fill rate in GB/s; aux may be NULL).
 * Writes dense TFLOP/s (2 operations per multiply-accumulate) to *tflops.  Each loop runs
 * for a few milliseconds.  Returns XE_OK or an XE_* code. */
int xe_peak_probe(int kind, double *tflops, double *aux);

/* Tuning / diagnostic options (process-wide; take effect on the next call):
 *   "operand_bytes"  1 = FP8 e4m3 tensor-core operands (default), 2 = f16 operands;
 *   "exact_chunk_t"  samples summed by one f32 tensor-memory accumulation before the
 *                    partial sum is moved to int32 (64 .. 131072, default 131072);
 *   "n_cta"          persistent CTAs per launch (0 = one per SM, the default);
 *   "sched"          triangle schedule, -1 = automatic (default), 0..4 as in xe_plan_dump;
 *   "tile_n"         tile width 0 = automatic (default), 128 or 256;
 *   "autotune"       1 = time every (tile width, schedule) candidate the first time a
 *                    batch shape is correlated and keep the fastest for that shape;
 *   "timing"         1 = record device times of each call (see xe_last_timing);
 *   "checks"         1 = before every tensor-core correlation launch, one block checks its
 *                    descriptors on the device (job shapes, operand planes inside the
 *                    staging scratch, every tile, k-range and workspace slot of the plan
 *                    inside what was allocated) and on a violation sets the stream's status
 *                    word instead of trapping; the staging and correlation kernels then
 *                    return at once and xe_device_status (or the host-buffer calls) report
 *                    XE_ECHECK.  Default 0; the environment variable XE_CHECKS=1 turns it on
 *                    when the library loads;
 *   "check_corrupt"  test hook for "checks" (accepted only while it is on): 1 = the plan of
 *                    each launch claims no tiles, 2 = job 0's per-channel plane stride is off
 *                    by 64 bytes; both are caught before any kernel reads through them;
 *   "count_launch"   1 = the valid-sample counts of a masked call run as a second
 *                    correlation launch after the visibilities' (default); 0 = one mixed launch;
 *   "count_weight"   cost of a count job's k-iteration (two sample blocks) in schedule 4,
 *                    percent of a data job's (1 .. 100, default 75);
 *   "part_overhead"  modelled fix-up cost of one extra tile part in schedule 4, percent of
 *                    a whole tile (0 .. 100, default 2), never below the measured absolute
 *                    cost of a split (8 k-blocks for two parts, 20 per part beyond);
 *   "implicit_plans" 1 = batches of the streaming server run whole tiles dealt round-robin
 *                    over the CTAs, decoded in the kernel from the job table, with no plan
 *                    built on the host (default); 0 = host-built plans as for other calls;
 *   "host_chunk_t"   samples per chunk of xe_correlate_host's copy/correlate pipeline
 *                    (0 = one copy then one correlation; else a multiple of 64; default
 *                    8192);
 *   "host_async_chunk_t"  the same for xe_correlate_host_async (default 0: its calls
 *                    overlap one another, and whole copies and correlations measured faster).
 * Returns XE_OK or XE_EINVAL. */
int xe_set_option(const char *key, int64_t value);

/* ---- autotuning cache ------------------------------------------------------------- */

/* With option "autotune" on, the first call of each batch shape times the candidate plans
 * (tile width x schedule) and keeps the fastest.  A tuning cache file keeps those choices
 * across processes: entries are keyed by the GPU (device name with blanks as '_', and SM
 * count), the operand width, and per job N, the channel count, the schedule weight and a T
 * bucket (64-sample blocks rounded up to a power of two).  A later process that sets the
 * same file takes a cached shape's plan configuration without timing anything.
 * File format: one text line per entry,
 *   xe-tune 1 <gpu> <n_sm> <operand_bytes> <n_jobs> {<N> <T bucket> <C> <weight>}... <n_cta> <tile_n> <sched>
 * (weight 100 for plain jobs); malformed lines are skipped, later lines win. */

/* Use `path` as the tuning cache (NULL or "" = none): reads its entries now (a missing file
 * is empty) and appends every configuration tuned from now on.  Without this call the
 * environment variable XE_TUNE_CACHE names the file.  Returns XE_OK. */
int xe_tune_cache(const char *path);

/* Record a plan configuration for a batch shape of plain jobs on GPU `gpu` (no blanks) with
 * `n_sm` SMs, in memory and (with a cache file set) in the file: lets a deployment seed
 * tuned plans.  n_cta in [1, 4096], tile_n 128 or 256, sched 0..4.  Host-only.  Returns
 * XE_OK or XE_EINVAL. */
int xe_tune_store(const char *gpu, int n_sm, const int *N, const int64_t *T, const int *n_chan, int n_jobs,
                  int operand_bytes, int n_cta, int tile_n, int sched);

/* The cached configuration of a batch shape for GPU `gpu` with `n_sm` SMs.  Host-only.
 * Returns XE_OK, XE_EAGAIN if none is cached, or XE_EINVAL. */
int xe_tune_lookup(const char *gpu, int n_sm, const int *N, const int64_t *T, const int *n_chan, int n_jobs,
                   int operand_bytes, int *n_cta, int *tile_n, int *sched);

/* Candidate plans the autotuner has timed in this process, and tuned shapes it took from
 * the cache file instead.  Returns XE_OK. */
int xe_tune_stats(int64_t *timed_candidates, int64_t *from_cache);

/* Process-wide counters of host work that can stall a caller, in this order: batches
 * whose launch records were built, host ns spent building them, plans built for new batch
 * shapes, host ns spent on those plans, scratch regrowths and plan-cache trims (each of
 * these two synchronises the device).  Writes min(n, 6) values; returns that count or
 * XE_EINVAL. */
int xe_runtime_counters(int64_t *out, int n);

/* Synchronise `stream`, then read and clear the device status word of the scratch bound
 * to it.  Returns XE_OK, XE_ETIMEOUT if a kernel gave up on a bounded wait (its output is
 * then invalid), or XE_ECHECK if a descriptor check failed (option "checks"; the launch
 * wrote nothing). */
int xe_device_status(void *stream);

/* The library keeps scratch memory (staged operand planes, workspace, counters, a status
 * word) per CUDA stream it has run on.  Call this before destroying a stream the library
 * was used on, to free that memory: it waits for the stream's work first.  A later call on
 * a stream with the same handle allocates afresh.  The streaming server does this for its
 * own streams.  Returns XE_OK (also for a stream the library never used), XE_ECUDA or
 * XE_ENODEV. */
int xe_release_stream(void *stream);

/* Streaming multiprocessors of the current device.  Returns an XE_* code. */
int xe_device_info(int *n_sm);

/* Bit pattern of the small integer v in [-16, 16] as an MMA operand: e4m3 when
 * elem_bytes == 1, f16 when elem_bytes == 2.  Host-only; for tests of the encoder. */
uint32_t xe_debug_operand_code(int v, int elem_bytes);

/* Record CUDA events around the kernels of the following calls of this process (enable
 * = 1) or not (0, the default: the events and the host waits on them add a few
 * microseconds to every call).  Returns XE_OK. */
int xe_set_timing(int enable);

/* Device time in milliseconds of the kernels of the last xe_correlate* call on this
 * thread, split as {stage, correlate}; filled only when timing was enabled with
 * xe_set_timing(1).  Waits for that call's events.  Returns XE_OK or XE_EAGAIN if nothing
 * was recorded. */
int xe_last_timing(float *stage_ms, float *correlate_ms);
/* As xe_last_timing, plus the device time of work after the correlation kernel for the
 * valid-sample counts of a masked call.  The count jobs run inside the correlation kernel
 * and write the counts directly, so this is 0 (kept for callers that split the time). */
int xe_last_timing_counts(float *stage_ms, float *correlate_ms, float *count_ms);

#ifdef __cplusplus
}
#endif
#endif /* XE_H */
