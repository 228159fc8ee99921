/*
 * xe_oracle.c -- CPU oracle for the X-engine correlation.  TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may
 * load this library.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (Denman et al., "A GPU Spatial Processing System for CHIME",
 * arXiv 2005.09481):
 *   - section 1 (introduction): the signal of each receiver is correlated against every
 *     other receiver, per frequency channel, after channelisation ("FX" correlator);
 *   - section 2.2 ("Computational Requirements"): the X stage includes the
 *     autocorrelations, i.e. N(N+1)/2 complex multiply-accumulates per sample, and the
 *     samples carry 4 bits of real and 4 bits of imaginary part (d = 8 bits);
 *   - section 2.3 ("GPU Processing Nodes"): frequency channels are processed
 *     independently.
 * The quantity itself is the visibility V_ij = sum_t x_i(t) * conj(x_j(t)) for i <= j,
 * accumulated exactly in integers.  The paper prints no formula for V_ij; the readings
 * taken where it is silent are:
 *   (R1) byte layout: high nibble = real part, low nibble = imaginary part;
 *   (R2) nibble encoding: two's complement, values -8..7;
 *   (R3) conjugation on the second index: x_i * conj(x_j);
 *   (R4) output: row-major upper triangle including the diagonal,
 *        idx(i,j) = i*N - i*(i-1)/2 + (j - i), {Re, Im} interleaved.
 *
 * This file is the plain definition: decode each byte, then a triple loop over
 * (i <= j, t) accumulating in int64.  No blocking, no reordering, no vectorisation
 * tricks.  OpenMP only distributes the independent rows i over cores.
 */
#include <stdint.h>
#include <stddef.h>

/* (R1), (R2): one packed sample byte -> (re, im), each a two's-complement 4-bit integer. */
static void decode_sample(uint8_t byte, int64_t *re, int64_t *im)
{
    int64_t hi = (byte >> 4) & 0xF;
    int64_t lo = byte & 0xF;
    *re = (hi >= 8) ? hi - 16 : hi;
    *im = (lo >= 8) ? lo - 16 : lo;
}

/* Exported decode, for the decode-table pin (all 256 bytes). */
void xe_oracle_decode(const uint8_t *bytes, int64_t n, int64_t *re, int64_t *im)
{
    for (int64_t k = 0; k < n; ++k)
        decode_sample(bytes[k], &re[k], &im[k]);
}

/* (R4): position of baseline (i, j), i <= j, in the packed upper triangle. */
int64_t xe_oracle_tri_index(int64_t N, int64_t i, int64_t j)
{
    return i * N - (i * (i - 1)) / 2 + (j - i);
}

/* Number of baselines including autocorrelations, N(N+1)/2 (section 2.2). */
int64_t xe_oracle_n_baselines(int64_t N)
{
    return N * (N + 1) / 2;
}

/* One visibility: V_ij = sum_t x_i(t) conj(x_j(t)) over channel data in[t][n].
 * Re{(a + ib)(p - iq)} = a p + b q,  Im{(a + ib)(p - iq)} = b p - a q. */
static void visibility(const uint8_t *chan, int64_t N, int64_t T, int64_t i, int64_t j,
                       int64_t *sr, int64_t *si)
{
    int64_t acc_re = 0, acc_im = 0;
    for (int64_t t = 0; t < T; ++t) {
        int64_t a, b, p, q;
        decode_sample(chan[t * N + i], &a, &b);
        decode_sample(chan[t * N + j], &p, &q);
        acc_re += a * p + b * q;
        acc_im += b * p - a * q;
    }
    *sr = acc_re;
    *si = acc_im;
}

/*
 * Full correlation.  in: uint8 [C][T][N]; vis: int64 [C][N(N+1)/2][2].
 * Returns 0, or -1 on bad sizes.
 */
int xe_oracle_correlate(const uint8_t *in, int64_t N, int64_t T, int64_t C, int64_t *vis)
{
    if (N < 1 || T < 0 || C < 1 || !in || !vis)
        return -1;
    const int64_t B = xe_oracle_n_baselines(N);
    for (int64_t c = 0; c < C; ++c) {
        const uint8_t *chan = in + c * T * N;
        int64_t *out = vis + c * B * 2;
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t i = 0; i < N; ++i) {
            for (int64_t j = i; j < N; ++j) {
                int64_t sr, si;
                visibility(chan, N, T, i, j, &sr, &si);
                int64_t k = xe_oracle_tri_index(N, i, j);
                out[2 * k + 0] = sr;
                out[2 * k + 1] = si;
            }
        }
    }
    return 0;
}

/*
 * Selected baselines only (for sampled checks at full size): for each k,
 * (c[k], i[k], j[k]) with i <= j; out: int64 [n][2].  Returns 0, or -1 on a bad pair.
 */
int xe_oracle_pairs(const uint8_t *in, int64_t N, int64_t T, int64_t n,
                    const int64_t *c, const int64_t *i, const int64_t *j, int64_t *out)
{
    for (int64_t k = 0; k < n; ++k)
        if (i[k] < 0 || j[k] < i[k] || j[k] >= N || c[k] < 0)
            return -1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; ++k) {
        int64_t sr, si;
        visibility(in + c[k] * T * N, N, T, i[k], j[k], &sr, &si);
        out[2 * k + 0] = sr;
        out[2 * k + 1] = si;
    }
    return 0;
}

/*
 * Flag-masked correlation, optional offset-binary samples.
 *
 * Denman et al. 2020, section 2.2 and Table tab:data-flow: the F-engine sends flags and
 * metadata with the voltages (644 B per 4096 B of data), and RFI excision runs on the GPU
 * before the correlation (Table tab:computing).  Readings (the paper gives no format):
 *   (R10) flags are validity bits per (time sample, input): byte t*ceil(N/8) + n/8 of a
 *         channel, bit n%8; 1 = valid.  A flagged sample contributes nothing, i.e.
 *         V_ij = sum_t f_i(t) f_j(t) x_i(t) conj(x_j(t));  flags == NULL means all valid.
 *   (R11) encoding 1 = offset binary: each nibble u encodes the value u - 8 (encoding 0 is
 *         the two's complement of R2).
 */
static void decode_sample_enc(uint8_t byte, int encoding, int64_t *re, int64_t *im)
{
    if (encoding == 1) {
        *re = (int64_t)((byte >> 4) & 0xF) - 8;
        *im = (int64_t)(byte & 0xF) - 8;
    } else {
        decode_sample(byte, re, im);
    }
}

static int flag_valid(const uint8_t *chan_flags, int64_t N, int64_t t, int64_t n)
{
    if (!chan_flags) return 1;
    const int64_t row = (N + 7) / 8;
    return (chan_flags[t * row + n / 8] >> (n % 8)) & 1;
}

/* in: uint8 [C][T][N]; flags: uint8 [C][T][ceil(N/8)] or NULL; vis: int64 [C][B][2]. */
int xe_oracle_correlate_masked(const uint8_t *in, const uint8_t *flags, int64_t N, int64_t T,
                               int64_t C, int encoding, int64_t *vis)
{
    if (N < 1 || T < 0 || C < 1 || !in || !vis || (encoding != 0 && encoding != 1))
        return -1;
    const int64_t B = xe_oracle_n_baselines(N);
    const int64_t frow = (N + 7) / 8;
    for (int64_t c = 0; c < C; ++c) {
        const uint8_t *chan = in + c * T * N;
        const uint8_t *cf = flags ? flags + c * T * frow : NULL;
        int64_t *out = vis + c * B * 2;
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t i = 0; i < N; ++i) {
            for (int64_t j = i; j < N; ++j) {
                int64_t acc_re = 0, acc_im = 0;
                for (int64_t t = 0; t < T; ++t) {
                    if (!flag_valid(cf, N, t, i) || !flag_valid(cf, N, t, j)) continue;
                    int64_t a, b, p, q;
                    decode_sample_enc(chan[t * N + i], encoding, &a, &b);
                    decode_sample_enc(chan[t * N + j], encoding, &p, &q);
                    acc_re += a * p + b * q;
                    acc_im += b * p - a * q;
                }
                int64_t k = xe_oracle_tri_index(N, i, j);
                out[2 * k + 0] = acc_re;
                out[2 * k + 1] = acc_im;
            }
        }
    }
    return 0;
}

/* Valid-sample counts per baseline: n_ij = sum_t f_i(t) f_j(t); counts int64 [C][B]. */
int xe_oracle_flag_counts(const uint8_t *flags, int64_t N, int64_t T, int64_t C, int64_t *counts)
{
    if (N < 1 || T < 0 || C < 1 || !flags || !counts)
        return -1;
    const int64_t B = xe_oracle_n_baselines(N);
    const int64_t frow = (N + 7) / 8;
    for (int64_t c = 0; c < C; ++c) {
        const uint8_t *cf = flags + c * T * frow;
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t i = 0; i < N; ++i)
            for (int64_t j = i; j < N; ++j) {
                int64_t n = 0;
                for (int64_t t = 0; t < T; ++t)
                    n += flag_valid(cf, N, t, i) & flag_valid(cf, N, t, j);
                counts[c * B + xe_oracle_tri_index(N, i, j)] = n;
            }
    }
    return 0;
}

/*
 * Phased-array beams (section 2.1: besides the correlation, the X-engine nodes form 10
 * phased-array beams for pulsar timing; Table tab:computing lists "Pulsar Beamforming").
 * The paper gives no formula; the reading (R12) is the weighted coherent sum over inputs,
 *     y_b(t) = sum_i w_{b,i} x_i(t),
 * with complex integer weights w (int8 real and imaginary parts), exact in integers.
 * in: uint8 [C][T][N]; w: int8 [B][N][2] {re, im}; y: int64 [C][T][B][2].
 */
int xe_oracle_beamform(const uint8_t *in, const int8_t *w, int64_t N, int64_t T, int64_t C,
                       int64_t B, int64_t *y)
{
    if (N < 1 || T < 0 || C < 1 || B < 1 || !in || !w || !y)
        return -1;
    for (int64_t c = 0; c < C; ++c) {
        const uint8_t *chan = in + c * T * N;
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < T; ++t) {
            for (int64_t b = 0; b < B; ++b) {
                int64_t acc_re = 0, acc_im = 0;
                for (int64_t i = 0; i < N; ++i) {
                    int64_t a, bb;
                    decode_sample(chan[t * N + i], &a, &bb);
                    const int64_t wr = w[(b * N + i) * 2 + 0], wi = w[(b * N + i) * 2 + 1];
                    acc_re += wr * a - wi * bb;     /* Re{(wr + i wi)(a + i bb)} */
                    acc_im += wr * bb + wi * a;     /* Im{(wr + i wi)(a + i bb)} */
                }
                y[((c * T + t) * B + b) * 2 + 0] = acc_re;
                y[((c * T + t) * B + b) * 2 + 1] = acc_im;
            }
        }
    }
    return 0;
}

/*
 * Corner turn at the X-engine (section 2.1: the F-engine's inter-crate stage delivers
 * "bundles" of four frequency channels, each bundle holding one cylinder's inputs; each GPU
 * node combines four bundles into full-array data for those frequencies; section 2.3: the
 * node completes the transpose; Table tab:computing: "Re-Order and Pre-Sum").  Reading
 * (R13): a bundle is uint8 [T][n_freq][n_in] (time, then frequency, then the cylinder's
 * inputs); input n of the full array is cyl * n_in + i.
 *   bundles: uint8 [n_cyl][T][n_freq][n_in]  ->  frames: uint8 [n_freq][T][n_cyl * n_in]
 */
int xe_oracle_corner_turn(const uint8_t *bundles, int64_t n_cyl, int64_t n_freq, int64_t n_in,
                          int64_t T, uint8_t *frames)
{
    if (n_cyl < 1 || n_freq < 1 || n_in < 1 || T < 0 || !bundles || !frames)
        return -1;
    const int64_t N = n_cyl * n_in;
    for (int64_t f = 0; f < n_freq; ++f)
        for (int64_t t = 0; t < T; ++t)
            for (int64_t cyl = 0; cyl < n_cyl; ++cyl)
                for (int64_t i = 0; i < n_in; ++i)
                    frames[(f * T + t) * N + cyl * n_in + i] =
                        bundles[((cyl * T + t) * n_freq + f) * n_in + i];
    return 0;
}

/*
 * Pre-sum (reading R14): the per-input time sums s_n = sum_t x_n(t) of one block of samples,
 * re and im separately.  frames: uint8 [C][T][N]; sums: int64 [C][N][2].
 */
int xe_oracle_presum(const uint8_t *frames, int64_t N, int64_t T, int64_t C, int64_t *sums)
{
    if (N < 1 || T < 0 || C < 1 || !frames || !sums)
        return -1;
    for (int64_t c = 0; c < C; ++c)
        for (int64_t n = 0; n < N; ++n) {
            int64_t sr = 0, si = 0;
            for (int64_t t = 0; t < T; ++t) {
                int64_t a, b;
                decode_sample(frames[(c * T + t) * N + n], &a, &b);
                sr += a;
                si += b;
            }
            sums[(c * N + n) * 2 + 0] = sr;
            sums[(c * N + n) * 2 + 1] = si;
        }
    return 0;
}

/* Complex multiply-accumulates of one correlation: C * T * N(N+1)/2 (section 2.2). */
double xe_oracle_cmac(int64_t N, int64_t T, int64_t C)
{
    return (double)C * (double)T * (double)xe_oracle_n_baselines(N);
}

/* Threads OpenMP will use (reported beside the CPU timing). */
int xe_oracle_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set the threads of the OpenMP loops (n >= 1); returns the count now in force.  Used by a
 * timing harness whose launcher pinned OMP_NUM_THREADS to 1 for every process. */
int xe_oracle_set_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
    return xe_oracle_threads();
}
