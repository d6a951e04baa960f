/*
 * Plain reference Viterbi decoder for convolutional codes.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA decoder
 * is checked against.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * helper with the CUDA library: it builds its own trellis from the generator
 * polynomials and walks it in the most direct way.
 *
 * Paper: "High-Throughput Parallel Viterbi Decoder on GPU Tensor Cores"
 * (arXiv 2011.13579).
 *
 *   encoder / FSM ........ Sec. II-A, Eq. (encoder): output bit b is the XOR of
 *                          g_b[m] * in_{t-k+1+m}; g_{k-1} taps the current
 *                          input; the state is the previous k-1 inputs.
 *   branch metric ........ Sec. II-B, Eq. (BM): delta = sum_b (-1)^{alpha_out[b]} * l_t[b]
 *   path metric / ACS .... Sec. II-B, Eq. (PM): lambda^j_t = max_{i in prv(j)} (lambda^i_{t-1} + delta^{ij}_t)
 *   survivor ............. Sec. II-B, Eq. (SP0): phi^j_t = argmax of the same
 *   forward procedure .... Algorithm 1 (strict ">" keeps the first predecessor,
 *                          so a tie selects the second one)
 *   backward procedure ... Algorithm 2 (argmax at the last stage, then walk phi)
 *   frames with overlap .. Sec. III: the n stages are cut into frames of f
 *                          stages; neighbouring frames overlap so every frame
 *                          has history (read here as v stages on both sides).
 *
 * Readings where the paper is silent or ambiguous:
 *   - state s holds (in_{t-1} .. in_{t-k+1}) with in_{t-1} as its MSB; with
 *     input u the register is r = (u << (k-1)) | s, output bit b =
 *     parity(g_b & r), next state (u << (k-2)) | (s >> 1).  Predecessors of j
 *     are p0 = (j << 1) & mask (the "first", i') and p1 = p0 | 1 (i'').
 *   - Algorithm 1's strict ">" means a tie selects p1 (decision bit 1).
 *   - Algorithm 2's argmax takes the lowest state index among equal maxima.
 *   - positive LLR means bit 0; metrics are maximised.
 *   - a frame at the start of the stream starts from the reset state 0
 *     (others -infinity) unless the caller says the start is unknown; every
 *     other frame starts from all-zero metrics (Algorithm 1 initialises the
 *     path metrics to zero).
 *   - a terminated stream has k-1 zero tail inputs; a frame that reaches the
 *     end of a terminated stream traces back from state 0.
 *   - puncturing: pattern rows are output bits b, columns the stage phase
 *     (t mod period); the received stream holds only the kept positions in
 *     stage-major, b-ascending order; erased positions get LLR 0.
 *   - decoded bits are packed LSB-first: bit t goes to word t>>5, bit t&31.
 *
 * Arithmetic: int64 path metrics for integer LLRs (no normalisation, so no
 * overflow is possible for |LLR| < 2^24 and any practical length), double
 * for the floating-point study.  Radix-2 only.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <math.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OR_MAX_BETA 4
#define OR_MAX_PERIOD 8
#define OR_NEG_INF_I64 (INT64_MIN / 4)

typedef struct {
    int K;                                  /* constraint length k */
    int beta;                               /* outputs per input bit */
    uint32_t gens[OR_MAX_BETA];             /* generator polynomials, bit k-1 = current input */
    int period;                             /* puncture period, 1 = none */
    uint8_t punct[OR_MAX_BETA][OR_MAX_PERIOD]; /* 1 = transmitted */
} or_code;

static int or_parity(uint32_t x)
{
    int p = 0;
    while (x) { p ^= (int)(x & 1u); x >>= 1; }
    return p;
}

/* Branch output bit b for the branch leaving state s on input u (Eq. encoder). */
static int or_out_bit(const or_code *c, uint32_t s, int u, int b)
{
    uint32_t r = ((uint32_t)u << (c->K - 1)) | s;
    return or_parity(c->gens[b] & r);
}

/* Branch metric (Eq. BM) for integer LLRs of one stage. */
static int64_t or_bm_i64(const or_code *c, uint32_t s, int u, const int32_t *l)
{
    int64_t d = 0;
    for (int b = 0; b < c->beta; ++b)
        d += or_out_bit(c, s, u, b) ? -(int64_t)l[b] : (int64_t)l[b];
    return d;
}

static double or_bm_f64(const or_code *c, uint32_t s, int u, const double *l)
{
    double d = 0.0;
    for (int b = 0; b < c->beta; ++b)
        d += or_out_bit(c, s, u, b) ? -l[b] : l[b];
    return d;
}

/* ---------------------------------------------------------------- encoder */

/* Encodes n_in input bits (already including any tail) from state 0 and
 * writes beta output bits per stage, stage-major.  Used by the re-encoding
 * check; the FSM form of Sec. II-A. */
void or_encode(const or_code *c, const uint8_t *in, int64_t n_in, uint8_t *out)
{
    uint32_t s = 0;
    for (int64_t t = 0; t < n_in; ++t) {
        int u = in[t] & 1;
        for (int b = 0; b < c->beta; ++b)
            out[t * c->beta + b] = (uint8_t)or_out_bit(c, s, u, b);
        s = ((uint32_t)u << (c->K - 2)) | (s >> 1);
    }
}

/* Encodes from an arbitrary origin state (for re-encoding a survivor path). */
void or_encode_from(const or_code *c, uint32_t s, const uint8_t *in, int64_t n_in, uint8_t *out)
{
    for (int64_t t = 0; t < n_in; ++t) {
        int u = in[t] & 1;
        for (int b = 0; b < c->beta; ++b)
            out[t * c->beta + b] = (uint8_t)or_out_bit(c, s, u, b);
        s = ((uint32_t)u << (c->K - 2)) | (s >> 1);
    }
}

/* ------------------------------------------------------------- depuncture */

/* Expands a kept-only received stream to beta LLRs per stage for T stages;
 * erased positions get 0.  Returns the number of kept values consumed, or
 * -1 if the input is too short. */
int64_t or_depuncture_i32(const or_code *c, const int32_t *kept, int64_t n_kept,
                          int64_t T, int32_t *full)
{
    int64_t k = 0;
    for (int64_t t = 0; t < T; ++t) {
        int ph = (int)(t % c->period);
        for (int b = 0; b < c->beta; ++b) {
            if (c->punct[b][ph]) {
                if (k >= n_kept) return -1;
                full[t * c->beta + b] = kept[k++];
            } else {
                full[t * c->beta + b] = 0;
            }
        }
    }
    return k;
}

int64_t or_depuncture_f64(const or_code *c, const double *kept, int64_t n_kept,
                          int64_t T, double *full)
{
    int64_t k = 0;
    for (int64_t t = 0; t < T; ++t) {
        int ph = (int)(t % c->period);
        for (int b = 0; b < c->beta; ++b) {
            if (c->punct[b][ph]) {
                if (k >= n_kept) return -1;
                full[t * c->beta + b] = kept[k++];
            } else {
                full[t * c->beta + b] = 0.0;
            }
        }
    }
    return k;
}

/* ---------------------------------------------------------------- windows */

/* Frame geometry: frame s decodes stages [o, e) and runs the trellis over
 * [a, b), i.e. v extra stages on each side, clipped to the stream. */
typedef struct { int64_t a, b, o, e; } or_window;

static or_window or_window_of(int64_t s, int64_t n_info, int64_t T, int64_t f, int64_t v)
{
    or_window w;
    w.o = s * f;
    w.e = (s + 1) * f < n_info ? (s + 1) * f : n_info;
    w.a = w.o - v > 0 ? w.o - v : 0;
    w.b = (s + 1) * f + v < T ? (s + 1) * f + v : T;
    return w;
}

int64_t or_num_windows(int64_t n_info, int64_t f)
{
    return n_info <= 0 ? 0 : (n_info + f - 1) / f;
}

/* ------------------------------------------------------ one window, int64 */

typedef struct {
    const or_code *c;
    const int32_t *llr;      /* [T][beta], depunctured */
    int64_t n_info, T, f, v;
    int terminated, start_unknown;
    uint8_t *bits;           /* [n_info] decoded bits, one per byte */
    int64_t *final_pm;       /* [n_windows][NS] canonical final metrics, or NULL */
    int64_t n_windows;
    int nthreads, tid;
    int status;
} or_job_i64;

/* Runs Algorithms 1 and 2 over one frame.  pm, pm_new: NS int64; phi: W*NS bytes. */
static void or_window_i64(const or_job_i64 *J, int64_t s, int64_t *pm, int64_t *pm_new, uint8_t *phi)
{
    const or_code *c = J->c;
    const int NS = 1 << (c->K - 1);
    const uint32_t mask = (uint32_t)NS - 1u;
    or_window w = or_window_of(s, J->n_info, J->T, J->f, J->v);

    /* initial path metrics */
    for (int j = 0; j < NS; ++j) pm[j] = 0;
    if (w.a == 0 && !J->start_unknown)
        for (int j = 1; j < NS; ++j) pm[j] = OR_NEG_INF_I64;

    /* forward procedure (Algorithm 1) */
    for (int64_t t = w.a; t < w.b; ++t) {
        const int32_t *l = J->llr + t * c->beta;
        uint8_t *ph = phi + (t - w.a) * NS;
        for (uint32_t j = 0; j < (uint32_t)NS; ++j) {
            int u = (int)(j >> (c->K - 2));
            uint32_t p0 = (j << 1) & mask, p1 = p0 | 1u;
            int64_t c0 = pm[p0] + or_bm_i64(c, p0, u, l);
            int64_t c1 = pm[p1] + or_bm_i64(c, p1, u, l);
            if (c0 > c1) { pm_new[j] = c0; ph[j] = 0; }
            else         { pm_new[j] = c1; ph[j] = 1; }
        }
        memcpy(pm, pm_new, sizeof(int64_t) * (size_t)NS);
    }

    /* traceback start */
    uint32_t js = 0;
    if (!(w.b == J->T && J->terminated)) {
        for (uint32_t j = 1; j < (uint32_t)NS; ++j)
            if (pm[j] > pm[js]) js = j;
    }

    /* backward procedure (Algorithm 2) */
    for (int64_t t = w.b - 1; t >= w.o; --t) {
        if (t < w.e) J->bits[t] = (uint8_t)(js >> (c->K - 2));
        js = ((js << 1) & mask) | phi[(t - w.a) * NS + js];
    }

    if (J->final_pm) {
        int64_t mn = pm[0];
        for (int j = 1; j < NS; ++j) if (pm[j] < mn) mn = pm[j];
        for (int j = 0; j < NS; ++j) J->final_pm[s * NS + j] = pm[j] - mn;
    }
}

static void *or_worker_i64(void *arg)
{
    or_job_i64 *J = (or_job_i64 *)arg;
    const int NS = 1 << (J->c->K - 1);
    int64_t Wmax = J->f + 2 * J->v;
    if (Wmax > J->T) Wmax = J->T;
    int64_t *pm = (int64_t *)malloc(sizeof(int64_t) * (size_t)NS);
    int64_t *pm_new = (int64_t *)malloc(sizeof(int64_t) * (size_t)NS);
    uint8_t *phi = (uint8_t *)malloc((size_t)(Wmax > 0 ? Wmax : 1) * (size_t)NS);
    if (!pm || !pm_new || !phi) { J->status = -2; free(pm); free(pm_new); free(phi); return NULL; }
    for (int64_t s = J->tid; s < J->n_windows; s += J->nthreads)
        or_window_i64(J, s, pm, pm_new, phi);
    free(pm); free(pm_new); free(phi);
    return NULL;
}

static void or_pack_bits(const uint8_t *bits, int64_t n, uint32_t *words)
{
    int64_t nw = (n + 31) / 32;
    for (int64_t i = 0; i < nw; ++i) words[i] = 0;
    for (int64_t t = 0; t < n; ++t)
        if (bits[t]) words[t >> 5] |= 1u << (t & 31);
}

static int or_check_code(const or_code *c)
{
    if (c->K < 3 || c->K > 12 || c->beta < 1 || c->beta > OR_MAX_BETA) return -1;
    if (c->period < 1 || c->period > OR_MAX_PERIOD) return -1;
    return 0;
}

/*
 * Segmented decode with int64 metrics.
 *   llr:  [T][beta] depunctured LLRs, T = n_info + (terminated ? k-1 : 0)
 *   out:  ceil(n_info/32) packed words (LSB-first)
 *   final_pm: optional [n_windows][2^(k-1)] canonical metrics lambda - min lambda
 * Full-length decoding is the special case f >= n_info, v >= k-1.
 * Returns 0 on success.
 */
int or_decode_i64(const or_code *c, const int32_t *llr, int64_t n_info,
                  int terminated, int start_unknown, int64_t f, int64_t v,
                  uint32_t *out, int64_t *final_pm, int nthreads)
{
    if (or_check_code(c) || n_info < 0 || f <= 0 || v < 0) return -1;
    if (n_info == 0) return 0;
    int64_t T = n_info + (terminated ? c->K - 1 : 0);
    uint8_t *bits = (uint8_t *)calloc((size_t)n_info, 1);
    if (!bits) return -2;
    if (nthreads < 1) nthreads = 1;
    int64_t nwin = or_num_windows(n_info, f);
    if (nthreads > nwin) nthreads = (int)nwin;
    or_job_i64 *jobs = (or_job_i64 *)calloc((size_t)nthreads, sizeof(or_job_i64));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(bits); free(jobs); free(th); return -2; }
    for (int i = 0; i < nthreads; ++i) {
        or_job_i64 J = { c, llr, n_info, T, f, v, terminated, start_unknown, bits,
                         final_pm, nwin, nthreads, i, 0 };
        jobs[i] = J;
    }
    int rc = 0;
    if (nthreads == 1) {
        or_worker_i64(&jobs[0]);
    } else {
        for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, or_worker_i64, &jobs[i]);
        for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
    }
    for (int i = 0; i < nthreads; ++i) if (jobs[i].status) rc = jobs[i].status;
    if (rc == 0) or_pack_bits(bits, n_info, out);
    free(bits); free(jobs); free(th);
    return rc;
}

/* ------------------------------------------------------- one window, fp64 */

typedef struct {
    const or_code *c;
    const double *llr;
    int64_t n_info, T, f, v;
    int terminated, start_unknown;
    uint8_t *bits;
    double *min_gap;         /* [n_windows]: smallest |c1-c0| on the traced path, and the final argmax gap */
    double *max_abs_pm;      /* [n_windows]: largest |lambda| seen in the frame */
    int64_t n_windows;
    int nthreads, tid;
    int status;
} or_job_f64;

static void or_window_f64(const or_job_f64 *J, int64_t s, double *pm, double *pm_new,
                          uint8_t *phi, double *gap)
{
    const or_code *c = J->c;
    const int NS = 1 << (c->K - 1);
    const uint32_t mask = (uint32_t)NS - 1u;
    or_window w = or_window_of(s, J->n_info, J->T, J->f, J->v);
    double maxabs = 0.0;

    /* initial path metrics; the reset start uses a true -infinity, so a
     * candidate from an unreachable state never ties with a live one */
    for (int j = 0; j < NS; ++j) pm[j] = 0.0;
    if (w.a == 0 && !J->start_unknown)
        for (int j = 1; j < NS; ++j) pm[j] = -INFINITY;

    for (int64_t t = w.a; t < w.b; ++t) {
        const double *l = J->llr + t * c->beta;
        uint8_t *ph = phi + (t - w.a) * NS;
        double *gp = gap + (t - w.a) * NS;
        for (uint32_t j = 0; j < (uint32_t)NS; ++j) {
            int u = (int)(j >> (c->K - 2));
            uint32_t p0 = (j << 1) & mask, p1 = p0 | 1u;
            double c0 = pm[p0] + or_bm_f64(c, p0, u, l);
            double c1 = pm[p1] + or_bm_f64(c, p1, u, l);
            if (c0 > c1) { pm_new[j] = c0; ph[j] = 0; }
            else         { pm_new[j] = c1; ph[j] = 1; }
            /* decision gap; both -inf (unreachable state) gives NaN, which
             * the traced path never visits */
            gp[j] = fabs(c1 - c0);
        }
        memcpy(pm, pm_new, sizeof(double) * (size_t)NS);
        for (int j = 0; j < NS; ++j)
            if (isfinite(pm[j]) && fabs(pm[j]) > maxabs) maxabs = fabs(pm[j]);
    }

    uint32_t js = 0;
    double gmin = INFINITY;
    if (!(w.b == J->T && J->terminated)) {
        for (uint32_t j = 1; j < (uint32_t)NS; ++j)
            if (pm[j] > pm[js]) js = j;
        /* gap between the best and the runner-up final metric */
        for (uint32_t j = 0; j < (uint32_t)NS; ++j) {
            if (j == js) continue;
            double g = pm[js] - pm[j];
            if (g < gmin) gmin = g;
        }
    }
    for (int64_t t = w.b - 1; t >= w.o; --t) {
        if (t < w.e) J->bits[t] = (uint8_t)(js >> (c->K - 2));
        double g = gap[(t - w.a) * NS + js];
        if (g < gmin) gmin = g;
        js = ((js << 1) & mask) | phi[(t - w.a) * NS + js];
    }
    J->min_gap[s] = gmin;
    J->max_abs_pm[s] = maxabs;
}

static void *or_worker_f64(void *arg)
{
    or_job_f64 *J = (or_job_f64 *)arg;
    const int NS = 1 << (J->c->K - 1);
    int64_t Wmax = J->f + 2 * J->v;
    if (Wmax > J->T) Wmax = J->T;
    if (Wmax < 1) Wmax = 1;
    double *pm = (double *)malloc(sizeof(double) * (size_t)NS);
    double *pm_new = (double *)malloc(sizeof(double) * (size_t)NS);
    uint8_t *phi = (uint8_t *)malloc((size_t)Wmax * (size_t)NS);
    double *gap = (double *)malloc(sizeof(double) * (size_t)Wmax * (size_t)NS);
    if (!pm || !pm_new || !phi || !gap) {
        J->status = -2; free(pm); free(pm_new); free(phi); free(gap); return NULL;
    }
    for (int64_t s = J->tid; s < J->n_windows; s += J->nthreads)
        or_window_f64(J, s, pm, pm_new, phi, gap);
    free(pm); free(pm_new); free(phi); free(gap);
    return NULL;
}

/*
 * Segmented decode in double precision (fp64 path metrics), with the
 * -infinity start handled exactly.  Besides the bits it reports, per frame,
 * the smallest decision gap |c1 - c0| on the traced survivor path (including
 * the final argmax gap) and the largest |lambda| in the frame.
 */
int or_decode_f64(const or_code *c, const double *llr, int64_t n_info,
                  int terminated, int start_unknown, int64_t f, int64_t v,
                  uint32_t *out, double *min_gap, double *max_abs_pm, int nthreads)
{
    if (or_check_code(c) || n_info < 0 || f <= 0 || v < 0) return -1;
    if (n_info == 0) return 0;
    int64_t T = n_info + (terminated ? c->K - 1 : 0);
    uint8_t *bits = (uint8_t *)calloc((size_t)n_info, 1);
    if (!bits) return -2;
    if (nthreads < 1) nthreads = 1;
    int64_t nwin = or_num_windows(n_info, f);
    if (nthreads > nwin) nthreads = (int)nwin;
    or_job_f64 *jobs = (or_job_f64 *)calloc((size_t)nthreads, sizeof(or_job_f64));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(bits); free(jobs); free(th); return -2; }
    for (int i = 0; i < nthreads; ++i) {
        or_job_f64 J = { c, llr, n_info, T, f, v, terminated, start_unknown, bits,
                         min_gap, max_abs_pm, nwin, nthreads, i, 0 };
        jobs[i] = J;
    }
    int rc = 0;
    if (nthreads == 1) {
        or_worker_f64(&jobs[0]);
    } else {
        for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, or_worker_f64, &jobs[i]);
        for (int i = 0; i < nthreads; ++i) pthread_join(th[i], NULL);
    }
    for (int i = 0; i < nthreads; ++i) if (jobs[i].status) rc = jobs[i].status;
    if (rc == 0) or_pack_bits(bits, n_info, out);
    free(bits); free(jobs); free(th);
    return rc;
}

/* -------------------------------------------- full survivor path, int64 */

/*
 * For one frame s: runs the forward procedure and traces the survivor all the
 * way back to the frame's first stage a (not only to o).  Writes the input
 * bits along that path for stages [a, b) into path_bits[0 .. b-a), and
 * returns the origin state, the metric of the traceback start state and the
 * initial metric of the origin state.  Used by the re-encoding check: the
 * correlation of the re-encoded path over [a, b) must equal
 * end_metric - init_metric.  Returns the frame length b-a, or -1.
 */
int64_t or_trace_full_i64(const or_code *c, const int32_t *llr, int64_t n_info,
                          int terminated, int start_unknown, int64_t f, int64_t v,
                          int64_t s, uint8_t *path_bits, uint32_t *origin_state,
                          int64_t *end_metric, int64_t *init_metric)
{
    if (or_check_code(c) || f <= 0 || v < 0) return -1;
    int64_t T = n_info + (terminated ? c->K - 1 : 0);
    if (s < 0 || s >= or_num_windows(n_info, f)) return -1;
    const int NS = 1 << (c->K - 1);
    const uint32_t mask = (uint32_t)NS - 1u;
    or_window w = or_window_of(s, n_info, T, f, v);
    int64_t W = w.b - w.a;
    int64_t *pm = (int64_t *)malloc(sizeof(int64_t) * (size_t)NS);
    int64_t *pm_new = (int64_t *)malloc(sizeof(int64_t) * (size_t)NS);
    int64_t *pm0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)NS);
    uint8_t *phi = (uint8_t *)malloc((size_t)(W > 0 ? W : 1) * (size_t)NS);
    if (!pm || !pm_new || !pm0 || !phi) { free(pm); free(pm_new); free(pm0); free(phi); return -1; }
    for (int j = 0; j < NS; ++j) pm[j] = 0;
    if (w.a == 0 && !start_unknown)
        for (int j = 1; j < NS; ++j) pm[j] = OR_NEG_INF_I64;
    memcpy(pm0, pm, sizeof(int64_t) * (size_t)NS);
    for (int64_t t = w.a; t < w.b; ++t) {
        const int32_t *l = llr + t * c->beta;
        for (uint32_t j = 0; j < (uint32_t)NS; ++j) {
            int u = (int)(j >> (c->K - 2));
            uint32_t p0 = (j << 1) & mask, p1 = p0 | 1u;
            int64_t c0 = pm[p0] + or_bm_i64(c, p0, u, l);
            int64_t c1 = pm[p1] + or_bm_i64(c, p1, u, l);
            if (c0 > c1) { pm_new[j] = c0; phi[(t - w.a) * NS + j] = 0; }
            else         { pm_new[j] = c1; phi[(t - w.a) * NS + j] = 1; }
        }
        memcpy(pm, pm_new, sizeof(int64_t) * (size_t)NS);
    }
    uint32_t js = 0;
    if (!(w.b == T && terminated)) {
        for (uint32_t j = 1; j < (uint32_t)NS; ++j)
            if (pm[j] > pm[js]) js = j;
    }
    *end_metric = pm[js];
    for (int64_t t = w.b - 1; t >= w.a; --t) {
        path_bits[t - w.a] = (uint8_t)(js >> (c->K - 2));
        js = ((js << 1) & mask) | phi[(t - w.a) * NS + js];
    }
    *origin_state = js;
    *init_metric = pm0[js];
    free(pm); free(pm_new); free(pm0); free(phi);
    return W;
}

/* ------------------------------------------------ selected frames, int64 */

/*
 * Decodes only the listed frames of a stream (same rules and arithmetic as
 * or_decode_i64).  bits_out: [n_sel][f] bytes, frame k's decided bits of
 * stages [o, e) at bits_out[k*f ..]; final_pm: optional [n_sel][NS].
 */
int or_decode_frames_i64(const or_code *c, const int32_t *llr, int64_t n_info,
                         int terminated, int start_unknown, int64_t f, int64_t v,
                         const int64_t *frames, int64_t n_sel, uint8_t *bits_out,
                         int64_t *final_pm)
{
    if (or_check_code(c) || n_info <= 0 || f <= 0 || v < 0) return -1;
    const int NS = 1 << (c->K - 1);
    int64_t T = n_info + (terminated ? c->K - 1 : 0);
    int64_t nwin = or_num_windows(n_info, f);
    int64_t Wmax = f + 2 * v;
    if (Wmax > T) Wmax = T;
    uint8_t *bits = (uint8_t *)calloc((size_t)n_info, 1);
    int64_t *pm = (int64_t *)malloc(sizeof(int64_t) * (size_t)NS);
    int64_t *pm_new = (int64_t *)malloc(sizeof(int64_t) * (size_t)NS);
    int64_t *fpm = (int64_t *)malloc(sizeof(int64_t) * (size_t)NS * (size_t)nwin);
    uint8_t *phi = (uint8_t *)malloc((size_t)Wmax * (size_t)NS);
    int rc = 0;
    if (!bits || !pm || !pm_new || !fpm || !phi) { rc = -2; goto done; }
    for (int64_t k = 0; k < n_sel; ++k) {
        int64_t s = frames[k];
        if (s < 0 || s >= nwin) { rc = -1; goto done; }
        or_job_i64 J = { c, llr, n_info, T, f, v, terminated, start_unknown, bits,
                         fpm, nwin, 1, 0, 0 };
        or_window_i64(&J, s, pm, pm_new, phi);
        or_window w = or_window_of(s, n_info, T, f, v);
        for (int64_t t = w.o; t < w.e; ++t) bits_out[k * f + (t - w.o)] = bits[t];
        if (final_pm)
            for (int j = 0; j < NS; ++j) final_pm[k * NS + j] = fpm[s * NS + j];
    }
done:
    free(bits); free(pm); free(pm_new); free(fpm); free(phi);
    return rc;
}

/* --------------------------------------------- hard decisions, Sec. II-C */

/*
 * Hard-decision decode (Sec. II-C, hard-decision mode: every received value
 * is a bit).  rx is [T][beta] with 0 or 1 per received bit and 2 at a
 * position the puncturing pattern erased (it carries no information).  The
 * branch metric is the Hamming distance between the branch output and the
 * received bits over the positions that are not erased; the path metric of
 * a state is the smallest accumulated distance of a path into it (the
 * forward procedure of Algorithm 1 with the distance minimised), and a tie
 * keeps the second predecessor, as the strict comparison of Algorithm 1
 * does; the traceback (Algorithm 2) starts from the state with the smallest
 * distance, the lowest index on ties, or from state 0 at a terminated end.
 * Frames as in or_decode_i64; a frame at stage 0 starts from state 0 (the
 * others at an infinite distance) unless the start is unknown.
 */
int or_decode_hard(const or_code *c, const uint8_t *rx, int64_t n_info, int terminated,
                   int start_unknown, int64_t f, int64_t v, uint32_t *out)
{
    if (or_check_code(c) || n_info < 0 || f <= 0 || v < 0) return -1;
    if (n_info == 0) return 0;
    const int NS = 1 << (c->K - 1);
    const uint32_t mask = (uint32_t)NS - 1u;
    const int64_t T = n_info + (terminated ? c->K - 1 : 0);
    const int64_t INF = INT64_MAX / 4;
    int64_t Wmax = f + 2 * v;
    if (Wmax > T) Wmax = T;
    uint8_t *bits = (uint8_t *)calloc((size_t)n_info, 1);
    int64_t *d = (int64_t *)malloc(sizeof(int64_t) * (size_t)NS);
    int64_t *dn = (int64_t *)malloc(sizeof(int64_t) * (size_t)NS);
    uint8_t *phi = (uint8_t *)malloc((size_t)(Wmax > 0 ? Wmax : 1) * (size_t)NS);
    if (!bits || !d || !dn || !phi) { free(bits); free(d); free(dn); free(phi); return -2; }
    const int64_t nwin = or_num_windows(n_info, f);
    for (int64_t s = 0; s < nwin; ++s) {
        or_window w = or_window_of(s, n_info, T, f, v);
        for (int j = 0; j < NS; ++j) d[j] = 0;
        if (w.a == 0 && !start_unknown)
            for (int j = 1; j < NS; ++j) d[j] = INF;
        for (int64_t t = w.a; t < w.b; ++t) {
            const uint8_t *r = rx + t * c->beta;
            uint8_t *ph = phi + (t - w.a) * NS;
            for (uint32_t j = 0; j < (uint32_t)NS; ++j) {
                const int u = (int)(j >> (c->K - 2));
                const uint32_t p0 = (j << 1) & mask, p1 = p0 | 1u;
                int64_t h0 = 0, h1 = 0;
                for (int b = 0; b < c->beta; ++b) {
                    if (r[b] > 1) continue;                       /* erased */
                    h0 += or_out_bit(c, p0, u, b) != r[b];
                    h1 += or_out_bit(c, p1, u, b) != r[b];
                }
                const int64_t c0 = d[p0] + h0, c1 = d[p1] + h1;
                if (c0 < c1) { dn[j] = c0; ph[j] = 0; }
                else         { dn[j] = c1; ph[j] = 1; }
            }
            memcpy(d, dn, sizeof(int64_t) * (size_t)NS);
        }
        uint32_t js = 0;
        if (!(w.b == T && terminated)) {
            for (uint32_t j = 1; j < (uint32_t)NS; ++j)
                if (d[j] < d[js]) js = j;
        }
        for (int64_t t = w.b - 1; t >= w.o; --t) {
            if (t < w.e) bits[t] = (uint8_t)(js >> (c->K - 2));
            js = ((js << 1) & mask) | phi[(t - w.a) * NS + js];
        }
    }
    or_pack_bits(bits, n_info, out);
    free(bits); free(d); free(dn); free(phi);
    return 0;
}

/* ------------------------------------ transmitter and channel, Sec. IX-B */

/*
 * Philox4x64-10, the counter-based generator of Salmon, Moraes, Dror and
 * Shaw ("Parallel random numbers: as easy as 1, 2, 3", SC 2011), written
 * from its published definition: ten rounds, each multiplying counter words
 * 0 and 2 by two fixed 64-bit constants into 128-bit products and mixing
 * the halves with counter words 1 and 3 and the key; the key is bumped by
 * two Weyl constants between rounds.
 */
static void or_mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    const uint64_t a0 = a & 0xFFFFFFFFu, a1 = a >> 32, b0 = b & 0xFFFFFFFFu, b1 = b >> 32;
    const uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
    const uint64_t mid = (p00 >> 32) + (p01 & 0xFFFFFFFFu) + (p10 & 0xFFFFFFFFu);
    *lo = (mid << 32) | (p00 & 0xFFFFFFFFu);
    *hi = p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
}

void or_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    uint64_t c[4] = { ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3] };
    uint64_t k[2] = { key_in[0], key_in[1] };
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        or_mulhilo64(0xD2E7470EE14C6C93ull, c[0], &hi0, &lo0);
        or_mulhilo64(0xCA5A826395121157ull, c[2], &hi1, &lo1);
        const uint64_t n0 = hi1 ^ c[1] ^ k[0], n1 = lo1, n2 = hi0 ^ c[3] ^ k[1], n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        if (r < 9) { k[0] += 0x9E3779B97F4A7C15ull; k[1] += 0xBB67AE8584CAA73Bull; }
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* Uniform in (0, 1] from the top 53 bits of a 64-bit word. */
static double or_unit(uint64_t x) { return (double)((x >> 11) + 1u) * 0x1.0p-53; }

/*
 * The four standard normals of counter block q of a stream: Philox4x64-10
 * with key (seed, stream_id) and counter (q, 0, 0, 0), turned into normals
 * by the Box-Muller transform on word pairs (0, 1) and (2, 3):
 * sqrt(-2 ln u) cos(2 pi v), sqrt(-2 ln u) sin(2 pi v).
 */
static void or_normals4(uint64_t seed, uint64_t stream_id, uint64_t q, double z[4])
{
    const uint64_t ctr[4] = { q, 0, 0, 0 }, key[2] = { seed, stream_id };
    uint64_t w[4];
    or_philox4x64(ctr, key, w);
    for (int p = 0; p < 2; ++p) {
        const double u = or_unit(w[2 * p]), v = or_unit(w[2 * p + 1]);
        const double rad = sqrt(-2.0 * log(u)), ang = 2.0 * M_PI * v;
        z[2 * p] = rad * cos(ang);
        z[2 * p + 1] = rad * sin(ang);
    }
}

/*
 * Transmitter and channel of the verification system (Sec. IX-B): the
 * information bits (one per byte) go through the encoder from state 0
 * (Sec. II-A, with k-1 zero tail bits when terminated), the puncturing
 * pattern keeps the transmitted positions (stage-major, b ascending), BPSK
 * maps bit 0 to +1 and 1 to -1, and AWGN adds sigma times the k-th normal
 * of the stream to the k-th kept value.  Writes the n_kept received samples
 * y (double) and returns n_kept, or -1.  Quantisation is the caller's.
 */
int64_t or_transmit(const or_code *c, const uint8_t *bits, int64_t n_info, int terminated, double sigma,
                    uint64_t seed, uint64_t stream_id, double *y, int64_t y_cap)
{
    if (or_check_code(c) || n_info < 0) return -1;
    const int64_t T = n_info + (terminated ? c->K - 1 : 0);
    uint8_t *in = (uint8_t *)calloc((size_t)(T > 0 ? T : 1), 1);
    uint8_t *cw = (uint8_t *)malloc((size_t)(T > 0 ? T : 1) * (size_t)c->beta);
    if (!in || !cw) { free(in); free(cw); return -1; }
    for (int64_t t = 0; t < n_info; ++t) in[t] = bits[t] & 1u;
    or_encode(c, in, T, cw);
    int64_t k = 0;
    double z[4];
    for (int64_t t = 0; t < T; ++t) {
        const int ph = (int)(t % c->period);
        for (int b = 0; b < c->beta; ++b) {
            if (!c->punct[b][ph]) continue;
            if (k >= y_cap) { free(in); free(cw); return -1; }
            if ((k & 3) == 0) or_normals4(seed, stream_id, (uint64_t)k >> 2, z);
            y[k] = (cw[t * c->beta + b] ? -1.0 : 1.0) + sigma * z[k & 3];
            ++k;
        }
    }
    free(in); free(cw);
    return k;
}

/* ------------------------------------------------ many packets, int64 */

/* One packet of a batch: its code, where its kept int8 values start in the
 * arena, its length and flags, the frame length and overlap to decode it
 * with, and where its packed output words go. */
typedef struct {
    int32_t code;
    int32_t terminated, start_unknown;
    int32_t pad;
    int64_t kept_off, n_info, f, v, out_word_off;
} or_packet;

typedef struct {
    const or_code *codes;
    const or_packet *pk;
    int64_t n_packets;
    const int8_t *arena;
    uint32_t *out;
    int nthreads, tid, status;
} or_batch_job;

static void *or_batch_worker(void *arg)
{
    or_batch_job *J = (or_batch_job *)arg;
    int32_t *kept = NULL, *full = NULL;
    int64_t cap_kept = 0, cap_full = 0;
    for (int64_t i = J->tid; i < J->n_packets; i += J->nthreads) {
        const or_packet *p = &J->pk[i];
        const or_code *c = &J->codes[p->code];
        const int64_t T = p->n_info + (p->terminated ? c->K - 1 : 0);
        int64_t n_kept = 0;
        for (int64_t t = 0; t < T; ++t)
            for (int b = 0; b < c->beta; ++b) n_kept += c->punct[b][t % c->period] != 0;
        if (n_kept > cap_kept) { free(kept); cap_kept = n_kept; kept = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap_kept); }
        if (T * c->beta > cap_full) { free(full); cap_full = T * c->beta; full = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap_full); }
        if (!kept || !full) { J->status = -2; break; }
        for (int64_t k = 0; k < n_kept; ++k) kept[k] = J->arena[p->kept_off + k];
        if (or_depuncture_i32(c, kept, n_kept, T, full) < 0) { J->status = -1; break; }
        const int rc = or_decode_i64(c, full, p->n_info, p->terminated, p->start_unknown, p->f, p->v,
                                     J->out + p->out_word_off, NULL, 1);
        if (rc) { J->status = rc; break; }
    }
    free(kept); free(full);
    return NULL;
}

/*
 * Decodes every packet of a batch with or_decode_i64 (Algorithms 1 and 2
 * over the frames of Sec. III, after depuncturing), packets spread over
 * nthreads host threads.  arena: the kept int8 values of all packets.
 */
int or_decode_packets_i64(const or_code *codes, const or_packet *pk, int64_t n_packets, const int8_t *arena,
                          uint32_t *out, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n_packets) nthreads = (int)(n_packets > 0 ? n_packets : 1);
    or_batch_job *jobs = (or_batch_job *)calloc((size_t)nthreads, sizeof(or_batch_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -2; }
    for (int i = 0; i < nthreads; ++i) {
        or_batch_job J = { codes, pk, n_packets, arena, out, nthreads, i, 0 };
        jobs[i] = J;
    }
    for (int i = 0; i < nthreads; ++i) pthread_create(&th[i], NULL, or_batch_worker, &jobs[i]);
    int rc = 0;
    for (int i = 0; i < nthreads; ++i) { pthread_join(th[i], NULL); if (jobs[i].status) rc = jobs[i].status; }
    free(jobs); free(th);
    return rc;
}
