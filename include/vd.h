/*
 * vd.h — C ABI of the GB300 soft-decision Viterbi decoder (libvd).
 *
 * Method: "High-Throughput Parallel Viterbi Decoder on GPU Tensor Cores",
 * arXiv 2011.13579.  The decoder computes, for a convolutional code of
 * constraint length k and beta generator polynomials (Sec. II-A, Eq. encoder):
 *   - branch metrics   delta^{ij}_t = sum_b (-1)^{alpha_out^{ij}[b]} l_t[b]      (Eq. BM)
 *   - path metrics     lambda^j_t = max_{i in prv(j)} lambda^i_{t-1} + delta^{ij}_t  (Eq. PM)
 *   - survivors        phi^j_t = argmax of the same                             (Eq. SP0)
 *   - the forward and backward procedures of Algorithms 1 and 2,
 *   - over frames of f stages that overlap their neighbours (Sec. III), here
 *     by v stages on each side,
 *   - in radix-2 (one stage per step) or radix-4 (two stages per step,
 *     Sec. VII, Eq. radix4:PM / radix4:SP0) form; both give identical bits.
 *
 * Conventions fixed by this library (the paper is silent on them):
 *   - generators are given as in the paper's octal notation, e.g. 0171, 0133
 *     for the (2,1,7) code; the most significant of the k bits taps the
 *     current input;
 *   - a positive LLR means bit 0 (Sec. II-C); metrics are maximised;
 *   - ties in the ACS select the odd predecessor 2f+1 (Algorithm 1 keeps the
 *     first candidate only if it is strictly larger); the final argmax of
 *     Algorithm 2 takes the lowest state index among equal metrics;
 *   - frame s decodes stages [s f, min(n_info, (s+1) f)) and runs the trellis
 *     over [max(0, s f - v), min(T, (s+1) f + v)), T = n_info (+ k-1 when
 *     terminated).  The frame at stage 0 starts from state 0 unless
 *     VD_START_UNKNOWN is given; other frames start from all-equal metrics;
 *     a frame that reaches the end of a terminated stream traces back from
 *     state 0, others from the best state;
 *   - decoded bit t is bit (t & 31) of word t >> 5 (LSB-first);
 *   - received LLRs are time-interleaved: l_t[0..beta-1] for t = 0, 1, ...;
 *     a punctured code transmits only the kept positions (stage-major, b
 *     ascending, pattern column t mod period) and the decoder inserts 0 at
 *     the erased ones.
 *
 * Ownership and threading: the caller owns every device buffer it passes and
 * the stream.  The library owns the vd_code objects and a per-device,
 * per-stream scratch pool for survivors, which it allocates on first use and
 * grows as needed (cudaMalloc), and frees in vd_release_scratch() or at
 * process exit.  Calls on one stream are ordered; calls on different streams
 * use different scratch buffers.  Launches are asynchronous on the given
 * stream; errors detected on the host are returned immediately.
 *
 * Errors: every function returns a vd_status; no exception, abort or exit
 * crosses the ABI.  vd_last_error() gives a message for the calling thread's
 * last failure.
 */
#ifndef VD_H
#define VD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VD_OK = 0,
    VD_EINVAL = -1,        /* bad argument (message in vd_last_error) */
    VD_ENOMEM = -2,        /* device or host allocation failed */
    VD_ECUDA = -3,         /* a CUDA runtime call failed */
    VD_EUNSUPPORTED = -4,  /* valid request the library has no kernel for */
    VD_ETIMEOUT = -5,      /* a bounded device wait ran out */
    VD_EBOUNDS = -6        /* a device-side bounds check fired */
} vd_status;

/* LLR element types */
enum { VD_LLR_S8 = 0,      /* int8 in [-127, 127] */
       VD_LLR_S4 = 1,      /* 4-bit in [-7, 7], two per byte, low nibble = earlier value */
       VD_LLR_F16 = 2,     /* IEEE half; metrics in fp32 */
       VD_LLR_HARD = 3 };  /* hard decisions (Sec. II-C, hard-decision mode): one bit per
                              received value, the detected code bit, eight per byte with the
                              earliest value in bit 0.  Decoded as LLR +1 (bit 0) or -1 (bit 1):
                              Eq. BM then gives beta - 2 x (Hamming distance between the branch
                              output and the received bits) on unpunctured stages, so the
                              maximum-metric path is the minimum-Hamming-distance path. */

/* flags */
enum { VD_TERMINATED = 1u,     /* stream ends with k-1 zero tail inputs (state 0) */
       VD_START_UNKNOWN = 2u,  /* do not assume the encoder starts in state 0 */
       VD_RETURN_PM = 4u };    /* reserved */

typedef struct vd_code vd_code;   /* opaque, owned by the library */

/* Decoder configuration chosen for one call (by the caller or the tuner). */
typedef struct vd_tune {
    int32_t f;         /* frame length (stages decoded per frame) */
    int32_t v;         /* overlap on each side */
    int32_t radix;     /* 2 or 4 */
    int32_t lanes;     /* threads per pair of frames: 1, 2, 4 (K=7), 4, 8 (K=9); 0 = default */
    int32_t threads;   /* threads per block */
    int32_t form;      /* vd_decode kernel form: 0 = by stream length, 1 = persistent
                          (warps pull tasks, interleaved traceback), 2 = one wave */
    int32_t reserved[2];
} vd_tune;

/*
 * Creates a code object.  Sec. II-A: constraint length K (3..9), beta
 * generator polynomials (2..4) each < 2^K with bit K-1 set (they tap the
 * current input; the corollary of Thm. 2 needs bit 0 set too, which holds for
 * all standard codes), given as integers whose octal spelling is the
 * paper's, e.g. 0171.  rate_num/rate_den: the nominal rate after puncturing
 * (1/beta when unpunctured); checked against the pattern.  puncture: NULL,
 * or a beta x period row-major 0/1 matrix (period 1..8, no all-zero column)
 * whose column t mod period says which outputs of stage t are transmitted.
 * On success *out owns a new object; on failure *out is NULL.
 * VD_EUNSUPPORTED: a code the library has no kernel for (see vd_code_supported).
 */
vd_status vd_code_create(vd_code **out, int K, int beta, const uint32_t *gens_octal,
                         int rate_num, int rate_den, const uint8_t *puncture, int period);

/* Frees a code object (NULL is ignored). */
void vd_code_destroy(vd_code *code);

/* 1 if the library has a decode kernel for (K, beta, generators), else 0. */
int vd_code_supported(int K, int beta, const uint32_t *gens_octal);

/*
 * Segmented (or full-length) stream decode, Algorithms 1-2 over the frames
 * of Sec. III.  Long int8 / 4-bit streams (at least one task of frame pairs
 * per resident warp) run a persistent kernel whose warps pull tasks and trace
 * one task back while decoding the next forward; shorter ones a kernel with
 * one frame pair per lane group (tune->form overrides).  Both give the same
 * bits.
 *   d_llr:    device pointer to the received LLRs of the whole stream, of
 *             llr_type, in transmitted order (kept positions only when the
 *             code is punctured): n_kept(T) values, T = n_info (+K-1 if
 *             VD_TERMINATED).  Any alignment.
 *   n_info:   information bits to decode (0 is a no-op).
 *   f, v:     frame length and overlap; f must be a multiple of 32 unless
 *             f >= n_info (a single frame).  v >= 0.  A full-length decode is
 *             f >= n_info with v >= K-1.
 *   radix:    2 or 4 (same bits either way).
 *   flags:    VD_TERMINATED, VD_START_UNKNOWN.
 *   d_out:    device pointer to ceil(n_info/32) uint32 words (written).
 *   d_pm:     NULL, or device pointer to n_frames x 2^(K-1) int32 receiving
 *             each frame's final metrics minus their minimum (for parity
 *             checks); n_frames = ceil(n_info/f).
 *   tune:     NULL for the library's choice, else lanes/threads to use
 *             (f, v and radix come from the arguments).
 *   stream:   a cudaStream_t (NULL = the legacy default stream).
 * Errors: VD_EINVAL for bad arguments, VD_EUNSUPPORTED for an LLR type the
 * code has no kernel for, VD_ENOMEM if scratch cannot grow, VD_ECUDA if a
 * launch fails.
 */
vd_status vd_decode(const vd_code *code, const void *d_llr, int llr_type, int64_t n_info,
                    int f, int v, int radix, uint32_t flags, uint32_t *d_out, int32_t *d_pm,
                    const vd_tune *tune, void *stream);

/*
 * vd_decode_host — vd_decode from and to host memory, for n_streams streams
 * of the same length and configuration: the library uploads each stream's
 * received values, decodes it (the persistent batch kernel, one stream per
 * launch on two alternating decode streams) and downloads its packed bits,
 * so stream i+1 uploads while stream i decodes and stream i's words come
 * back while later streams decode.  Same frames (Sec. III) and bits as
 * vd_decode; radix as given, the library's lane count.
 *   h_llr[i]: stream i's int8 LLRs (unpunctured), (n_info (+K-1)) x beta
 *             bytes; page-locked memory for the copies to overlap (pageable
 *             works, without overlap).
 *   h_out[i]: ceil(n_info/32) words (written when `stream` completes).
 * The device copies and the two plans live in library memory kept for this
 * stream (allocated on the first call and when the configuration changes).
 * Asynchronous: the caller waits on `stream`.  A call starts after earlier
 * work on `stream`, so consecutive calls on one stream do not overlap.
 * VD_EINVAL / VD_EUNSUPPORTED / VD_ENOMEM / VD_ECUDA as vd_decode.
 */
vd_status vd_decode_host(const vd_code *code, int n_streams, const void *const *h_llr, int llr_type,
                         int64_t n_info, int f, int v, int radix, uint32_t flags, uint32_t *const *h_out,
                         void *stream);

/*
 * The configuration vd_decode uses for this code and LLR type when its tune
 * argument is NULL: f, v and radix as given, and the lanes per frame pair and
 * threads per block it picks.  The decoded bits depend only on f, v and the
 * flags, so this is what a reference decoder needs to reproduce a call.
 * VD_EINVAL on bad arguments, VD_EUNSUPPORTED if there is no kernel.
 */
vd_status vd_get_tune(const vd_code *code, int llr_type, int f, int v, int radix, vd_tune *out);

/* ------------------------------------------------------------------ batches
 *
 * Many packets (terminated or not, of up to 16 codes, punctured or not,
 * int8 or 4-bit) decoded by one persistent launch per code kind.  Every frame
 * of every packet is cut as in vd_decode (Sec. III); the frames are sorted by
 * length, paired, and pulled by resident warps longest first.  The paper has
 * no batch API; this is the data-parallel form of its frame decoding applied
 * across packets.
 */
typedef struct vd_packet {
    int32_t code_id;         /* index into the codes array */
    int32_t llr_type;        /* VD_LLR_S8 or VD_LLR_S4 */
    int64_t llr_offset;      /* first received value of the packet in the LLR arena, counted in
                                values (bytes for int8, nibbles for 4-bit; must be even then) */
    int64_t n_info;          /* information bits, > 0 */
    uint32_t flags;          /* VD_TERMINATED, VD_START_UNKNOWN */
    int32_t f;               /* frame length; 0 = chosen by the library (then v is too) */
    int32_t v;               /* overlap on each side (used when f > 0) */
    int32_t reserved;
    int64_t out_word_offset; /* first uint32 word of the packet's decoded bits in the output arena */
} vd_packet;

typedef struct vd_batch_plan vd_batch_plan;   /* opaque, owns device memory */

typedef struct vd_batch_info {
    int64_t n_packets, n_frames, n_pairs;
    int64_t scratch_bytes;       /* survivor + depunctured-LLR device memory held by the plan */
    int64_t resident_warps;      /* persistent warps per launch (last code kind) */
    int32_t lanes, radix;        /* kernel shape (last code kind) */
    int32_t n_launches;          /* kernel launches per vd_batch_plan_launch */
    int32_t reserved;
} vd_batch_info;

/*
 * Builds a batch plan: checks every descriptor on the host, chooses f and v
 * for packets with f == 0 (one frame length per code kind that minimises the
 * predicted makespan of the persistent launch; packets no longer than it are
 * decoded as one full-length frame; v = 42 for K=7, 64 for K=9, or tune->v),
 * sorts and pairs all frames, and uploads descriptors and work list (device
 * memory owned by the plan).  tune: NULL, or lanes / radix / f / v overrides.
 * When tune is NULL or leaves radix (or lanes) at 0, the plan measures the
 * candidate kernel shapes (radix 2 and 4; 1 or 2 lanes per frame pair for
 * K=7, 4 or 8 for K=9) by running its own work list on zero LLRs on
 * `stream`, and keeps the fastest; the shape never changes the decoded bits.
 * The arenas are given at launch.  Synchronises `stream` before returning.
 */
vd_status vd_batch_plan_create(vd_batch_plan **out, const vd_code *const *codes, int n_codes,
                               const vd_packet *packets, int64_t n_packets, const vd_tune *tune,
                               void *stream);

/* Launches the plan on `stream`: the input pre-pass (if any packet is
 * punctured or 4-bit), then one persistent kernel per code kind.  d_llr_arena
 * holds every packet's received values at its llr_offset; d_out_arena receives
 * the packed bits at each packet's out_word_offset (ceil(n_info/32) words;
 * packets must not share words).  A plan's survivor scratch and task
 * counters are its own: launches of one plan must not overlap on the GPU
 * (keep them on one stream, or order the streams).  Asynchronous. */
vd_status vd_batch_plan_launch(vd_batch_plan *plan, const void *d_llr_arena, uint32_t *d_out_arena,
                               void *stream);

/* Same as vd_batch_plan_launch, but the decode kernels may start while the
 * kernel before them on `stream` is still running (programmatic dependent
 * launch), so back-to-back launches of a stream of batches overlap one
 * launch's last tasks and final tracebacks with the next one's first tasks.
 * Ordering that still holds: each kernel waits for the kernel before it to
 * complete before it writes any output word and before it lets the kernel
 * after it start, so outputs land in stream order and a launch never runs
 * beside the one two back (consecutive launches alternate between two
 * scratch buffers and two sets of task counters; the second scratch is
 * allocated by the first call that needs it: VD_ENOMEM if that fails).
 * Contract: the kernel just before this launch on `stream` must not write
 * d_llr_arena (the decode kernels read it before they wait).  A copy or a
 * memset before the launch is not a kernel and orders as usual; the previous
 * launch of a plan, reading its own arenas, is the intended predecessor.
 * Plans with a pre-pass (punctured, 4-bit or hard-decision packets) launch
 * exactly as vd_batch_plan_launch.  The overlap is between consecutive
 * launches on one stream: chained launches of one plan on several streams
 * at once are not ordered and must not be made.  Asynchronous. */
vd_status vd_batch_plan_launch_chained(vd_batch_plan *plan, const void *d_llr_arena, uint32_t *d_out_arena,
                                       void *stream);

/* Same as vd_batch_plan_launch, through a CUDA graph captured on the first call
 * for these arenas and replayed afterwards.  Needs a non-default stream. */
vd_status vd_batch_plan_launch_graph(vd_batch_plan *plan, const void *d_llr_arena,
                                     uint32_t *d_out_arena, void *stream);

/* Sizes and shape of a plan. */
vd_status vd_batch_plan_info(const vd_batch_plan *plan, vd_batch_info *info);

/* The f and v used for each packet (arrays of n_packets). */
vd_status vd_batch_plan_packet_tune(const vd_batch_plan *plan, int32_t *f_out, int32_t *v_out);

/* Waits for `stream`; VD_EBOUNDS if a launch of this plan refused work. */
vd_status vd_batch_plan_status(vd_batch_plan *plan, void *stream);

/* Frees a plan after the device is idle (NULL is ignored). */
void vd_batch_plan_destroy(vd_batch_plan *plan);

/*
 * vd_decode_each — the plain form a batch is measured against: one vd_decode
 * call (one or two launches) per packet, issued from C in packet order and
 * spread round-robin over n_streams caller streams.  Each packet's f and v
 * must be set (f > 0), e.g. from vd_batch_plan_packet_tune, so that the bits
 * equal the batch's.  Offsets and arenas as in vd_batch_plan_launch.
 * Asynchronous; the first failing call's status is returned and later
 * packets are not launched.
 */
vd_status vd_decode_each(const vd_code *const *codes, int n_codes, const vd_packet *packets,
                         int64_t n_packets, const void *d_llr_arena, uint32_t *d_out_arena, int radix,
                         void *const *streams, int n_streams);

/*
 * vd_decode_tc — the paper's tensor-core formulation of the radix-4 forward
 * procedure (Sec. VIII: D = Theta_hat L + Lambda per stage pair, the
 * dragonfly groups of Sec. VIII-D-2 so that four Theta_hat in one A operand
 * serve all 16 dragonflies), as a measured variant of vd_decode.  Two
 * mma.sync.m16n8k16 (f16 x f16 -> f32, exact for int8 LLRs) per stage pair
 * and frame, one warp per frame; same frames, tie rules and bits as
 * vd_decode.  Arguments as vd_decode for unpunctured int8 LLRs of K=7,
 * beta=2 codes whose dragonflies form at most four groups (the (2,1,7)
 * 171/133 code); frames of at most 1024 stages (f + 2 v).
 * VD_EUNSUPPORTED otherwise.  Asynchronous on stream.
 */
vd_status vd_decode_tc(const vd_code *code, const void *d_llr, int64_t n_info, int f, int v, uint32_t flags,
                       uint32_t *d_out, void *stream);

/*
 * vd_decode_radix — the general radix-2^rho forward procedure of Sec. VI as a
 * measured variant of vd_decode: rho = 1, 2 or 3 trellis stages per step
 * (radix 2, 4, 8), the states of each group of 2^rho left and right states
 * indexed by Eq. general:S, every right state taking the best of its 2^rho
 * candidates (rho branch metrics each) with a rho-bit survivor; one warp per
 * frame, metrics in shared memory, survivors in the library's scratch pool
 * (allocated on first use).  Same frames, tie rules and bits as vd_decode.
 * Arguments as vd_decode for unpunctured int8 LLRs of the K=7 and K=9 codes.
 * VD_EINVAL on bad arguments (rho outside 1..3), VD_EUNSUPPORTED otherwise.
 * Asynchronous on stream.
 */
vd_status vd_decode_radix(const vd_code *code, const void *d_llr, int64_t n_info, int f, int v, int rho,
                          uint32_t flags, uint32_t *d_out, void *stream);

/* One-shot batch decode: plan, launch, wait for `stream`, free. */
vd_status vd_decode_batch(const vd_code *const *codes, int n_codes, const vd_packet *packets,
                          int64_t n_packets, const void *d_llr_arena, uint32_t *d_out_arena,
                          const vd_tune *tune, void *stream);

/* ------------------------------------------------------------------ serving
 *
 * Continuous batching: packets arriving from many sources are queued on the
 * host, admitted while the server's device arena has room for their LLRs
 * and outputs (admission by device memory), and decoded in micro-batches of
 * everything admitted — one persistent launch per code kind, on a pool of
 * CUDA streams, so a batch formed while earlier ones are still running
 * overlaps them on the device.  Frames as in vd_decode: f = 256, v = 42 for
 * K=7 and f = 512, v = 64 for K=9 unless configured; a packet no longer than
 * f is one full-length frame.  Each packet's result is the same whether it is
 * decoded alone or in a mix (the same frames, the same arithmetic).  The
 * paper has no serving layer.
 */
typedef struct vd_server vd_server;

typedef struct vd_server_config {
    int64_t device_bytes;    /* device arena for admitted packets (default 256 MiB) */
    int32_t max_batch;       /* packets per micro-batch (default 4096) */
    int32_t n_streams;       /* CUDA streams that overlap micro-batches (default 3, max 8) */
    int32_t max_packet_bits; /* largest n_info accepted (default 12000) */
    int32_t lanes, radix;    /* kernel shape, 0 = defaults */
    int32_t f7, v7, f9, v9;  /* frame length / overlap per code kind, 0 = defaults */
    int32_t reserved[5];
} vd_server_config;

typedef struct vd_completion {
    uint64_t tag;            /* as given to vd_server_submit */
    int32_t status;          /* VD_OK, or VD_ECUDA if the device reported an error */
    int32_t n_words;         /* ceil(n_info/32) decoded words */
    int64_t word_offset;     /* where they start in the words buffer of vd_server_poll */
    int64_t submit_ns, admit_ns, done_ns;   /* host steady-clock times: submitted, admitted to
                                               the device, completion seen by the server */
} vd_completion;

typedef struct vd_server_stats {
    int64_t submitted, completed, batches, bits_decoded;
    int64_t pending;         /* waiting for admission */
    int64_t arena_used;      /* bytes of the device arena in use */
    int64_t error;           /* last CUDA error seen by the worker (0 = none) */
} vd_server_stats;

/* Creates a server (allocates its arena, pinned mirror and per-stream buffers,
 * and starts its worker thread) on the current device. */
vd_status vd_server_create(vd_server **out, const vd_code *const *codes, int n_codes,
                           const vd_server_config *cfg);

/* Queues one packet: n_values received values (int8, 4-bit two per byte, or
 * hard decisions eight per byte) in host memory, copied before returning into
 * the server's pinned staging area (from where its batch uploads it into the
 * device arena; the kernels read device memory only); n_info information
 * bits; flags as vd_decode.  Never blocks on the device. */
vd_status vd_server_submit(vd_server *server, int code_id, int llr_type, const void *host_llr,
                           int64_t n_values, int64_t n_info, uint32_t flags, uint64_t tag);

/* Queues n host packets in one call (one staging lock and one queue lock):
 * packet i as vd_server_submit(code_id[i], llr_type[i], host_llr +
 * llr_offset[i] bytes, n_values[i], n_info[i], flags[i], tags[i]).  Every
 * packet is checked first; on an error nothing is queued. */
vd_status vd_server_submit_many(vd_server *server, int64_t n, const int32_t *code_id, const int32_t *llr_type,
                                const void *host_llr, const int64_t *llr_offset, const int64_t *n_values,
                                const int64_t *n_info, const uint32_t *flags, const uint64_t *tags);

/* As vd_server_submit, for values already in device memory (an upstream
 * stage on the GPU produced them): nothing is copied; the kernels read the
 * caller's buffer in place, so it must stay valid and unchanged until the
 * packet's completion has been polled.  Punctured / 4-bit packets are still
 * expanded into the server's arena. */
vd_status vd_server_submit_device(vd_server *server, int code_id, int llr_type, const void *d_llr,
                                  int64_t n_values, int64_t n_info, uint32_t flags, uint64_t tag);

/* Moves up to max_completions finished packets out: their records into comp
 * and their decoded words into words (capacity words_cap).  Returns the
 * number of records written (0 if none is ready). */
int64_t vd_server_poll(vd_server *server, vd_completion *comp, int64_t max_completions,
                       uint32_t *words, int64_t words_cap);

/* Counters of the server. */
vd_status vd_server_stats_get(vd_server *server, vd_server_stats *out);

/* Stops the worker, waits for the device, frees everything. */
void vd_server_destroy(vd_server *server);

/*
 * vd_server_replay — open-loop trace replay against a server (a load
 * generator for latency measurement; the paper has no counterpart).
 *
 * Submits packet i (tag i) once arrival_ns[i] nanoseconds (nondecreasing)
 * have passed since the call started — for host packets with n >= 4096
 * from 4 submitting threads, packet i from thread i mod 4, each thread
 * submitting every packet of its share that has arrived in one
 * vd_server_submit_many call — while the calling thread collects
 * completions, until all n packets have completed.  Packet i: code_id[i],
 * llr_type[i], n_values[i] values at host_llr + llr_offset[i] bytes,
 * n_info[i], flags[i].  Outputs: latency_ns[i] = completion time - the
 * packet's scheduled arrival time (host steady clock, so any submit delay
 * counts; -1 if unfinished); if words is not NULL, packet i's decoded words at
 * words + word_offset[i]; *span_ns (if not NULL) = last completion - first
 * submit.  The server must be idle (nothing submitted and unpolled).
 * Errors: VD_EINVAL (bad arguments, busy server), a submit error,
 * VD_ECUDA (device error), VD_ETIMEOUT after timeout_ms (> 0) — packets then
 * still in the server stay there until it is destroyed.
 */
vd_status vd_server_replay(vd_server *server, int64_t n, const int32_t *code_id, const int32_t *llr_type,
                           const void *host_llr, const int64_t *llr_offset, const int64_t *n_values,
                           const int64_t *n_info, const uint32_t *flags, const int64_t *arrival_ns,
                           int64_t timeout_ms, int64_t *latency_ns, uint32_t *words,
                           const int64_t *word_offset, int64_t *span_ns);

/* vd_server_replay with the packets' values in device memory (d_llr +
 * llr_offset[i] bytes), submitted with vd_server_submit_device from one
 * submitting thread. */
vd_status vd_server_replay_device(vd_server *server, int64_t n, const int32_t *code_id, const int32_t *llr_type,
                                  const void *d_llr, const int64_t *llr_offset, const int64_t *n_values,
                                  const int64_t *n_info, const uint32_t *flags, const int64_t *arrival_ns,
                                  int64_t timeout_ms, int64_t *latency_ns, uint32_t *words,
                                  const int64_t *word_offset, int64_t *span_ns);

/*
 * vd_bm_gate — the measurement behind the choice of CUDA cores over tensor
 * cores for the branch metrics (Eq. BM; the paper computes them as the
 * product of the code's +-1 output patterns with the LLRs, Sec. V).  For the
 * (2,1,7) code, computes the four branch metrics of every (stage, frame pair)
 * with variant 0 = CUDA-core 16x2 arithmetic (the decoder's form) or
 * 1 = mma.sync m16n8k32 s8 tensor-core products plus a shared-memory
 * transpose into the decoder's per-lane layout.
 *   d_llr:      [n_stages][n_pairs] words, bytes l0, l1 of frame 0 then of frame 1 (int8)
 *   n_pairs:    a positive multiple of 32; n_stages > 0
 *   d_checksum: [n_pairs] words, a fold of every metric of the pair (same for both variants)
 *   d_metrics:  NULL, or [n_stages][4][n_pairs] words: pattern x (bit b set: -l_b) as s16x2
 * Asynchronous on stream; VD_EINVAL on bad arguments, VD_ECUDA on launch failure.
 */
vd_status vd_bm_gate(int variant, const void *d_llr, int64_t n_pairs, int32_t n_stages,
                     uint32_t *d_checksum, uint32_t *d_metrics, void *stream);

/*
 * vd_int_peak — the integer-issue microbenchmark behind the decoder's
 * roofline (the add-compare-select of Eq. PM runs on the SM's integer units).
 * Runs one variant on n_blocks blocks of 1024 threads (one per SM), each
 * thread 8 independent dependency chains for iters x 16 bodies:
 *   0: 16x2 add   1: 16x2 max   2: fused 16x2 add-then-max   3: 32-bit
 *   multiply-add   4: three-input logic   5: byte permute   6: funnel shift
 *   7: 16x2 add + multiply-add, 1:1   8: fused add-max + multiply-add, 1:1
 *   9: 16x2 max + three-input logic, 1:1   10: the decoder's radix-2
 *   butterfly (two 16x2 adds and two fused add-max per register pair).
 * A body is 8 operations of the variant (16 for variant 10: 4 butterflies).
 *   d_cycles: [n_blocks] int64 — each block's clock64() span between two block
 *             barriers around the timed loop (SM clocks).
 *   d_sink:   [n_blocks x 1024] words the chains are folded into.
 * Asynchronous on stream; VD_EINVAL on bad arguments, VD_ECUDA on launch failure.
 */
vd_status vd_int_peak(int variant, int64_t iters, int n_blocks, int64_t *d_cycles, uint32_t *d_sink,
                      void *stream);

/*
 * Waits for the stream, then reads and clears the device status words of the
 * current device: that of vd_decode_noalloc first, then the library's own.
 * VD_EBOUNDS if a kernel refused work that would have overrun its scratch
 * since the last check (the affected outputs are not written).  Allocates
 * nothing (a status word that does not exist yet has not been written).
 */
vd_status vd_sync(void *stream);

/*
 * vd_decode_noalloc — the stream decode of vd_decode without any device
 * allocation.  The paper has no counterpart: this is a deployment variant.
 *
 * For callers that must not allocate device memory while they run: a
 * real-time receiver thread that cannot absorb the latency of cudaMalloc (it
 * can block and synchronise the device), a program whose device memory is
 * reserved up front by another allocator or a fixed budget, or a process that
 * must not grow after start-up.  This call makes no allocation at all (no
 * cudaMalloc, cudaFree or allocating library routine); the caller passes the
 * input and output buffers as for vd_decode.
 *
 * Survivor scratch: a file-scope device array of vd_noalloc_scratch_limit()
 * bytes (32 MiB), which occupies that much memory on every GPU where the
 * library's device code is loaded, until the process exits.  A stream whose
 * scratch would not fit is rejected with VD_EINVAL and a message giving both
 * sizes (for the K=7 code at f=256, v=42 this is about 2 million info bits).
 *
 * Arguments as vd_decode, restricted to unpunctured int8 LLRs (VD_LLR_S8);
 * no metric output.  The first call on each device sets that device up: it
 * looks up the device address of the array (cudaGetSymbolAddress) with the
 * device current, which under lazy module loading also loads the library's
 * device code and materialises the array.  So make one call first, before
 * the phase that must not allocate and before any stream capture; a call
 * with n_info = 0 does only this set-up.  Every call on a device shares the
 * one array: calls that overlap on the GPU (different streams, or concurrent
 * host threads) race on it and corrupt each other's results; serialise them
 * (one stream).
 *
 * Device-side errors: a kernel that refuses a frame pair which would overrun
 * the array (host checks make this unreachable) sets a status word in a
 * second static array and leaves that pair's output unwritten.  The word is
 * zero at load, is not cleared by decode calls, and is read and cleared by
 * vd_sync(stream), which then returns VD_EBOUNDS.
 */
vd_status vd_decode_noalloc(const vd_code *code, const void *d_llr, int64_t n_info, int f, int v,
                            int radix, uint32_t flags, uint32_t *d_out, void *stream);

/* Size in bytes of the fixed survivor scratch used by vd_decode_noalloc. */
int64_t vd_noalloc_scratch_limit(void);

/*
 * vd_transmit — the transmitter and channel of the paper's verification
 * system (Sec. IX-B) on the GPU, a source of received values that never
 * touches the host: information bits -> convolutional encoder from state 0
 * (Sec. II-A; k-1 zero tail bits when flags has VD_TERMINATED) -> the code's
 * puncturing (kept positions, stage-major, b ascending) -> BPSK (bit 0 ->
 * +1, bit 1 -> -1) -> AWGN y = x + sigma z -> quantiser of llr_type:
 *   VD_LLR_S8: clip(rint(32 y), -127, 127)     VD_LLR_S4: clip(rint(2 y), -7, 7), packed
 *   VD_LLR_F16: half(2 y / sigma^2)            VD_LLR_HARD: y < 0, packed
 * z of the k-th kept value is standard normal number k of the stream:
 * Philox4x64-10 (Salmon et al., SC 2011) with key (seed, stream_id) on
 * counter (k / 4, 0, 0, 0), four normals per counter by the Box-Muller
 * transform (words 0,1 and 2,3: u = ((w >> 11) + 1) 2^-53; sqrt(-2 ln u)
 * cos(2 pi v), sqrt(-2 ln u) sin(2 pi v)) in double precision.  The same
 * (seed, stream_id) give the same samples on every call.
 *   d_bits:  ceil(n_info/32) device words of information bits, LSB-first.
 *   sigma:   noise standard deviation >= 0 (> 0 for VD_LLR_F16); for Eb/N0
 *            in dB and code rate R, sigma = sqrt(1 / (2 R 10^(EbN0/10))).
 *   d_out:   vd_transmit_bytes() bytes of device memory (written).
 * Asynchronous on stream.  VD_EINVAL on bad arguments, VD_ECUDA on launch
 * failure.
 */
vd_status vd_transmit(const vd_code *code, const uint32_t *d_bits, int64_t n_info, uint32_t flags,
                      double sigma, uint64_t seed, uint64_t stream_id, int llr_type, void *d_out,
                      void *stream);

/* Bytes vd_transmit writes for these arguments (-1 on bad arguments). */
int64_t vd_transmit_bytes(const vd_code *code, int64_t n_info, uint32_t flags, int llr_type);

/* Number of frames of a stream decode: ceil(n_info / f) (0 if n_info <= 0). */
int64_t vd_num_frames(int64_t n_info, int f);

/* Number of transmitted LLRs for T stages of this code (puncturing applied). */
int64_t vd_num_kept(const vd_code *code, int64_t T);

/* Bytes of survivor scratch one stream decode needs (informational, int8
 * LLRs).  A stream with at least one task of frame pairs per resident warp
 * of the persistent kernel needs a fixed two buffers per resident warp; a
 * shorter one needs one buffer per frame pair's lane group. */
int64_t vd_scratch_bytes(const vd_code *code, int64_t n_info, int f, int v, int radix,
                         const vd_tune *tune);

/* Frees this thread's current device's scratch pool (all streams). */
vd_status vd_release_scratch(void);

/* Message for the calling thread's last error ("" if none). */
const char *vd_last_error(void);

/* ABI version: major * 10000 + minor * 100 + patch. */
int vd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VD_H */
