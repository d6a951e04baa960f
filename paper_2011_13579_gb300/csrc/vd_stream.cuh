// Segmented stream decode: branch metrics, radix-2 / radix-4 add-compare-select
// with packed survivors, and traceback from the overlap, fused in one kernel.
//
// Paper: arXiv 2011.13579.  Eq. BM (branch metric), Eq. PM / Eq. SP0 (ACS and
// survivor), Algorithms 1 and 2 (forward and backward procedures), Sec. III
// (frames of f stages with overlap), Thm. 1 (butterfly state indices),
// Thm. 2 and its corollary (all four branch outputs of a butterfly follow
// from its main output), Sec. VIII-A / Eq. radix4:PM, radix4:SP0 (two stages
// per step, traceback two stages per step).
//
// Mapping (one group of L lanes per PAIR of frames):
//   * the two frames of a pair are the two 16-bit halves of every register;
//   * register R (K-1 bits; the top log2(L) bits select the lane) holds, at
//     stage tau, the metric of state ROTR^tau(R).  With this rotation the two
//     left states 2g, 2g+1 of every butterfly sit in registers that differ
//     only in bit (tau mod (K-1)), and its two right states g, g+2^(K-2) land
//     in the same two registers: the ACS is in place.  When that bit is a
//     lane bit the partner comes from the other lane by one shuffle;
//   * the main output alpha of butterfly g is linear in the bits of g, so the
//     part contributed by the lane bits is folded into the LLR signs of that
//     lane and the rest is a compile-time constant per register;
//   * frames of a pair are right-aligned on a common padded length Wpad (a
//     multiple of the unroll period U), so they end together; the shorter
//     frame is preceded by stages of zero LLRs, which keep all-equal metrics
//     all-equal, and a frame that starts from the reset state gets its head
//     start on state 0 when its first stage arrives;
//   * decisions go, packed one bit per state and frame, to a global scratch
//     buffer; a warp's stores for one stage are contiguous.  Bit (r & 31) of
//     word (r >> 5) holds register r of the lane (r & 15 at bit 16h for a
//     lane with 16 registers; frame h = 0, 1);
//   * radix-2 K=7 embeds the decisions in the metrics instead (see
//     StreamCfg::ES and forward_pair): each group of three stages leaves one
//     record of 4-bit fields per register, word r >> 2 at bits 4 (r & 3) +
//     16h, whose bit 2 is the register's decision at the record's last
//     stage, bit 1 the decision at the stage before of the register it came
//     from, and bit 0 the decision one stage earlier along the same
//     survivor (the two-stage form, ES = 2, has 2-bit fields, word r >> 3);
//   * radix-4: stages are taken in pairs (t-1, t).  The metrics are two
//     radix-2 steps (grouping the four candidates of a right state by their
//     middle state, as Eq. radix4:PM allows, gives exactly the same integers
//     and ties), and the survivor of right state j is the 2-bit pair
//     (d_m, d_i): the decision of j at stage t and the decision of the
//     middle state it selects at stage t-1 — exactly the 2-bit field of the
//     embedded stage-pair records, which the radix-4 kernels use wherever
//     their range fits (StreamCfg::ES2M_OK); otherwise the two bits go to
//     per-stage decision words at the same bit position, so that one
//     traceback step crosses two stages;
//   * traceback (Algorithm 2) walks groups of K-1 stages whose survivor words
//     are staged in shared memory; a group's decoded bits are the register
//     index at the group's start.  The persistent kernels (vd_batch.cuh) run
//     one pair's traceback, two groups every second group of stages, during
//     the next pair's forward pass.
#pragma once
#include <utility>
#include "vd_device.cuh"

namespace vd {

struct StreamParams {
    const int8_t *llr;      // depunctured received LLRs, [T][beta], int8
    int64_t llr_bytes;      // T * beta
    int64_t n_info, T, f, v;
    int64_t n_win, n_pairs;
    uint32_t flags;         // bit0: terminated, bit1: start state unknown
    int32_t wpad_max;       // padded frame length the scratch of one warp holds
    uint32_t *out;          // packed decoded bits, LSB-first
    uint32_t *surv;         // survivor scratch: wpad_max x 32 x SW words per warp
    int32_t *pm_out;        // optional [n_win][2^(K-1)] canonical final metrics
    int *status;            // device status word (bit 0: a frame pair exceeded the scratch)
    int *counter;           // persistent form: task counter, zero at launch
    int64_t n_tasks;        // persistent form: tasks of 32/L frame pairs
};

// One frame as the decoder core sees it: stage indices are relative to the
// first stage of its stream (or packet), whose LLRs start at llr and whose
// decoded bits start at bit 0 of out.
struct FrameTask {
    const int8_t *llr;      // [T][beta] int8 of the frame's stream
    uint32_t *out;          // packed output of the frame's stream
    int32_t *pm;            // NULL, or 2^(K-1) canonical final metrics of this frame
    int64_t a, b, o, e;     // trellis stages [a, b), decoded stages [o, e)
    int valid, known, term; // real frame / starts from state 0 / ends at a terminated end
};

__host__ __device__ __forceinline__ FrameTask frame_task(const int8_t *llr, uint32_t *out, int32_t *pm,
                                                        int64_t s, int64_t n_win, int64_t n_info,
                                                        int64_t T, int64_t f, int64_t v,
                                                        uint32_t flags) {
    FrameTask t;
    t.llr = llr;
    t.out = out;
    t.valid = s < n_win;
    const Frame w = frame_of(t.valid ? s : 0, n_info, T, f, v, flags);
    t.a = w.a; t.b = w.b; t.o = w.o; t.e = w.e;
    t.known = t.valid && w.known_start;
    t.term = t.valid && w.term_end;
    t.pm = t.valid ? pm : nullptr;
    return t;
}

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// Unroll period: an even multiple of K-1 (rotation period) whose chunk of LLR
// bytes is a whole number of 32-bit words.
__host__ __device__ constexpr int chunk_stages(int K, int beta) {
    int u = K - 1;
    while ((u * beta) % 4 || (u % 2)) u += K - 1;
    return u;
}

template <int K, int BETA, uint64_t GENS, int L, bool RADIX4>
struct StreamCfg {
    using C = Code<K, BETA, GENS>;
    static constexpr int NB = C::NB;
    static constexpr int NS = C::NS;
    static constexpr int NR = NS / L;                 // registers per lane
    static constexpr int LR = ilog2(NR);              // local register bits
    static constexpr int U = chunk_stages(K, BETA);   // stages per chunk
    static constexpr int UW = U * BETA / 4;           // LLR words per chunk per frame
    static constexpr int NW = NR >= 32 ? NR / 16 : 1; // survivor words per lane per stage
    static constexpr int WPF = NR >= 32 ? NR / 32 : 1;// survivor words per frame per lane per stage
    static constexpr int NACC = NR >= 16 ? NR / 16 : 1;
    // Embedded decisions (radix-2, when the range allows): metrics are kept
    // as 2^ES m + j, the ES low bits j of each half carrying the decisions of
    // the current record of ES stages; see forward_pair.  ES = 0: one
    // decision word per stage instead.
    //
    // Min-normalised forms (MINNORM; records of ES = 3 stages, scale 8, or
    // ES = 2, scale 4): every branch metric carries + B, so it lies in
    // [0, 2B] and no metric falls within a chunk (a common per-stage offset
    // changes no decision, Eq. PM); every chunk starts by subtracting the
    // minimum over the states (folded into its first stage), which brings
    // it to the floor FM = 0, and a frame that starts from the reset state
    // gets the exact head start C::HT.  Bounds on m (per half):
    //   * steady state: after a normalisation m is in [0, SP] with
    //     SP = (K-1)(delta_max - delta_min) the spread of all metrics once
    //     every state is reachable; a chunk adds at most 2 U B, so m stays in
    //     [0, SP + 2 U B];
    //   * after a head start with t < K-1 stages left in its chunk, states
    //     not yet reachable from state 0 lie within 2 t B of the old floor and
    //     the others within 2 t B of it plus HT, so the next normalisation
    //     leaves m <= HT + 2 t B, and the next chunk adds 2 U B.
    // The largest 2^ES m + 2^ES - 1 must stay within 16 unsigned bits.
    static constexpr int FM = 0;
    static constexpr int TMAX = U < NB - 1 ? U : NB - 1;
    static constexpr int TOPM_STEADY = 2 * NB * C::B + 2 * U * C::B;
    static constexpr int TOPM_RESET = C::HT + (2 * TMAX + 2 * U) * C::B;
    static constexpr int TOPM = FM + (TOPM_STEADY > TOPM_RESET ? TOPM_STEADY : TOPM_RESET);
    static constexpr bool ES3_OK = !RADIX4 && NB % 3 == 0 && U % 3 == 0 && NR % 4 == 0 &&
                                   8 * TOPM + 7 <= 65535;
    // Radix-4 takes stage-pair records: a field's two bits are the radix-4
    // survivor of Eq. radix4:SP0 (the decision at the pair's second stage
    // and that of the middle state it selects), the candidates grouped by
    // middle state as two exact radix-2 steps (R10).
    static constexpr bool ES2M_OK = NB % 2 == 0 && NR % 8 == 0 && 4 * TOPM + 3 <= 65535;
    // ES = 2 with state 0 as the reference every NORM_CHUNKS chunks and the
    // loose head start C::S (for codes whose min-normalised range does not
    // fit).  Longest normalisation period (stages) that keeps
    // 4 (F + 2S + (N+1) B) + 3 within 16 unsigned bits:
    static constexpr int NMAX_EMB = (16383 - 2 * C::S) / (2 * C::B) - 1;
    static constexpr bool ES2_OK = NB % 2 == 0 && NR % 8 == 0 && NMAX_EMB >= U;
    static constexpr int ES = ES3_OK ? 3 : ((ES2M_OK || ES2_OK) ? 2 : 0);
    static constexpr bool MINNORM = ES3_OK || ES2M_OK;
    static constexpr bool EMB = ES != 0;
    static constexpr int SC = 1 << ES;                // metric scale
    static constexpr int FW = ES == 3 ? 4 : 2;        // record field width (bits)
    static constexpr int RPW = 16 / FW;               // registers per record word (per half)
    static constexpr int NWE = NR / RPW;              // record words per lane per record (EMB)
    static constexpr int HS = MINNORM ? C::HT : C::S; // head start of a frame from the reset state
    // scratch words per lane per stage (records of ES stages, or words per stage)
    static constexpr int SW = EMB ? ((NWE + ES - 1) / ES > NW ? (NWE + ES - 1) / ES : NW) : NW;
    // normalisation period (multiple of U), see the header of vd_device.cuh
    static constexpr int NMAX = ES == 2 ? NMAX_EMB : (32767 - 2 * C::S) / (2 * C::B) - 1;
    static constexpr int NORM_CHUNKS = MINNORM ? 1 : ((NMAX / U) > 0 ? (NMAX / U) : 1);
    static constexpr int F = MINNORM ? FM : (NORM_CHUNKS * U + 1) * C::B;   // floor after normalisation
    static_assert(NS % L == 0 && L <= 32 && (L & (L - 1)) == 0, "L must be a power of two");
    static_assert(NR >= 2, "at least one butterfly per lane");
    static_assert(!RADIX4 || NB % 2 == 0, "radix-4 pairs need an even rotation period");
    static_assert(MINNORM || NORM_CHUNKS * U <= NMAX, "normalisation period too long for 16-bit metrics");
    static_assert(MINNORM ? SC * TOPM + SC - 1 <= 65535
                  : ES == 2 ? 4 * (F + 2 * C::S + (NORM_CHUNKS * U + 1) * C::B) + 3 <= 65535
                            : F + 2 * C::S + (NORM_CHUNKS * U + 1) * C::B <= 32767,
                  "metric range");
    static_assert(!EMB || NWE * 32 <= 32 * ES * SW, "a record fits the scratch of its ES stages");
    // The state-0 ES = 2 form normalises without a clamp.  Below the
    // reference only states not yet reachable from a head-start state 0 can
    // fall (for fewer than K-1 stages), by at most 2(K-1)B before and
    // (K-1)B + B after a normalisation, so a floor F >= (3(K-1) + 1) B keeps
    // them >= 0.
    static_assert(MINNORM || ES != 2 || F >= (3 * NB + 1) * C::B, "unclamped normalisation floor");
    static_assert(!MINNORM || F == 0, "biased branch metrics: min-normalisation to zero");
};

template <typename Fn, int... S>
__device__ __forceinline__ void static_for_impl(Fn &&fn, std::integer_sequence<int, S...>) {
    (fn(std::integral_constant<int, S>{}), ...);
}
// Calls fn(integral_constant<int, i>) for i = 0 .. N-1: loop indices are compile-time.
template <int N, typename Fn>
__device__ __forceinline__ void static_for(Fn &&fn) {
    static_for_impl(fn, std::make_integer_sequence<int, N>{});
}

// LLR chunk loading in two steps so the loads of chunk c+1 are in flight while
// chunk c is decoded: fetch() issues the aligned 32-bit loads of bytes
// [vb, vb + 4*UW) relative to the frame's first byte `base`, finish()
// re-aligns them with funnel shifts.  A chunk that is not wholly inside the
// frame's bytes [0, hi) (the first chunk of a padded frame) is assembled byte
// by byte in finish() with zeros outside the range.  Offsets are 32-bit: a
// frame spans far fewer than 2^31 bytes.
template <int UW>
struct ChunkRaw {
    uint32_t raw[UW + 1];
    uint32_t sh;
    bool fast;
};

template <int UW>
__device__ __forceinline__ void fetch_chunk(const int8_t *base, int32_t vb, int32_t hi, ChunkRaw<UW> &c) {
    c.fast = vb >= 0 && vb + 4 * UW <= hi;
    if (c.fast) {
        const uintptr_t addr = reinterpret_cast<uintptr_t>(base) + (uintptr_t)(uint32_t)vb;
        const uint32_t mis = (uint32_t)(addr & 3u);
        const uint32_t *p = reinterpret_cast<const uint32_t *>(addr - mis);
#pragma unroll
        for (int i = 0; i < UW; ++i) c.raw[i] = __ldg(p + i);
        // the extra word holds the last bytes of the chunk when it is misaligned;
        // it contains at least one byte inside the stream, so it is readable
        c.raw[UW] = mis ? __ldg(p + UW) : 0u;
        c.sh = 8u * mis;
    }
}

template <int UW>
__device__ __forceinline__ void finish_chunk(const int8_t *base, int32_t vb, int32_t hi,
                                             const ChunkRaw<UW> &c, uint32_t (&w)[UW]) {
    if (c.fast) {
#pragma unroll
        for (int i = 0; i < UW; ++i) w[i] = funnel_r(c.raw[i], c.raw[i + 1], c.sh);
    } else {
#pragma unroll
        for (int i = 0; i < UW; ++i) {
            uint32_t x = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int32_t pos = vb + 4 * i + k;
                if (pos >= 0 && pos < hi) x |= (uint32_t)(uint8_t)base[pos] << (8 * k);
            }
            w[i] = x;
        }
    }
}

// Selects element idx of a small register array without local memory.
template <int N>
__device__ __forceinline__ uint32_t pick(const uint32_t *a, uint32_t idx) {
    uint32_t r = a[0];
#pragma unroll
    for (int i = 1; i < N; ++i) r = (idx == (uint32_t)i) ? a[i] : r;
    return r;
}

// Mask of bit positions whose bit k is set (k < 5).
__host__ __device__ constexpr uint32_t bitk_mask(int k) {
    return k == 0 ? 0xAAAAAAAAu : k == 1 ? 0xCCCCCCCCu : k == 2 ? 0xF0F0F0F0u
         : k == 3 ? 0xFF00FF00u : 0xFFFF0000u;
}

// Per-half minimum of N packed registers: a tree of three-input minima.
template <int N>
__device__ __forceinline__ uint32_t min_tree(const uint32_t (&v)[N]) {
    if constexpr (N == 1) {
        return v[0];
    } else if constexpr (N == 2) {
        return min_u16x2(v[0], v[1]);
    } else {
        constexpr int M = (N + 2) / 3;
        uint32_t w[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            if (3 * i + 2 < N) w[i] = __vimin3_u16x2(v[3 * i], v[3 * i + 1], v[3 * i + 2]);
            else if (3 * i + 1 < N) w[i] = min_u16x2(v[3 * i], v[3 * i + 1]);
            else w[i] = v[3 * i];
        }
        return min_tree<M>(w);
    }
}

// ------------------------------------------------------------ traceback
//
// Backward procedure (Algorithm 2) for one pair of frames, resumable: it walks
// groups of K-1 stages (so the phase of every stage in a group is a
// compile-time constant) from Wpad-1 down to the frames' first decoded
// stages.  A persistent warp calls step() once per chunk of the NEXT frame
// pair's forward pass, so the traceback's dependent chain and its memory
// latency hide behind forward work.  The survivor words of the next two
// groups are copied into a per-warp shared-memory staging area by cp.async
// while earlier groups are walked; the per-lane state lives in shared memory
// between steps.  Every lane of a group follows both frames; the lane that
// owns the current register supplies its decision bit (one shuffle).
// Survivor words: bit (r & 31) of word (r >> 5) holds register r of the lane
// (r & 15 at bit 16h when a lane has 16 registers or fewer), frame 0 first.

// All fields are 32-bit words (pointers and the 64-bit bit accumulator are
// split in two): 23 words, an odd stride, so the per-thread records in shared
// memory are read and written without bank conflicts.
struct TbState {
    uint32_t out_w[2][2];    // packed output of each frame's stream (pointer words)
    uint32_t surv_w[2];      // this lane's survivor records (pointer words)
    uint32_t oacc_w[2][2];   // decoded bits not yet stored: bit i = stage (lowest emitted + i)
    uint32_t R[2];           // current register of each frame (traceback state)
    int32_t onb[2];          // number of bits in oacc
    int32_t t0;              // first stage of the next group; finished when t0 < tau_store
    int32_t tau_store;
    int32_t tauo[2], taue[2];
    int32_t toff[2];         // stage in the frame's stream = tau + toff
    int32_t slot;            // not read (a step walks both slots); keeps the record at 23 words

    __device__ __forceinline__ static uint64_t join(uint32_t lo, uint32_t hi) {
        return ((uint64_t)hi << 32) | lo;
    }
    __device__ __forceinline__ uint32_t *out(int h) const {
        return reinterpret_cast<uint32_t *>(join(out_w[h][0], out_w[h][1]));
    }
    __device__ __forceinline__ void set_out(int h, uint32_t *p) {
        const uint64_t x = reinterpret_cast<uint64_t>(p);
        out_w[h][0] = (uint32_t)x;
        out_w[h][1] = (uint32_t)(x >> 32);
    }
    __device__ __forceinline__ const uint32_t *surv() const {
        return reinterpret_cast<const uint32_t *>(join(surv_w[0], surv_w[1]));
    }
    __device__ __forceinline__ void set_surv(const uint32_t *p) {
        const uint64_t x = reinterpret_cast<uint64_t>(p);
        surv_w[0] = (uint32_t)x;
        surv_w[1] = (uint32_t)(x >> 32);
    }
    __device__ __forceinline__ uint64_t oacc(int h) const { return join(oacc_w[h][0], oacc_w[h][1]); }
    __device__ __forceinline__ void set_oacc(int h, uint64_t v) {
        oacc_w[h][0] = (uint32_t)v;
        oacc_w[h][1] = (uint32_t)(v >> 32);
    }
};
static_assert(sizeof(TbState) == 23 * 4 && alignof(TbState) == 4, "odd-word traceback record");

__device__ __forceinline__ void cp_async_bytes16(void *smem, const void *gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_bytes8(void *smem, const void *gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_bytes4(void *smem, const void *gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int K, int L, bool RADIX4, int NR, int NW, int ES = 0>
struct Traceback {
    static constexpr int NB = K - 1;
    static constexpr int G = NB;                 // stages per group
    static constexpr int LR = ilog2(NR);
    static constexpr int WPF = NR >= 32 ? NR / 32 : 1;
    static constexpr bool EMB = ES != 0;
    static constexpr int FW = ES == 3 ? 4 : 2;   // record field width (bits)
    static constexpr int RPW = 16 / FW;          // registers per record word (per half)
    // survivor records: one per stage (NW words per lane), or with embedded
    // decisions one per ES stages (NR / RPW words per lane, FW-bit fields)
    static constexpr int REC = EMB ? G / ES : G; // records per group
    static constexpr int RW = EMB ? NR / RPW : NW;   // words per record and lane
    static constexpr int SLOT_WORDS = REC * 32 * RW;
    static constexpr int STAGE_WORDS = 2 * SLOT_WORDS;   // per warp
    static_assert(!EMB || (G % ES == 0 && (!RADIX4 || ES == 2)), "embedded decisions: whole records per group");

    // Copies the records of stages t0, t0-1, .., t0-G+1 (those >= tau_store)
    // to a slot (the caller commits the copies as one group).
    __device__ static void issue_slot(const TbState &s, int t0, uint32_t *slot, int wlane) {
#pragma unroll
        for (int g = 0; g < REC; ++g) {
            const int t = t0 - (EMB ? ES * g : g);   // EMB: the last stage of a record
            if (t >= s.tau_store) {
                uint32_t *dst = slot + (g * 32 + wlane) * RW;
                // this lane's words of scratch row t / ES (EMB) or t
                const uint32_t *src = s.surv() + (size_t)(EMB ? (t / ES) : t) * 32 * RW;
                if constexpr (RW == 1) {
                    cp_async_bytes4(dst, src);
                } else if constexpr (RW == 2) {
                    cp_async_bytes8(dst, src);
                } else {
#pragma unroll
                    for (int i = 0; i < RW; i += 4) cp_async_bytes16(dst + i, src + i);
                }
            }
        }
    }

    // Copies the groups of top stages t0 and t0 - G to slots 0 and 1 as one group of copies.
    __device__ static void issue_pair(const TbState &s, int t0, uint32_t *stg, int wlane) {
        issue_slot(s, t0, stg, wlane);
        issue_slot(s, t0 - G, stg + SLOT_WORDS, wlane);
        cp_async_commit();
    }

    __device__ static bool active(const TbState &s) { return s.t0 >= s.tau_store; }

    // Starts the copies of the first two groups.
    __device__ static void begin(TbState &s, uint32_t *stg, int wlane) {
        s.slot = 0;
        issue_pair(s, s.t0, stg, wlane);
    }

    // A step walks the two staged groups: open() before the first group's
    // first record, walk<j>() per record of each group, close() after the
    // second group's last record.
    static constexpr int STEPS = EMB ? G / ES : (RADIX4 ? G / 2 : G);   // walk<> calls per group
    struct Live {
        uint32_t R[2];           // traceback registers of both frames
        const uint32_t *slot;    // staging slot of the group
        bool act;
    };

    // Branch-free: an inactive walk (act false) reads in-bounds staging words
    // and changes nothing that close() keeps, so the embedded-decision walk
    // runs unconditionally (measured 3% faster than a branch around it).
    __device__ static void open(const TbState &s, const uint32_t *stg, Live &v) {
        v.act = active(s);
        cp_async_wait<0>();
        v.slot = stg;
        v.R[0] = s.R[0] & (uint32_t)((1 << NB) - 1);
        v.R[1] = s.R[1] & (uint32_t)((1 << NB) - 1);
    }

    template <int j>
    __device__ static void walk(Live &v, int wlane, unsigned gmask, int grp_base) {
        if (!EMB && !v.act) return;
        auto words = [&](int g, uint32_t (&wd)[RW]) {
            const uint32_t *p = v.slot + (g * 32 + wlane) * RW;
            if constexpr (RW == 1) {
                wd[0] = p[0];
            } else if constexpr (RW == 2) {
                const uint2 x = *reinterpret_cast<const uint2 *>(p);
                wd[0] = x.x; wd[1] = x.y;
            } else {
#pragma unroll
                for (int i = 0; i < RW; i += 4) {
                    const uint4 x = *reinterpret_cast<const uint4 *>(p + i);
                    wd[i] = x.x; wd[i + 1] = x.y; wd[i + 2] = x.z; wd[i + 3] = x.w;
                }
            }
        };
        // The survivor word of register R in frame h, rotated right so that
        // R's decision bit lands at bit position ph.
        auto rotated = [&](const uint32_t (&wd)[RW], int h, uint32_t R, int ph) -> uint32_t {
            uint32_t word, bit;
            if constexpr (NR >= 32) {
                word = pick<WPF>(&wd[h * WPF], (R >> 5) & (uint32_t)(WPF - 1));
                bit = R;
            } else {
                word = wd[0];
                bit = (R & (uint32_t)(NR - 1)) + 16u * (uint32_t)h;
            }
            return __funnelshift_r(word, word, bit - (uint32_t)ph);
        };
        auto owner = [&](uint32_t x, uint32_t R) -> uint32_t {
            if constexpr (L > 1) return __shfl_sync(gmask, x, grp_base + (int)(R >> LR));
            else return x;
        };
        if constexpr (EMB) {
            // record of stages (t-ES+1 .. t): register R's field holds the
            // decision of R at stage t (bit ES-1), the decision at stage t-1
            // of the register it came from (bit ES-2), and so on.  The phases
            // of the record's stages are adjacent (a group starts at phase 0
            // and holds whole records), so one rotation puts every bit in
            // place and one select replaces those bits of R.
            constexpr int phh = ((NB - 1 - ES * j) % NB + NB) % NB;   // phase of stage t
            constexpr int ph0 = phh - (ES - 1);
            static_assert(ph0 >= 0, "a record's phases do not wrap");
            constexpr uint32_t m = ((1u << ES) - 1u) << ph0;
            const uint32_t *rec = v.slot + (j * 32 + wlane) * RW;   // this lane's record
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t R = v.R[h];
                const uint32_t word = rec[(R / RPW) & (uint32_t)(RW - 1)];   // the word holding R
                const uint32_t sh = (uint32_t)FW * (R & (uint32_t)(RPW - 1)) + 16u * (uint32_t)h;
                const uint32_t t = owner(__funnelshift_r(word, word, sh - (uint32_t)ph0), R);
                v.R[h] = (R & ~m) | (t & m);
            }
        } else if constexpr (!RADIX4) {
            constexpr int ph = ((NB - 1 - j) % NB + NB) % NB;   // group starts at -1 mod (K-1)
            uint32_t wd[RW];
            words(j, wd);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t t = owner(rotated(wd, h, v.R[h], ph), v.R[h]);
                v.R[h] = (v.R[h] & ~(1u << ph)) | (t & (1u << ph));
            }
        } else {
            // pairs (t, t-1): t is the second stage of a pair; both decisions
            // of register R sit at the same bit position in the two words
            constexpr int g = 2 * j;
            constexpr int ph2 = ((NB - 1 - g) % NB + NB) % NB;
            constexpr int ph1 = ((NB - 2 - g) % NB + NB) % NB;
            constexpr uint32_t m2 = 1u << ph2, m1 = 1u << ph1;
            uint32_t w2[RW], w1[RW];
            words(g, w2);
            words(g + 1, w1);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t t2 = rotated(w2, h, v.R[h], ph2);
                const uint32_t t1 = rotated(w1, h, v.R[h], ph1);
                const uint32_t t = owner((t2 & m2) | (t1 & ~m2), v.R[h]);
                v.R[h] = (v.R[h] & ~(m2 | m1)) | (t & (m2 | m1));
            }
        }
    }

    // Emits the two groups' decoded bits, refills both slots with the two
    // groups after them and advances.  RB: the registers after group A (the
    // start of group B).
    __device__ static void close(TbState &s, uint32_t *stg, const Live &v, const uint32_t (&RB)[2], int wlane,
                                 int lane) {
        if (!v.act) return;
        const int t0 = s.t0;
        const int tl = t0 - (2 * G - 1);   // lowest stage of group B
        // Each bit position of R is replaced once per group, so a group's
        // decoded bits (the input bit of each stage's state) are the bits of
        // R at the start of the group: group A's from s.R, group B's from RB;
        // stage tl + i is bit i of (R_A << G) | R_B.
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int lo = tl > s.tauo[h] ? tl : s.tauo[h];
            const int hi = (t0 + 1) < s.taue[h] ? (t0 + 1) : s.taue[h];
            if (hi > lo) {
                const int m = hi - lo;
                const uint32_t X = ((s.R[h] & (uint32_t)((1 << NB) - 1)) << G) | RB[h];
                const uint64_t bits = (uint64_t)((X >> (lo - tl)) & ((1u << m) - 1u));
                uint64_t acc = (s.oacc(h) << m) | bits;
                int nb = s.onb[h] + m;
                const int a = lo + s.toff[h];              // stream stage of bit 0
                const int wb = (a + nb - 1) & ~31;         // first stage of the top word
                if (a <= wb) {
                    if (lane == (L > 1 ? h : 0)) s.out(h)[wb >> 5] = (uint32_t)(acc >> (wb - a));
                    nb = wb - a;
                    acc &= (1ull << nb) - 1ull;
                }
                s.set_oacc(h, acc);
                s.onb[h] = nb;
            }
        }
        s.R[0] = v.R[0];
        s.R[1] = v.R[1];
        // refill both slots with the next two groups, then advance
        issue_pair(s, t0 - 2 * G, stg, wlane);
        s.t0 = t0 - 2 * G;
    }

    // The traceback work that belongs after stage S of chunk c of a forward
    // pass (chunks of U stages, a whole number of groups): one step (two
    // groups) after the last stage of every second group, so the state
    // bookkeeping, the wait and the commit are paid once per two groups.
    // (Spreading the records over the stages was measured 2% slower: the
    // forward stages schedule better as whole blocks.)
    template <int S, int U>
    __device__ static void sub(TbState &s, uint32_t *stg, Live &, int wlane, int lane, unsigned gmask,
                               int grp_base, int c) {
        static_assert(U % G == 0, "chunks hold whole groups");
        if constexpr (S % G == G - 1) {
            if ((c * (U / G) + S / G) & 1) step(s, stg, wlane, lane, gmask, grp_base);
        }
    }

    // Walks the two staged groups (those that remain) and refills both slots.
    __device__ static void step(TbState &s, uint32_t *stg, int wlane, int lane, unsigned gmask,
                                int grp_base) {
        Live v;
        open(s, stg, v);
        static_for<STEPS>([&](auto jc) { walk<decltype(jc)::value>(v, wlane, gmask, grp_base); });
        const uint32_t RB[2] = {v.R[0], v.R[1]};
        const bool act = v.act;
        v.slot = stg + SLOT_WORDS;
        v.act = act && s.t0 - G >= s.tau_store;
        static_for<STEPS>([&](auto jc) { walk<decltype(jc)::value>(v, wlane, gmask, grp_base); });
        v.act = act;
        close(s, stg, v, RB, wlane, lane);
    }

    // Walks every remaining group and waits for all copies.
    __device__ static void drain(TbState &s, uint32_t *stg, int wlane, int lane, unsigned gmask,
                                 int grp_base) {
        while (active(s)) step(s, stg, wlane, lane, gmask, grp_base);
        cp_async_wait<0>();
    }
};

// Forward procedure (Algorithm 1) and survivor storage for one pair of frames.
// Called by one group of L lanes; surv is the frame pair's survivor buffer in
// this warp's scratch (wpad_cap stages x 32 lanes x SW words); wlane is the
// lane in the warp.  hook(integral_constant<int, S>, c) runs after stage S of
// every chunk c of U stages (the persistent kernels walk a previous pair's
// traceback there, two groups of K-1 stages every second group).  On return tb
// holds the traceback start of this pair; returns false (tb inactive) if the
// pair does not fit the scratch, which host plans never produce.
template <int K, int BETA, uint64_t GENS, int L, bool RADIX4, typename Hook>
__device__ __forceinline__ bool forward_pair(const FrameTask (&ft)[2], uint32_t *surv, int wpad_cap,
                                             int wlane, int lane, unsigned gmask, int grp_base,
                                             int *status, TbState &tb, Hook &&hook) {
    using Cfg = StreamCfg<K, BETA, GENS, L, RADIX4>;
    using C = typename Cfg::C;
    constexpr int NB = Cfg::NB, NR = Cfg::NR, LR = Cfg::LR, U = Cfg::U, UW = Cfg::UW;
    constexpr int NW = Cfg::NW, WPF = Cfg::WPF, NACC = Cfg::NACC, NWE = Cfg::NWE;
    constexpr bool EMB = Cfg::EMB;
    constexpr uint32_t LV = C::lv(), MV = C::mv();
    constexpr uint32_t F2 = (uint32_t)(Cfg::SC * Cfg::F) * 0x00010001u;
    constexpr uint32_t S2 = (uint32_t)(Cfg::SC * Cfg::HS) * 0x00010001u;   // head start
    // all-equal start and normalisation target: state 0 at F + S (state-0
    // forms), or the minimum over the states at the floor F = 0 (min-normalised)
    constexpr uint32_t SEED0 = (uint32_t)(Cfg::SC * (Cfg::MINNORM ? Cfg::F : Cfg::F + C::S)) * 0x00010001u;
    constexpr int ES = Cfg::ES, RPW = Cfg::RPW, FW = Cfg::FW;

    // ---------------------------------------------------------- frame plan
    int64_t fa[2], fb[2], fo[2], fe[2];
    bool known[2], term[2], valid[2];
    int64_t W[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        fa[h] = ft[h].a; fb[h] = ft[h].b; fo[h] = ft[h].o; fe[h] = ft[h].e;
        valid[h] = ft[h].valid != 0;
        known[h] = ft[h].known != 0;
        term[h] = ft[h].term != 0;
        W[h] = valid[h] ? (fb[h] - fa[h]) : 0;
    }
    const int64_t Wmax = W[0] > W[1] ? W[0] : W[1];
    const int Wpad = (int)(((Wmax + U - 1) / U) * U);
    tb.t0 = -1;
    tb.tau_store = 0;
    tb.slot = 0;
    tb.R[0] = tb.R[1] = 0;
    if (Wpad > wpad_cap) {   // never happens for plans built by the host; refuse, do not overrun
        if (lane == 0) atomicOr(status, 1);
        return false;
    }
    int tau0[2], tauo[2], taue[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        tau0[h] = Wpad - (int)W[h];
        tauo[h] = valid[h] ? tau0[h] + (int)(fo[h] - fa[h]) : Wpad;
        taue[h] = valid[h] ? tau0[h] + (int)(fe[h] - fa[h]) : Wpad;
    }
    const int tau_store = tauo[0] < tauo[1] ? tauo[0] : tauo[1];
    const int reset_at0 = known[0] ? tau0[0] : -1;
    const int reset_at1 = known[1] ? tau0[1] : -1;

    // the traceback's fixed parameters are written now (tb may live in
    // shared memory), so they hold no registers during the forward pass
    tb.set_out(0, ft[0].out);
    tb.set_out(1, ft[1].out);
    tb.set_surv(surv + (size_t)wlane * (EMB ? NWE : NW));
    tb.set_oacc(0, 0u);
    tb.set_oacc(1, 0u);
    tb.onb[0] = tb.onb[1] = 0;
    tb.tau_store = tau_store;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        tb.tauo[h] = tauo[h];
        tb.taue[h] = taue[h];
        tb.toff[h] = (int32_t)(fa[h] - tau0[h]);
    }

    // lane part of the branch output per phase, folded into LLR signs
    uint32_t cbits = 0;
    if constexpr (L > 1) {
#pragma unroll
        for (int ph = 0; ph < NB; ++ph) {
            uint32_t lp = (uint32_t)lane;
            if (ph >= LR) lp &= ~(1u << (ph - LR));
            const uint32_t G = C::rotr(lp << LR, ph) >> 1;
            cbits |= alpha_rt<K, BETA, GENS>(G) << (ph * BETA);
        }
    }

    // ------------------------------------------------------------ metrics
    uint32_t P[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) P[r] = SEED0;   // all-equal: unknown start

    // LLR bytes relative to each frame's first stage; stage tau of the pair is
    // frame stage tau - tau0
    const int8_t *fbase0 = ft[0].llr + fa[0] * BETA, *fbase1 = ft[1].llr + fa[1] * BETA;
    const int32_t hi0 = valid[0] ? (int32_t)W[0] * BETA : 0, hi1 = valid[1] ? (int32_t)W[1] * BETA : 0;
    int32_t vb0 = -tau0[0] * BETA, vb1 = -tau0[1] * BETA;   // offset of the chunk being fetched

    // Scratch rows (a record, or a stage's decision words) of W words per
    // lane, lane-major: row r of lane l starts at word (32 r + l) W.
    // EMB: the record of stages (tau - ES + 1 .. tau) is row tau / ES.
    auto store_row = [&](size_t row, auto const &v) {
        constexpr int W = (int)(sizeof(v) / sizeof(uint32_t));
        uint32_t *dst = surv + (row * 32 + (size_t)wlane) * W;
        if constexpr (W == 1) {
            *dst = v[0];
        } else if constexpr (W == 2) {
            *reinterpret_cast<uint2 *>(dst) = make_uint2(v[0], v[1]);
        } else {
#pragma unroll
            for (int i = 0; i < W; i += 4)
                *reinterpret_cast<uint4 *>(dst + i) = make_uint4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
    };
    auto store_rec = [&](int tau, const uint32_t (&rec)[NWE]) { store_row((size_t)(tau / (ES > 0 ? ES : 1)), rec); };
    auto store_words = [&](int tau, const uint32_t (&wd)[NW]) { store_row((size_t)tau, wd); };

    // runtime +1 / -1 for the FMA-pipe multiply-adds (blocks are one-dimensional)
    const uint32_t one = threadIdx.y + 1u;
    const uint32_t m1 = 0u - one;
    const uint32_t fwmul = one << FW;   // 2^FW: shifts a record word by one field
    const uint32_t mul16 = one << 4, mul64 = one << 6;   // 2-bit fields: shifts by two and three fields
    constexpr bool COROLLARY = LV == (1u << BETA) - 1u && MV == (1u << BETA) - 1u;

    const int nchunks = Wpad / U;
    uint32_t pmin = SEED0;   // ES = 3: per-half minimum metric at the end of the last chunk
    ChunkRaw<UW> nx0, nx1;
    if (nchunks > 0) {
        fetch_chunk<UW>(fbase0, vb0, hi0, nx0);
        fetch_chunk<UW>(fbase1, vb1, hi1, nx1);
    }
    for (int c = 0; c < nchunks; ++c) {
        uint32_t cw0[UW], cw1[UW];
        {
            const ChunkRaw<UW> cur0 = nx0, cur1 = nx1;
            const int32_t cb0 = vb0, cb1 = vb1;
            vb0 += U * BETA;
            vb1 += U * BETA;
            if (c + 1 < nchunks) {
                fetch_chunk<UW>(fbase0, vb0, hi0, nx0);
                fetch_chunk<UW>(fbase1, vb1, hi1, nx1);
            }
            finish_chunk<UW>(fbase0, cb0, hi0, cur0, cw0);
            finish_chunk<UW>(fbase1, cb1, hi1, cur1, cw1);
        }
        uint32_t W1[NW];   // radix-4: decisions of the first stage of a pair
        // embedded form: the normalisation at a chunk boundary is folded
        // into the branch metrics of the chunk's first stage (adding tn to
        // every candidate shifts every new metric by tn, as normalising
        // before the stage would).  Min-normalised forms: tn = -(minimum over
        // the states, taken at the end of the previous chunk) every chunk;
        // the state-0 form: tn = 4(F+S) - (metric of state 0) every
        // NORM_CHUNKS chunks, else 0.
        uint32_t tn = 0, tn1 = 0, tn2 = 0;
        if constexpr (Cfg::MINNORM) {
            tn = sub_s16x2(SEED0, pmin);
            tn2 = add_u16x2(tn, 0x00010001u);   // + the odd candidates' mark of stage 0
        } else if constexpr (EMB) {
            uint32_t ref = P[0];
            if constexpr (L > 1) ref = __shfl_sync(gmask, ref, grp_base);
            tn = (c > 0 && c % Cfg::NORM_CHUNKS == 0) ? sub_s16x2(SEED0, ref) : 0u;
            tn1 = add_u16x2(tn, 0x00010001u);   // -x + tn = ~x + tn1
            tn2 = add_u16x2(tn, 0x00020002u);   // -x + 1 + tn (odd candidates of stage 0)
        }

        static_for<U>([&](auto Sc) {
            constexpr int S = decltype(Sc)::value;
            constexpr int PH = S % NB;
            const int tau = c * U + S;

            // a frame that starts from the reset state gets its head start at
            // its first stage.  Until then its half of every metric is the
            // same value F+S (all-equal start, zero-LLR padding stages and
            // normalisation all keep metrics equal), so adding S to state 0
            // (register 0 of lane 0 at every stage: ROTR of 0 is 0) gives it
            // exactly the lead S over every other state, as in the bound of
            // the metric range.  (Rare: kept as a branch, not predicated.)
            if (__builtin_expect(tau == reset_at0 || tau == reset_at1, 0)) {
                const uint32_t hs = (tau == reset_at0 ? (S2 & 0xFFFFu) : 0u) |
                                    (tau == reset_at1 ? (S2 & 0xFFFF0000u) : 0u);
                if (lane == 0) P[0] = add_u16x2(P[0], hs);
            }

            // ---- branch metrics of this stage (Eq. BM), both frames at once
            uint32_t Lb[BETA], nLb[BETA];
#pragma unroll
            for (int b = 0; b < BETA; ++b) {
                const int j = S * BETA + b;
                const uint32_t k = (uint32_t)(j & 3);
                const uint32_t sel = k | ((k + 8u) << 4) | ((k + 4u) << 8) | ((k + 12u) << 12);
                Lb[b] = prmt(cw0[j >> 2], cw1[j >> 2], sel);   // sign-extended int8 pair
                nLb[b] = neg_s16x2(Lb[b]);
                if constexpr (L > 1) {
                    if ((cbits >> (PH * BETA + b)) & 1u) {
                        const uint32_t t = Lb[b];
                        Lb[b] = nLb[b];
                        nLb[b] = t;
                    }
                }
            }
            // A[x] = sum_b (-1)^{x_b} l_b for every output pattern x
            uint32_t A[1 << BETA];
            A[0] = Lb[0];
            A[1] = nLb[0];
#pragma unroll
            for (int b = 1; b < BETA; ++b) {
#pragma unroll
                for (int x = 0; x < (1 << b); ++x) {
                    A[x | (1 << b)] = add_s16x2(A[x], nLb[b]);
                    A[x] = add_s16x2(A[x], Lb[b]);
                }
            }
            if constexpr (EMB) {
                // ---- embedded decisions.  A metric half is 2^ES m + j: m the
                // path metric (Eq. PM) and j < 2^ES the decisions (Eq. SP0)
                // of the current record of ES stages along the state's
                // survivor.  Odd candidates carry + 2^k at the record's stage
                // k, so the max itself records "the odd predecessor wins or
                // ties" in bit k: with j_even, j_odd < 2^k a tie leaves the
                // odd candidate larger by 2^k + j_odd - j_even > 0, and a
                // metric difference of one (2^ES in these units) outweighs
                // 2^k + j_odd - j_even <= 2^(k+1) - 1 <= 2^ES - 1.  The
                // winner's own bits below k (its decisions at the record's
                // earlier stages) travel with it.  After the record's last
                // stage the fields are stored and cleared: no per-state
                // decision arithmetic.
                constexpr int KS = S % ES;   // stage within the record
                constexpr uint32_t OFF = 0x00010001u << KS;
                [[maybe_unused]] constexpr uint32_t SCM = (0xFFFFu & ~(uint32_t)(Cfg::SC - 1)) * 0x00010001u;
                uint32_t A4[1 << BETA], A4o[1 << BETA];
                if constexpr (Cfg::MINNORM) {
                    // biased pattern sums Ab[x] = A[x] + B in [0, 2B] per half,
                    // from u_b = l_b + 127 in [0, 254]: Ab[x] = sum_b (x_b ?
                    // 254 - u_b : u_b).  Every half of every intermediate and
                    // result is non-negative and below 2^16, so plain 32-bit
                    // arithmetic is exact per half (no masks, no per-half
                    // negation); the scaled sums 2^ES Ab are below 2^13.
                    constexpr uint32_t H127 = 127u * 0x00010001u, H254 = 254u * 0x00010001u;
                    uint32_t Ub[BETA];
#pragma unroll
                    for (int b = 0; b < BETA; ++b) Ub[b] = add_u16x2(Lb[b], H127);
                    uint32_t Ab[1 << BETA];
                    Ab[0] = Ub[0];
                    Ab[1] = H254 - Ub[0];
#pragma unroll
                    for (int b = 1; b < BETA; ++b) {
#pragma unroll
                        for (int x = 0; x < (1 << b); ++x) {
                            Ab[x | (1 << b)] = Ab[x] + (H254 - Ub[b]);
                            Ab[x] = Ab[x] + Ub[b];
                        }
                    }
                    if constexpr (COROLLARY) {
                        // complement patterns: 2^ES (2B - Ab[x])
                        constexpr int FULL = (1 << BETA) - 1;
                        constexpr uint32_t CC = (uint32_t)((2 * C::B) << ES) * 0x00010001u;
#pragma unroll
                        for (int x = 0; x < (1 << (BETA - 1)); ++x) {
                            const uint32_t a4 = Ab[x] << ES;
                            const uint32_t cm = CC - a4;
                            if constexpr (S == 0) {   // with the folded normalisation
                                A4[x] = add_u16x2(a4, tn);
                                A4[x ^ FULL] = add_u16x2(cm, tn);
                                A4o[x ^ FULL] = add_u16x2(cm, tn2);
                                A4o[x] = add_u16x2(A4[x], OFF);
                            } else {
                                A4[x] = a4;
                                A4[x ^ FULL] = cm;
                                A4o[x ^ FULL] = (CC + OFF) - a4;
                                A4o[x] = a4 + OFF;
                            }
                        }
                    } else {
#pragma unroll
                        for (int x = 0; x < (1 << BETA); ++x) {
                            const uint32_t a4 = Ab[x] << ES;
                            if constexpr (S == 0) {
                                A4[x] = add_u16x2(a4, tn);
                                A4o[x] = add_u16x2(A4[x], OFF);
                            } else {
                                A4[x] = a4;
                                A4o[x] = a4 + OFF;
                            }
                        }
                    }
                } else if constexpr (COROLLARY) {
                    // complement patterns have the negated metric: scale half
                    // of the table, negate per half (~x + 1) for the rest
                    constexpr int FULL = (1 << BETA) - 1;
#pragma unroll
                    for (int x = 0; x < (1 << (BETA - 1)); ++x) {
                        const uint32_t a4 = (A[x] << ES) & SCM;   // 2^ES delta per half
                        const uint32_t n = ~a4;
                        if constexpr (S == 0) {   // with the folded normalisation
                            A4[x] = add_u16x2(a4, tn);
                            A4[x ^ FULL] = add_u16x2(n, tn1);
                            A4o[x ^ FULL] = add_u16x2(n, tn2);
                        } else {
                            A4[x] = a4;
                            A4[x ^ FULL] = add_u16x2(n, 0x00010001u);
                            A4o[x ^ FULL] = add_u16x2(n, 0x00010001u + OFF);
                        }
                        A4o[x] = add_u16x2(A4[x], OFF);
                    }
                } else {
#pragma unroll
                    for (int x = 0; x < (1 << BETA); ++x) {
                        A4[x] = (A[x] << ES) & SCM;
                        if constexpr (S == 0) A4[x] = add_u16x2(A4[x], tn);
                        A4o[x] = add_u16x2(A4[x], OFF);
                    }
                }
                auto butterfly_e = [&](int ra) {
                    const int rb = ra | (1 << PH);
                    const uint32_t a = C::alpha(C::rotr((uint32_t)ra, PH) >> 1);
                    const uint32_t Pa = P[ra], Pb = P[rb];
                    const uint32_t cb0 = add_u16x2(Pb, A4o[a ^ LV]);        // odd -> j0
                    const uint32_t cb1 = add_u16x2(Pb, A4o[a ^ MV ^ LV]);   // odd -> j1
                    P[ra] = addmax_u16x2(Pa, A4[a], cb0);                   // even -> j0
                    P[rb] = addmax_u16x2(Pa, A4[a ^ MV], cb1);              // even -> j1
                };
                auto cross_e = [&](int r) {   // partner register in lane ^ (1 << (PH - LR))
                    constexpr int lb = PH >= LR ? PH - LR : 0;
                    const uint32_t xb = ((uint32_t)lane >> lb) & 1u;   // 1: this lane holds R_b (odd)
                    const uint32_t a = C::alpha(C::rotr((uint32_t)r, PH) >> 1);
                    const uint32_t own = P[r];
                    const uint32_t oth = __shfl_xor_sync(gmask, own, 1 << lb);
                    const uint32_t d_own = xb ? A4o[a ^ MV ^ LV] : A4[a];
                    const uint32_t d_oth = xb ? A4[a ^ MV] : A4o[a ^ LV];
                    P[r] = addmax_u16x2(own, d_own, add_u16x2(oth, d_oth));
                };
                if constexpr (PH < LR) {
#pragma unroll
                    for (int r = 0; r < NR; ++r)
                        if (!(r & (1 << PH))) butterfly_e(r);
                } else {
#pragma unroll
                    for (int r = 0; r < NR; ++r) cross_e(r);
                }
                if constexpr (KS == ES - 1) {
                    // record word m: register RPW m + i at bits FW i (frame 0)
                    // and 16 + FW i (frame 1).  Two forms, alternating by word
                    // so that the ALU and FMA pipes stay balanced (measured:
                    // either form alone is slower):
                    //  * byte permutes: the low byte of each half holds a
                    //    register's field (and metric bits above it, which
                    //    the traceback masks off); prmt(P[a], P[b], 0x6240)
                    //    puts a's low bytes at bits 0 and 16 and b's at 8 and
                    //    24, a multiply-add shifts a second such word by one
                    //    field and a select merges them; the fields are then
                    //    cleared by selects (ALU);
                    //  * extracted fields: d = P & FM (ALU), cleared by a
                    //    multiply-add P - d and gathered by multiply-adds
                    //    acc = 16 acc + d (FMA pipe).
                    constexpr uint32_t FM = ((1u << ES) - 1u) * 0x00010001u;
                    auto merge = [](uint32_t a, uint32_t b, uint32_t keep_a) { return (a & keep_a) | (b & ~keep_a); };
                    if constexpr (Cfg::MINNORM && S == U - 1) {
                        // the minimum over the states for the next chunk's
                        // normalisation: min of 8 m + j, fields masked off
                        pmin = min_tree<NR>(P) & ~FM;
                        if constexpr (L > 1) {
#pragma unroll
                            for (int m = 1; m < L; m <<= 1)
                                pmin = min_u16x2(pmin, __shfl_xor_sync(gmask, pmin, m));
                        }
                    }
                    uint32_t rec[NWE];
#pragma unroll
                    for (int m = 0; m < NWE; ++m) {
                        const int r0 = RPW * m;
                        if constexpr (RPW == 4) {
                            if (m & 1) {
                                uint32_t acc = 0;
#pragma unroll
                                for (int i = RPW - 1; i >= 0; --i) {
                                    const int r = r0 + i;
                                    const uint32_t d = P[r] & FM;
                                    P[r] = imad(d, m1, P[r]);
                                    acc = (i == RPW - 1) ? d : imad(acc, fwmul, d);
                                }
                                rec[m] = acc;
                            } else {
                                const uint32_t x = prmt(P[r0], P[r0 + 2], 0x6240u);
                                const uint32_t y = prmt(P[r0 + 1], P[r0 + 3], 0x6240u);
                                rec[m] = merge(x, imad(y, fwmul, 0u), 0x07070707u);
#pragma unroll
                                for (int i = 0; i < RPW; ++i) P[r0 + i] &= ~FM;
                            }
                        } else if (K >= 9 && (m & 1)) {
                            // 2-bit fields, extracted (K=9 only: the two forms
                            // alternating were measured 4.5% faster for the K=9
                            // stream kernel and 1.6% slower for K=7 radix-4,
                            // whose records are rarer per instruction)
                            static_assert(RPW == 8, "2-bit or 4-bit record fields");
                            uint32_t acc = 0;
#pragma unroll
                            for (int i = RPW - 1; i >= 0; --i) {
                                const int r = r0 + i;
                                const uint32_t d = P[r] & FM;
                                P[r] = imad(d, m1, P[r]);
                                acc = (i == RPW - 1) ? d : imad(acc, fwmul, d);
                            }
                            rec[m] = acc;
                        } else {
                            // 2-bit fields: registers r0 + i, r0 + i + 4 shifted by 2 i bits
                            static_assert(RPW == 8, "2-bit or 4-bit record fields");
                            const uint32_t x0 = prmt(P[r0], P[r0 + 4], 0x6240u);
                            const uint32_t x1 = imad(prmt(P[r0 + 1], P[r0 + 5], 0x6240u), fwmul, 0u);
                            const uint32_t x2 = imad(prmt(P[r0 + 2], P[r0 + 6], 0x6240u), mul16, 0u);
                            const uint32_t x3 = imad(prmt(P[r0 + 3], P[r0 + 7], 0x6240u), mul64, 0u);
                            rec[m] = merge(merge(x0, x1, 0x03030303u), merge(x2, x3, 0x30303030u), 0x0F0F0F0Fu);
#pragma unroll
                            for (int i = 0; i < RPW; ++i) P[r0 + i] &= ~FM;
                        }
                    }
                    if (tau >= tau_store) store_rec(tau, rec);
                }
                hook(Sc, c);
                return;
            }

            // decision offsets: E0[a] = d(odd->j0) - d(even->j0) + 0x8000 and
            // E1[a] = d(odd->j1) - d(even->j1) + 0x8000 per half, for main output a
            uint32_t E0[1 << BETA], E1[1 << BETA];
            if constexpr (COROLLARY) {
                // the odd branches carry the complement pattern: E = 0x8000 + 2 A
                uint32_t T2[1 << BETA];
#pragma unroll
                for (int x = 0; x < (1 << BETA); ++x) T2[x] = add_u16x2(add_s16x2(A[x], A[x]), 0x80008000u);
#pragma unroll
                for (int x = 0; x < (1 << BETA); ++x) {
                    E0[x] = T2[x ^ LV];
                    E1[x] = T2[x];
                }
            } else {
#pragma unroll
                for (int x = 0; x < (1 << BETA); ++x) {
                    E0[x] = add_u16x2(sub_s16x2(A[x ^ LV], A[x]), 0x80008000u);
                    E1[x] = add_u16x2(sub_s16x2(A[x ^ MV ^ LV], A[x ^ MV]), 0x80008000u);
                }
            }

            // ---- add-compare-select (Eq. PM), decisions (Eq. SP0), packing
            uint32_t X[NR];
            uint32_t acc[NACC];
#pragma unroll
            for (int i = 0; i < NACC; ++i) acc[i] = 0;

            auto butterfly = [&](int ra) {   // local pair (ra, ra | 1 << PH)
                const int rb = ra | (1 << PH);
                const uint32_t a = C::alpha(C::rotr((uint32_t)ra, PH) >> 1);
                const uint32_t Pa = P[ra], Pb = P[rb];
                // even -> j0: alpha, odd -> j0: alpha^LV, even -> j1: alpha^MV, odd -> j1: alpha^MV^LV
                const uint32_t cb0 = add_u16x2(Pb, A[a ^ LV]);        // FMA pipe
                const uint32_t cb1 = add_u16x2(Pb, A[a ^ MV ^ LV]);   // FMA pipe
                const uint32_t u = imad(Pa, m1, Pb);                  // Pb - Pa, FMA pipe
                P[ra] = addmax_u16x2(Pa, A[a], cb0);                  // ALU (fused add + max)
                P[rb] = addmax_u16x2(Pa, A[a ^ MV], cb1);             // ALU
                // bit 15 / 31 set: the odd predecessor wins or ties
                X[ra] = u + E0[a];
                X[rb] = imad(u, one, E1[a]);
            };
            auto cross = [&](int r) {   // partner register in lane ^ (1 << (PH - LR))
                constexpr int lb = PH >= LR ? PH - LR : 0;
                const uint32_t xb = ((uint32_t)lane >> lb) & 1u;   // 1: this lane holds R_b
                const uint32_t a = C::alpha(C::rotr((uint32_t)r, PH) >> 1);
                const uint32_t own = P[r];
                const uint32_t oth = __shfl_xor_sync(gmask, own, 1 << lb);
                const uint32_t d_own = xb ? A[a ^ MV ^ LV] : A[a];
                const uint32_t d_oth = xb ? A[a ^ MV] : A[a ^ LV];
                // holder of R_a: bit = (c_oth >= c_own); holder of R_b: bit = !(c_own >= c_oth),
                // inverted back after packing
                uint32_t e;
                if constexpr (COROLLARY) e = E0[a];
                else e = add_u16x2(sub_s16x2(d_oth, d_own), 0x80008000u);
                e -= xb ? 0x00010001u : 0u;
                P[r] = addmax_u16x2(own, d_own, add_u16x2(oth, d_oth));
                X[r] = imad(own, m1, oth) + e;
            };
            // 16 registers -> acc[blk]: each prmt turns the decision bits of
            // registers r1, r1+8 (both halves) into bytes 0x00/0xFF; a depth-3
            // tree of bitwise selects (one LOP3 each) then puts register
            // 16 blk + kk at bit kk of every byte
            auto pack_block = [&](int blk) {
                uint32_t t[8];
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) t[kk] = prmt(X[16 * blk + kk], X[16 * blk + kk + 8], 0xFDB9u);
                auto sel = [](uint32_t a, uint32_t b, uint32_t m) { return (a & m) | (b & ~m); };
                const uint32_t m0 = sel(t[0], t[1], 0x01010101u), m1 = sel(t[2], t[3], 0x04040404u);
                const uint32_t m2 = sel(t[4], t[5], 0x10101010u), m3 = sel(t[6], t[7], 0x40404040u);
                acc[blk] = sel(sel(m0, m1, 0x03030303u), sel(m2, m3, 0x30303030u), 0x0F0F0F0Fu);
            };

            if constexpr (NR >= 16) {
                if constexpr (PH < LR) {
                    // process blocks of 16 registers (block pairs when the
                    // butterfly partner is in another block) and pack each
                    // block as soon as it is complete
                    constexpr int PB = PH >= 4 ? (1 << (PH - 4)) : 0;   // partner block bit
#pragma unroll
                    for (int blk = 0; blk < NR / 16; ++blk) {
                        if (blk & PB) continue;
#pragma unroll
                        for (int r = 16 * blk; r < 16 * blk + 16; ++r)
                            if (!(r & (1 << PH))) butterfly(r);
                        pack_block(blk);
                        if (PB) pack_block(blk | PB);
                    }
                } else {
#pragma unroll
                    for (int blk = 0; blk < NR / 16; ++blk) {
#pragma unroll
                        for (int r = 16 * blk; r < 16 * blk + 16; ++r) cross(r);
                        pack_block(blk);
                    }
                }
            } else {
                if constexpr (PH < LR) {
#pragma unroll
                    for (int r = 0; r < NR; ++r)
                        if (!(r & (1 << PH))) butterfly(r);
                } else {
#pragma unroll
                    for (int r = 0; r < NR; ++r) cross(r);
                }
            }

            // ---- regroup into per-frame words, natural bit order
            uint32_t wd[NW];
            if constexpr (NR >= 32) {
#pragma unroll
                for (int m = 0; m < WPF; ++m) {
                    wd[m] = prmt(acc[2 * m], acc[2 * m + 1], 0x6420u);
                    wd[WPF + m] = prmt(acc[2 * m], acc[2 * m + 1], 0x7531u);
                }
            } else if constexpr (NR == 16) {
                wd[0] = prmt(acc[0], acc[0], 0x3120u);
            } else {
                uint32_t x = 0;
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    x |= ((X[r] >> 15) & 1u) << r | ((X[r] >> 31) & 1u) << (16 + r);
                wd[0] = x;
            }
            if constexpr (PH >= LR) {
                const uint32_t inv = 0u - (((uint32_t)lane >> (PH - LR)) & 1u);
#pragma unroll
                for (int i = 0; i < NW; ++i) wd[i] ^= inv;
            }

            if constexpr (!RADIX4) {
                if (tau >= tau_store) store_words(tau, wd);
            } else if constexpr ((S & 1) == 0) {
#pragma unroll
                for (int i = 0; i < NW; ++i) W1[i] = wd[i];
            } else {
                // second stage of a pair: low[R] = W1[R with bit PH := d_m(R)]
                uint32_t lo_w[NW];
                if constexpr (PH < 5 && PH < LR) {
                    constexpr uint32_t m1 = bitk_mask(PH), m0 = ~m1;
                    constexpr int sh = 1 << PH;
#pragma unroll
                    for (int i = 0; i < NW; ++i) {
                        const uint32_t e0 = (W1[i] & m0) | ((W1[i] & m0) << sh);
                        const uint32_t e1 = (W1[i] & m1) | ((W1[i] & m1) >> sh);
                        lo_w[i] = (wd[i] & e1) | (~wd[i] & e0);
                    }
                } else if constexpr (PH < LR) {
                    constexpr int wb = PH >= 5 ? (1 << (PH - 5)) : 0;   // word-index bit (NR >= 64)
#pragma unroll
                    for (int i = 0; i < NW; ++i) {
                        const int base = (i / WPF) * WPF, w = i % WPF;
                        const uint32_t e0 = W1[base + (w & ~wb)], e1 = W1[base + (w | wb)];
                        lo_w[i] = (wd[i] & e1) | (~wd[i] & e0);
                    }
                } else {
                    constexpr int lb = PH - LR;
                    const bool xb = ((lane >> lb) & 1) != 0;
#pragma unroll
                    for (int i = 0; i < NW; ++i) {
                        const uint32_t oth = __shfl_xor_sync(gmask, W1[i], 1 << lb);
                        const uint32_t e0 = xb ? oth : W1[i], e1 = xb ? W1[i] : oth;
                        lo_w[i] = (wd[i] & e1) | (~wd[i] & e0);
                    }
                }
                if (tau >= tau_store) {
                    store_words(tau, wd);
                    store_words(tau - 1, lo_w);
                }
            }
            hook(Sc, c);
        });

        // ---- normalisation: subtract state 0's metric, add F+S, clamp at F
        if (!EMB && (c + 1) % Cfg::NORM_CHUNKS == 0) {
            uint32_t ref = P[0];
            if constexpr (L > 1) ref = __shfl_sync(gmask, ref, grp_base);
            const uint32_t t = sub_s16x2(SEED0, ref);
#pragma unroll
            for (int r = 0; r < NR; ++r) P[r] = max_s16x2(add_s16x2(P[r], t), F2);
        }
    }

    // ------------------------------------------------- traceback start state
    // After Wpad stages (a multiple of K-1) register R holds state R again.
    // A frame that starts from the reset state and has fewer than K-1
    // stages can only be in a state whose low K-1-W bits are zero (the
    // others are -infinity for Algorithm 1 with a known start); the finite
    // head start does not keep every such state below them, so they are
    // left out of the argmax explicitly.
    uint32_t R[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint32_t unreach = (known[h] && W[h] < NB) ? ((1u << (NB - (int)W[h])) - 1u) : 0u;
        uint32_t best = 0;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const uint32_t v = h ? (P[r] >> 16) : (P[r] & 0xFFFFu);
            const uint32_t Rg = ((uint32_t)lane << LR) | (uint32_t)r;
            const uint32_t key = (v << 16) | (0xFFFFu - Rg);
            best = best > key ? best : key;
        }
        if (__builtin_expect(unreach != 0u, 0)) {
            best = 0;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const uint32_t v = h ? (P[r] >> 16) : (P[r] & 0xFFFFu);
                const uint32_t Rg = ((uint32_t)lane << LR) | (uint32_t)r;
                const uint32_t key = (Rg & unreach) ? 0u : ((v << 16) | (0xFFFFu - Rg));
                best = best > key ? best : key;
            }
        }
        if constexpr (L > 1) {
#pragma unroll
            for (int m = 1; m < L; m <<= 1) {
                const uint32_t o = __shfl_xor_sync(gmask, best, m);
                best = best > o ? best : o;
            }
        }
        R[h] = term[h] ? 0u : (0xFFFFu - (best & 0xFFFFu));
    }

    // optional canonical final metrics (lambda - min lambda), for parity checks
    if (ft[0].pm || ft[1].pm) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t mn = 0xFFFFu;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const uint32_t v = h ? (P[r] >> 16) : (P[r] & 0xFFFFu);
                mn = mn < v ? mn : v;
            }
            if constexpr (L > 1) {
#pragma unroll
                for (int m = 1; m < L; m <<= 1) {
                    const uint32_t o = __shfl_xor_sync(gmask, mn, m);
                    mn = mn < o ? mn : o;
                }
            }
            if (ft[h].pm) {
                int32_t *dst = ft[h].pm + ((int64_t)lane << LR);
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const uint32_t v = h ? (P[r] >> 16) : (P[r] & 0xFFFFu);
                    dst[r] = ((int32_t)v - (int32_t)mn) / Cfg::SC;
                }
            }
        }
    }

    tb.R[0] = R[0];
    tb.R[1] = R[1];
    tb.t0 = Wpad - 1;
    return true;
}

// Segmented decode of one stream: frame pair q = (2q, 2q+1) per group of L lanes.
template <int K, int BETA, uint64_t GENS, int L, bool RADIX4, int NT>
__global__ void __launch_bounds__(NT) stream_kernel(const StreamParams p) {
    constexpr int NS = 1 << (K - 1);
    using Cfg = StreamCfg<K, BETA, GENS, L, RADIX4>;
    using Tb = Traceback<K, L, RADIX4, Cfg::NR, Cfg::NW, Cfg::ES>;
    __shared__ TbState tbs[NT];
    __shared__ __align__(16) uint32_t stg[NT / 32][Tb::STAGE_WORDS];
    const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int64_t q = gtid / L;
    const int lane = (int)(gtid % L);
    if (q >= p.n_pairs) return;   // whole lane groups leave together
    const int wlane = (int)(threadIdx.x & 31u);
    const unsigned gmask = (L == 32) ? 0xFFFFFFFFu : (((1u << L) - 1u) << (wlane & ~(L - 1)));
    const int grp_base = wlane & ~(L - 1);
    FrameTask ft[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t s = 2 * q + h;
        ft[h] = frame_task(p.llr, p.out, p.pm_out ? p.pm_out + s * NS : nullptr, s, p.n_win,
                           p.n_info, p.T, p.f, p.v, p.flags);
    }
    uint32_t *surv = p.surv + (size_t)(gtid >> 5) * (size_t)p.wpad_max * 32u * (size_t)Cfg::SW;
    TbState &st = tbs[threadIdx.x];
    forward_pair<K, BETA, GENS, L, RADIX4>(ft, surv, p.wpad_max, wlane, lane, gmask, grp_base, p.status,
                                           st, [](auto, int) {});
    uint32_t *my_stg = stg[threadIdx.x >> 5];
    if (Tb::active(st)) {
        Tb::begin(st, my_stg, wlane);
        Tb::drain(st, my_stg, wlane, lane, gmask, grp_base);
    }
}

}  // namespace vd
