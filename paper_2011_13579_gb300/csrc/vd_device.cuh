// Device-side building blocks of the GB300 Viterbi decoder.
//
// Arithmetic model (int8 LLRs, exact):
//   * a register holds the path metrics of ONE state for TWO frames, as the
//     two 16-bit halves (frame 0 low, frame 1 high).  Every add-compare-select
//     is then a pure 16x2 SIMD instruction; the two frames never interact.
//   * metrics live in unsigned 16-bit halves.  Every N stages they are
//     normalised: subtract the metric of state 0, add F + S, clamp below at F.
//     S = (K-1)(delta_max - delta_min) + 1 bounds the spread of live metrics
//     (and is the head start given to state 0 of a frame that starts from the
//     reset state), B = beta * 127 bounds |branch metric| and F = (N+1) B.
//     Between normalisations a metric moves by at most B per stage, so every
//     metric and every candidate metric + branch metric stays in [0, 32767]
//     and the packed 16-bit additions and maxima are exact.  Subtracting a
//     per-stage constant from every metric changes no decision (Eq. PM is
//     invariant under it); the clamp only touches states that are not
//     reachable from the known start state, whose candidates lose every
//     comparison anyway, and it is gone after K-1 stages.
//   * the decision bit of Eq. SP0 (1 = the odd predecessor p1 = 2f+1 wins,
//     ties included, as Algorithm 1's strict ">" gives) is bit 15 / bit 31 of
//     the 32-bit sum  c_odd - c_even + 0x8000 (per half), which one 3-input
//     integer add computes without carries crossing the halves.
//   * embedded form (radix-2 K=7): a half holds 8 m + j, where the three
//     low bits j are the decisions of the current group of three stages
//     along the state's survivor.  The odd candidate of stage k of the group
//     carries + 2^k, so the max itself sets bit k exactly when the odd
//     predecessor wins or ties and carries the winner's lower bits along;
//     the fields are stored and cleared after the group.  Every chunk of
//     U = 6 stages starts by subtracting the minimum over the states down to
//     the floor F = U B (folded into the branch metrics of its first stage,
//     no clamp), and a frame that starts from the reset state gets the
//     code's tight head start HT (Code::HT) instead of S; the bound is
//     8 (F + HT + (2 (K-2) + U) B) + 7 <= 65535 (see StreamCfg).  A two-stage
//     form (4 m + j, state 0 as the reference every N = 18 stages, bound
//     4 (F + 2S + (N+1) B) + 3 <= 65535) serves codes where three stages do
//     not fit.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace vd {

// ------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t add_u16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("add.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t add_s16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("add.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// per-half modular subtraction (PTX has no 16x2 form of sub); only used in
// per-stage set-up, never per state
__device__ __forceinline__ uint32_t sub_s16x2(uint32_t a, uint32_t b) {
    return __vsub2(a, b);
}
__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t max_s16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// max(a + b, c) per unsigned half
__device__ __forceinline__ uint32_t addmax_u16x2(uint32_t a, uint32_t b, uint32_t c) {
    return max_u16x2(add_u16x2(a, b), c);
}
// a * b + c on the FMA pipe (IMAD).  Callers pass b = +1 / -1 held in a
// register whose value the compiler cannot know, so the multiply-add stays an
// IMAD instead of becoming an ALU-pipe add.
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
// per-half two's-complement negation (no 16x2 subtract exists)
__device__ __forceinline__ uint32_t neg_s16x2(uint32_t x) { return add_u16x2(~x, 0x00010001u); }
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}
__device__ __forceinline__ uint32_t funnel_r(uint32_t lo, uint32_t hi, uint32_t sh) {
    return __funnelshift_r(lo, hi, sh);
}

// ------------------------------------------------- compile-time code facts

// Generators are packed 16 bits each into a 64-bit template argument.
__host__ __device__ constexpr uint32_t gen_of(uint64_t gens, int b) {
    return (uint32_t)((gens >> (16 * b)) & 0xFFFFu);
}
__host__ __device__ constexpr int parity32(uint32_t x) {
    int p = 0;
    while (x) { p ^= (int)(x & 1u); x >>= 1; }
    return p;
}

template <int K, int BETA, uint64_t GENS>
struct Code {
    static constexpr int NB = K - 1;             // bits of a state index
    static constexpr int NS = 1 << NB;           // number of states
    static constexpr uint32_t MASK = NS - 1;
    static constexpr int B = BETA * 127;         // |branch metric| bound for int8 LLRs
    static constexpr int RANGE = 2 * B;          // delta_max - delta_min
    static constexpr int S = (K - 1) * RANGE + 1;  // head start / normalisation offset

    // Tight head start.  A path from a start state D != 0 can meet the path
    // from state 0 at a state j within K-1 stages only if both carry the
    // same inputs (j holds them), so their outputs differ only through the
    // bits of D still in the register: at the i-th stage the register
    // differs by D >> (i-1).  DMAX is the largest number of differing output
    // bits over all D, and 2 * 127 per differing bit bounds the lead such a
    // path can take over the path from state 0: HT = 254 DMAX + 1 keeps the
    // path from state 0 strictly ahead wherever the two meet.  (States not
    // yet reachable from state 0 may still lead their own comparisons in a
    // frame shorter than K-1 stages; the traceback start leaves them out.)
    __host__ __device__ static constexpr int dmax() {
        int best = 0;
        for (uint32_t D = 1; D < (uint32_t)NS; ++D) {
            int d = 0;
            for (int i = 0; i < NB; ++i)
                for (int b = 0; b < BETA; ++b) d += parity32(gen_of(GENS, b) & (D >> i));
            best = d > best ? d : best;
        }
        return best;
    }
    static constexpr int DMAX = dmax();
    static constexpr int HT = 2 * 127 * DMAX + 1;
    static_assert(HT <= S, "the tight head start never exceeds the loose one");

    // output pattern (beta bits, bit b = output b) of the branch leaving state s on input u
    __host__ __device__ static constexpr uint32_t out(uint32_t s, int u) {
        uint32_t r = ((uint32_t)u << (K - 1)) | s, a = 0;
        for (int b = 0; b < BETA; ++b) a |= (uint32_t)parity32(gen_of(GENS, b) & r) << b;
        return a;
    }
    // main output of butterfly g: branch 2g -> g (Thm. 2's alpha^{i0,j0})
    __host__ __device__ static constexpr uint32_t alpha(uint32_t g) { return out(2u * g, 0); }
    // Thm. 2: alpha^{i1,j0} = alpha ^ LV, alpha^{i0,j1} = alpha ^ MV, alpha^{i1,j1} = alpha ^ MV ^ LV
    __host__ __device__ static constexpr uint32_t lv() {
        uint32_t a = 0;
        for (int b = 0; b < BETA; ++b) a |= (gen_of(GENS, b) & 1u) << b;
        return a;
    }
    __host__ __device__ static constexpr uint32_t mv() {
        uint32_t a = 0;
        for (int b = 0; b < BETA; ++b) a |= ((gen_of(GENS, b) >> (K - 1)) & 1u) << b;
        return a;
    }
    __host__ __device__ static constexpr uint32_t rotr(uint32_t x, int k) {
        k %= NB;
        return k == 0 ? (x & MASK) : (((x >> k) | (x << (NB - k))) & MASK);
    }
};

// Runtime alpha of a butterfly index (linear over GF(2)), for lane offsets.
template <int K, int BETA, uint64_t GENS>
__device__ __forceinline__ uint32_t alpha_rt(uint32_t g) {
    uint32_t r = 2u * g, a = 0;
#pragma unroll
    for (int b = 0; b < BETA; ++b) a |= (uint32_t)(__popc(gen_of(GENS, b) & r) & 1) << b;
    return a;
}

// ------------------------------------------------------------- frame plan

// Frame s of a stream: decodes stages [o, e), runs the trellis over [a, b).
struct Frame {
    int64_t a, b, o, e;
    bool known_start;   // starts at stage 0 from the reset state
    bool term_end;      // ends at the end of a terminated stream (trace from state 0)
};

__host__ __device__ __forceinline__ Frame frame_of(int64_t s, int64_t n_info, int64_t T,
                                                   int64_t f, int64_t v, uint32_t flags) {
    Frame w;
    w.o = s * f;
    w.e = (s + 1) * f < n_info ? (s + 1) * f : n_info;
    w.a = w.o - v > 0 ? w.o - v : 0;
    w.b = (s + 1) * f + v < T ? (s + 1) * f + v : T;
    w.known_start = (w.a == 0) && !(flags & 2u);
    w.term_end = (w.b == T) && (flags & 1u);
    return w;
}

}  // namespace vd
