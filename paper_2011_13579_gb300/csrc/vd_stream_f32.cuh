// Frame-pair decoder with fp16 received LLRs and fp32 path metrics (the
// precision study of Sec. IX-B: the channel values in half precision, the
// accumulated metrics in single precision).  Same frame plan, register
// rotation, lane split, survivor layout and traceback as the integer decoder;
// the two frames of a pair live in two fp32 register arrays.
//
// Decisions: d = (c_odd >= c_even), read from the sign of c_odd - c_even
// computed from the same rounded candidates the maximum uses (an exact tie
// gives +0, so the odd predecessor wins it, as in Algorithm 1).  The metric of
// state 0 is subtracted from every metric every normalisation period, which
// keeps magnitudes (and so rounding) small; the reset start gives every state
// but 0 the metric -1e30, which no finite path metric approaches.
#pragma once
#include <cuda_fp16.h>

#include "vd_stream.cuh"

namespace vd {

template <int K, int BETA, uint64_t GENS, int L>
struct StreamCfgF32 {
    using C = Code<K, BETA, GENS>;
    static constexpr int NB = C::NB;
    static constexpr int NS = C::NS;
    static constexpr int NR = NS / L;
    static constexpr int LR = ilog2(NR);
    static constexpr int U = chunk_stages(K, 2 * BETA);   // 2 bytes per LLR
    static constexpr int UW = U * BETA / 2;               // 32-bit words per chunk per frame
    static constexpr int NW = 2 * (NR / 32);              // survivor words per lane per stage
    static constexpr int NORM_CHUNKS = 1;
    static_assert(NR >= 32 && NR % 32 == 0, "the fp32 decoder needs 32k registers per lane");
};

__device__ __forceinline__ float half_at(uint32_t word, int hi) {
    const unsigned short bits = (unsigned short)(hi ? (word >> 16) : (word & 0xFFFFu));
    return __half2float(__ushort_as_half(bits));
}

template <int K, int BETA, uint64_t GENS, int L>
__device__ __forceinline__ bool forward_pair_f32(const FrameTask (&ft)[2], uint32_t *surv, int wpad_cap,
                                                 int wlane, int lane, unsigned gmask, int grp_base,
                                                 int *status, TbState &tb) {
    using Cfg = StreamCfgF32<K, BETA, GENS, L>;
    using C = typename Cfg::C;
    constexpr int NB = Cfg::NB, NR = Cfg::NR, LR = Cfg::LR, U = Cfg::U, UW = Cfg::UW, NW = Cfg::NW;
    constexpr int WPF = NR / 32;
    constexpr uint32_t LV = C::lv(), MV = C::mv();
    constexpr float NEG = -1e30f;

    int64_t fa[2], fb[2], W[2];
    bool valid[2], known[2], term[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        fa[h] = ft[h].a;
        fb[h] = ft[h].b;
        valid[h] = ft[h].valid != 0;
        known[h] = ft[h].known != 0;
        term[h] = ft[h].term != 0;
        W[h] = valid[h] ? fb[h] - fa[h] : 0;
    }
    const int64_t Wmax = W[0] > W[1] ? W[0] : W[1];
    const int Wpad = (int)(((Wmax + U - 1) / U) * U);
    tb.t0 = -1;
    tb.tau_store = 0;
    if (Wpad > wpad_cap) {
        if (lane == 0) atomicOr(status, 1);
        return false;
    }
    int tau0[2], tauo[2], taue[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        tau0[h] = Wpad - (int)W[h];
        tauo[h] = valid[h] ? tau0[h] + (int)(ft[h].o - fa[h]) : Wpad;
        taue[h] = valid[h] ? tau0[h] + (int)(ft[h].e - fa[h]) : Wpad;
    }
    const int tau_store = tauo[0] < tauo[1] ? tauo[0] : tauo[1];
    const int reset0 = known[0] ? tau0[0] : -1;
    const int reset1 = known[1] ? tau0[1] : -1;

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

    float P[2][NR];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < NR; ++r) P[h][r] = 0.0f;

    // fp16 LLR bytes relative to each frame's first stage
    const int8_t *fbase0 = ft[0].llr + fa[0] * BETA * 2, *fbase1 = ft[1].llr + fa[1] * BETA * 2;
    const int32_t hi0 = valid[0] ? (int32_t)W[0] * BETA * 2 : 0, hi1 = valid[1] ? (int32_t)W[1] * BETA * 2 : 0;
    int32_t vb0 = -tau0[0] * BETA * 2, vb1 = -tau0[1] * BETA * 2;

    const int nchunks = Wpad / U;
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
            vb0 += U * BETA * 2;
            vb1 += U * BETA * 2;
            if (c + 1 < nchunks) {
                fetch_chunk<UW>(fbase0, vb0, hi0, nx0);
                fetch_chunk<UW>(fbase1, vb1, hi1, nx1);
            }
            finish_chunk<UW>(fbase0, cb0, hi0, cur0, cw0);
            finish_chunk<UW>(fbase1, cb1, hi1, cur1, cw1);
        }
        static_for<U>([&](auto Sc) {
            constexpr int S = decltype(Sc)::value;
            constexpr int PH = S % NB;
            const int tau = c * U + S;
            if (tau == reset0 || tau == reset1) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (tau == (h ? reset1 : reset0)) {
#pragma unroll
                        for (int r = 0; r < NR; ++r) P[h][r] = (r == 0 && lane == 0) ? 0.0f : NEG;
                    }
                }
            }
            // branch metrics (Eq. BM) per frame
            float A[2][1 << BETA];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float l[BETA];
#pragma unroll
                for (int b = 0; b < BETA; ++b) {
                    const int j = S * BETA + b;
                    l[b] = half_at(h ? cw1[j >> 1] : cw0[j >> 1], j & 1);
                    if constexpr (L > 1) {
                        if ((cbits >> (PH * BETA + b)) & 1u) l[b] = -l[b];
                    }
                }
                A[h][0] = l[0];
                A[h][1] = -l[0];
#pragma unroll
                for (int b = 1; b < BETA; ++b) {
#pragma unroll
                    for (int x = 0; x < (1 << b); ++x) {
                        A[h][x | (1 << b)] = A[h][x] - l[b];
                        A[h][x] = A[h][x] + l[b];
                    }
                }
            }
            // add-compare-select (Eq. PM) and decisions (Eq. SP0)
            uint32_t X[2][NR];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if constexpr (PH < LR) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        if (r & (1 << PH)) continue;
                        const int ra = r, rb = r | (1 << PH);
                        const uint32_t a = C::alpha(C::rotr((uint32_t)ra, PH) >> 1);
                        const float Pa = P[h][ra], Pb = P[h][rb];
                        const float ca0 = Pa + A[h][a], cb0 = Pb + A[h][a ^ LV];
                        const float ca1 = Pa + A[h][a ^ MV], cb1 = Pb + A[h][a ^ MV ^ LV];
                        P[h][ra] = fmaxf(ca0, cb0);
                        P[h][rb] = fmaxf(ca1, cb1);
                        X[h][ra] = __float_as_uint(cb0 - ca0);   // sign clear: odd wins or ties
                        X[h][rb] = __float_as_uint(cb1 - ca1);
                    }
                } else {
                    constexpr int lb = PH >= LR ? PH - LR : 0;
                    const uint32_t xb = ((uint32_t)lane >> lb) & 1u;
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const uint32_t a = C::alpha(C::rotr((uint32_t)r, PH) >> 1);
                        const float own = P[h][r];
                        const float oth = __shfl_xor_sync(gmask, own, 1 << lb);
                        // even predecessor: holder of R_a is `own`, of R_b is `oth`
                        const float pe = xb ? oth : own, po = xb ? own : oth;
                        const float ce = pe + (xb ? A[h][a ^ MV] : A[h][a]);
                        const float co = po + (xb ? A[h][a ^ MV ^ LV] : A[h][a ^ LV]);
                        P[h][r] = fmaxf(ce, co);
                        X[h][r] = __float_as_uint(co - ce);
                    }
                }
            }
            // pack !sign into words: bit (r & 31) of word r >> 5, frame 0 first
            uint32_t wd[NW];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int m = 0; m < WPF; ++m) {
                    uint32_t acc = 0;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int r = 32 * m + k;
                        const uint32_t t1 = prmt(X[h][r], X[h][r + 8], 0x00FBu);
                        const uint32_t t2 = prmt(X[h][r + 16], X[h][r + 24], 0x00FBu);
                        const uint32_t t = prmt(t1, t2, 0x5410u);
                        acc |= t & (0x01010101u << k);
                    }
                    wd[h * WPF + m] = ~acc;
                }
            }
            if (tau >= tau_store) {
                uint32_t *dst = surv + ((size_t)tau * 32 + wlane) * NW;
                if constexpr (NW == 2) {
                    *reinterpret_cast<uint2 *>(dst) = make_uint2(wd[0], wd[1]);
                } else {
#pragma unroll
                    for (int i = 0; i < NW; i += 4)
                        *reinterpret_cast<uint4 *>(dst + i) = make_uint4(wd[i], wd[i + 1], wd[i + 2], wd[i + 3]);
                }
            }
        });
        // normalisation: subtract state 0's metric (register 0 of lane 0) per frame
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float ref = P[h][0];
            if constexpr (L > 1) ref = __shfl_sync(gmask, ref, grp_base);
#pragma unroll
            for (int r = 0; r < NR; ++r) P[h][r] -= ref;
        }
    }

    // traceback start: after Wpad stages register R holds state R again
    uint32_t R[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float best = -INFINITY;
        uint32_t bR = 0;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (P[h][r] > best) { best = P[h][r]; bR = ((uint32_t)lane << LR) | (uint32_t)r; }
        }
        if constexpr (L > 1) {
#pragma unroll
            for (int m = 1; m < L; m <<= 1) {
                const float ob = __shfl_xor_sync(gmask, best, m);
                const uint32_t oR = __shfl_xor_sync(gmask, bR, m);
                if (ob > best || (ob == best && oR < bR)) { best = ob; bR = oR; }
            }
        }
        R[h] = term[h] ? 0u : bR;
    }
    tb.set_out(0, ft[0].out);
    tb.set_out(1, ft[1].out);
    tb.set_surv(surv + (size_t)wlane * NW);
    tb.R[0] = R[0];
    tb.R[1] = R[1];
    tb.set_oacc(0, 0u);
    tb.set_oacc(1, 0u);
    tb.onb[0] = tb.onb[1] = 0;
    tb.t0 = Wpad - 1;
    tb.tau_store = tau_store;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        tb.tauo[h] = tauo[h];
        tb.taue[h] = taue[h];
        tb.toff[h] = (int32_t)(fa[h] - tau0[h]);
    }
    return true;
}

template <int K, int BETA, uint64_t GENS, int L, int NT>
__global__ void __launch_bounds__(NT) stream_kernel_f32(const StreamParams p) {
    using Cfg = StreamCfgF32<K, BETA, GENS, L>;
    using Tb = Traceback<K, L, false, Cfg::NR, Cfg::NW>;
    __shared__ TbState tbs[NT];
    __shared__ __align__(16) uint32_t stg[NT / 32][Tb::STAGE_WORDS];
    const int64_t gtid = (int64_t)blockIdx.x * NT + threadIdx.x;
    const int64_t q = gtid / L;
    const int lane = (int)(gtid % L);
    if (q >= p.n_pairs) return;
    const int wlane = (int)(threadIdx.x & 31u);
    const unsigned gmask = (L == 32) ? 0xFFFFFFFFu : (((1u << L) - 1u) << (wlane & ~(L - 1)));
    const int grp_base = wlane & ~(L - 1);
    FrameTask ft[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t s = 2 * q + h;
        ft[h] = frame_task(p.llr, p.out, nullptr, s, p.n_win, p.n_info, p.T, p.f, p.v, p.flags);
    }
    uint32_t *surv = p.surv + (size_t)(gtid >> 5) * (size_t)p.wpad_max * 32u *
                                  (size_t)StreamCfgF32<K, BETA, GENS, L>::NW;
    TbState tb;
    forward_pair_f32<K, BETA, GENS, L>(ft, surv, p.wpad_max, wlane, lane, gmask, grp_base, p.status, tb);
    TbState &st = tbs[threadIdx.x];
    st = tb;
    uint32_t *my_stg = stg[threadIdx.x >> 5];
    if (Tb::active(st)) {
        Tb::begin(st, my_stg, wlane);
        Tb::drain(st, my_stg, wlane, lane, gmask, grp_base);
    }
}

}  // namespace vd
