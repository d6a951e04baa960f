// Input pre-pass helper: expands transmitted (kept) LLR values to beta int8
// LLRs per stage, inserting 0 at the positions a puncturing pattern erases,
// sign-extending 4-bit values and mapping hard decisions to +-1.  The kept values are stage-major with b
// ascending, so the values of puncturing period g (stages g*period ..) start
// at g * kept_per_period.
//
// A thread produces m whole periods at a time, m chosen so that their
// m * period * beta output bytes are a whole number of 32-bit words: the
// stores of a warp then cover full, contiguous sectors.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/vd.h"

namespace vd {

// One value of the kept stream (int8; 4-bit two per byte, low nibble
// first; or a hard decision, eight per byte, bit 0 first, mapped to +1 for
// bit 0 and -1 for bit 1); 0 at or past n_kept (the end of this packet's
// values), which is never read.
__device__ __forceinline__ int8_t prep_kept_value(const uint8_t *src, int64_t k, int64_t n_kept, int llr_type) {
    if (k >= n_kept) return 0;
    if (llr_type == VD_LLR_HARD) return ((src[k >> 3] >> (k & 7)) & 1u) ? (int8_t)-1 : (int8_t)1;
    if (llr_type == VD_LLR_S4) {
        const uint8_t byte = src[k >> 1];
        const uint8_t nib = (k & 1) ? (byte >> 4) : (byte & 0x0F);
        return (int8_t)((int8_t)(nib << 4) >> 4);
    }
    return (int8_t)src[k];
}

// The same for a compile-time (period, beta): the loops unroll, so a step's
// loads are independent and issue together.
template <int P, int B>
__device__ __forceinline__ void prep_expand_fixed(const uint8_t *src, int64_t k0, int64_t n_kept, int llr_type,
                                                  int64_t T, int kept_per_period, const uint8_t (&punct)[4][8],
                                                  int8_t *dst, int64_t tid, int64_t nthr) {
    constexpr int GB = P * B;
    constexpr int M = (GB % 4 == 0) ? 1 : (GB % 2 == 0) ? 2 : 4;
    constexpr int SPAN = M * GB;
    static_assert(SPAN <= 16, "step too wide");
    bool keep[B][P];
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
        for (int ph = 0; ph < P; ++ph) keep[b][ph] = punct[b][ph] != 0;
    const int64_t n_groups = (T + P - 1) / P;
    const int64_t n_steps = (n_groups + M - 1) / M;
    const int64_t full_steps = (T * B) / SPAN;   // steps wholly inside the output
    for (int64_t st = tid; st < n_steps; st += nthr) {
        int64_t k = k0 + st * M * kept_per_period;
        uint8_t v[SPAN];
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int ph = 0; ph < P; ++ph)
#pragma unroll
                for (int b = 0; b < B; ++b)
                    v[(i * P + ph) * B + b] = keep[b][ph] ? (uint8_t)prep_kept_value(src, k++, n_kept, llr_type) : 0;
        if (st < full_steps) {
            uint32_t *d = reinterpret_cast<uint32_t *>(dst + st * SPAN);
#pragma unroll
            for (int w = 0; w < SPAN / 4; ++w)
                d[w] = (uint32_t)v[4 * w] | ((uint32_t)v[4 * w + 1] << 8) | ((uint32_t)v[4 * w + 2] << 16) |
                       ((uint32_t)v[4 * w + 3] << 24);
        } else {
#pragma unroll
            for (int j = 0; j < SPAN; ++j)
                if (st * SPAN + j < T * B) dst[st * SPAN + j] = (int8_t)v[j];
        }
    }
}

// Expands stages [0, T) into dst ([T][beta] int8, 4-byte aligned) from the
// kept values src[k0 .. n_kept).  Threads tid, tid + nthr, .. of the caller
// share the work.
__device__ __forceinline__ void prep_expand(const uint8_t *src, int64_t k0, int64_t n_kept, int llr_type,
                                            int64_t T, int beta, int period, int kept_per_period,
                                            const uint8_t (&punct)[4][8], int8_t *dst, int64_t tid,
                                            int64_t nthr) {
    // the shapes of the supported codes, unrolled
    if (period == 2 && beta == 2)
        return prep_expand_fixed<2, 2>(src, k0, n_kept, llr_type, T, kept_per_period, punct, dst, tid, nthr);
    if (period == 3 && beta == 2)
        return prep_expand_fixed<3, 2>(src, k0, n_kept, llr_type, T, kept_per_period, punct, dst, tid, nthr);
    if (period == 1 && beta == 2)
        return prep_expand_fixed<1, 2>(src, k0, n_kept, llr_type, T, kept_per_period, punct, dst, tid, nthr);
    if (period == 1 && beta == 3)
        return prep_expand_fixed<1, 3>(src, k0, n_kept, llr_type, T, kept_per_period, punct, dst, tid, nthr);
    const int gb = period * beta;                               // output bytes per period
    const int m = (gb % 4 == 0) ? 1 : (gb % 2 == 0) ? 2 : 4;   // periods per thread step
    const int span = m * gb;                                    // bytes per thread step
    const int64_t out_bytes = T * beta;
    const int64_t n_groups = (T + period - 1) / period;
    const int64_t n_steps = (n_groups + m - 1) / m;
    for (int64_t st = tid; st < n_steps; st += nthr) {
        const int64_t byte0 = st * span;
        const int64_t g0 = st * m;
        if (span <= 16 && byte0 + span <= out_bytes) {
            // whole step inside the output: assemble up to 16 bytes in two
            // 64-bit registers, store them as 32-bit words
            uint64_t lo = 0, hi = 0;
            int pos = 0;
            for (int i = 0; i < m; ++i) {
                int64_t k = k0 + (g0 + i) * kept_per_period;
                for (int ph = 0; ph < period; ++ph) {
                    for (int b = 0; b < beta; ++b, ++pos) {
                        const int8_t x = punct[b][ph] ? prep_kept_value(src, k++, n_kept, llr_type) : (int8_t)0;
                        const uint64_t v = (uint64_t)(uint8_t)x;
                        if (pos < 8) lo |= v << (8 * pos);
                        else hi |= v << (8 * (pos - 8));
                    }
                }
            }
            uint32_t *d = reinterpret_cast<uint32_t *>(dst + byte0);
            d[0] = (uint32_t)lo;
            if (span > 4) d[1] = (uint32_t)(lo >> 32);
            if (span > 8) d[2] = (uint32_t)hi;
            if (span > 12) d[3] = (uint32_t)(hi >> 32);
        } else {
            // the last, partial step (or an unusually long period): byte stores
            for (int i = 0; i < m; ++i) {
                const int64_t g = g0 + i;
                int64_t k = k0 + g * kept_per_period;
                for (int ph = 0; ph < period; ++ph) {
                    const int64_t t = g * period + ph;
                    for (int b = 0; b < beta; ++b) {
                        const int8_t x = punct[b][ph] ? prep_kept_value(src, k++, n_kept, llr_type) : (int8_t)0;
                        if (t < T) dst[t * beta + b] = x;
                    }
                }
            }
        }
    }
}

}  // namespace vd
