// vd_decode_radix: the general radix-2^rho forward procedure of Sec. VI
// (Eq. general:S), rho = 1, 2 or 3 stages per step, as a measured variant of
// the stream decoder.  One warp decodes one frame at a time; each lane owns
// 2^(K-1)/32 right states of a step.
//
// A step over stages t-rho+1 .. t treats the trellis as 2^(K-1-rho) groups
// of 2^rho left and 2^rho right states (radix-2 butterflies for rho = 1,
// dragonflies for rho = 2).  Eq. general:S gives the state at local stage x
// (0 = left, rho = right) of group f and local index y:
//
//     s(x, y) = (y >> (rho - x)) << (K - 1 - x)  +  f << (rho - x)  +  (y mod 2^(rho - x))
//
// (the pre-bubble is the top x bits of y, the post-bubble its low rho - x
// bits; the printed post-bubble y_{rho-x-1:0} drops one bit, see the
// readings).  The unique path from left y_l to right y_r passes through
// local index ((y_r mod 2^x) << (rho - x)) | (y_l >> x) at stage x, so each
// of the 2^rho candidates of a right state is its left metric plus the
// branch metrics (Eq. BM) of rho branches, and the step keeps the maximum
// (Eq. PM generalised as Eq. radix4:PM is) with the survivor y_l (the left
// state is f 2^rho + y_l).  Ties go to the larger y_l, which is the tie order
// of rho radix-2 steps with ties to the odd predecessor, so the bits equal
// vd_decode's.  A frame whose length is not a multiple of rho starts with
// radix-2 steps.  Metrics are int32, normalised by their minimum every step;
// survivors are bytes in a per-warp global buffer; lane 0 walks the
// traceback rho stages per step (Algorithm 2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "../../include/vd.h"
#include "vd_code.h"

namespace {

constexpr int kRxWarps = 4;          // warps per block
constexpr int kRxWarpsPerSm = 16;    // resident warps per SM the grid provides

struct RadixParams {
    const int8_t *llr;       // [T][beta] int8
    uint32_t *out;
    uint8_t *surv;           // per warp: max_steps x 2^(K-1) bytes
    int64_t n_info, T, f, v, n_win;
    int32_t max_steps;
    uint32_t flags;
    uint32_t gens[4];
    int beta;
};

template <int K>
__device__ __forceinline__ int branch_metric(const RadixParams &p, uint32_t state, uint32_t u, const int *l) {
    const uint32_t r = (u << (K - 1)) | state;
    int d = 0;
    for (int b = 0; b < p.beta; ++b) d += (__popc(p.gens[b] & r) & 1) ? -l[b] : l[b];
    return d;
}

// Eq. general:S (with the post-bubble read as the low rho - x bits of y).
template <int K, int RHO>
__device__ __forceinline__ uint32_t general_state(uint32_t f, int x, uint32_t y) {
    const uint32_t pre = (y >> (RHO - x)) << (K - 1 - x);
    const uint32_t bubble = f << (RHO - x);
    const uint32_t post = y & ((1u << (RHO - x)) - 1u);
    return pre + bubble + post;
}

// One radix-2^R step over stages t0 .. t0 + R - 1: new metrics into dst and
// survivors into sv (one byte per right state).
template <int K, int R>
__device__ __forceinline__ void step(const RadixParams &p, int lane, const int *src, int *dst, uint8_t *sv,
                                     const int8_t *L) {
    constexpr int NS = 1 << (K - 1);
    constexpr int PER = NS / 32;
    int l[R][4];
#pragma unroll
    for (int x = 0; x < R; ++x)
        for (int b = 0; b < p.beta; ++b) l[x][b] = L[x * p.beta + b];
    int mn = 0x7FFFFFFF;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const uint32_t j = (uint32_t)lane + 32u * k;
        const uint32_t f = j & ((1u << (K - 1 - R)) - 1u), yr = j >> (K - 1 - R);
        int best = 0;
        uint32_t arg = 0;
#pragma unroll
        for (uint32_t yl = 0; yl < (1u << R); ++yl) {
            uint32_t s = general_state<K, R>(f, 0, yl);   // left state f 2^R + yl
            int c = src[s];
#pragma unroll
            for (int x = 1; x <= R; ++x) {
                const uint32_t yx = ((yr & ((1u << x) - 1u)) << (R - x)) | (yl >> x);
                const uint32_t nx = general_state<K, R>(f, x, yx);
                const uint32_t u = nx >> (K - 2);           // the input that leads s -> nx
                c += branch_metric<K>(p, s, u, l[x - 1]);
                s = nx;
            }
            if (yl == 0 || c >= best) { best = c; arg = yl; }   // ties to the larger left index
        }
        dst[j] = best;
        sv[j] = (uint8_t)arg;
        mn = min(mn, best);
    }
#pragma unroll
    for (int m = 1; m < 32; m <<= 1) mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, m));
    __syncwarp();
#pragma unroll
    for (int k = 0; k < PER; ++k) dst[lane + 32 * k] -= mn;
    __syncwarp();
}

template <int K, int RHO>
__global__ void __launch_bounds__(kRxWarps * 32) radix_kernel(const RadixParams p) {
    constexpr int NS = 1 << (K - 1);
    constexpr uint32_t MASK = NS - 1;
    __shared__ int lam[kRxWarps][2][NS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * kRxWarps + warp, n_warps = (int64_t)gridDim.x * kRxWarps;
    uint8_t *sv = p.surv + (size_t)gw * (size_t)p.max_steps * NS;
    for (int64_t s = gw; s < p.n_win; s += n_warps) {
        const int64_t o = s * p.f, e = min(p.n_info, (s + 1) * p.f);
        const int64_t a = max((int64_t)0, o - p.v), b = min(p.T, (s + 1) * p.f + p.v);
        const int W = (int)(b - a);
        const int rem = W % RHO, nsteps = W / RHO;
        if (rem + nsteps > p.max_steps) return;   // the host sizes max_steps for the longest frame
        const bool known = a == 0 && !(p.flags & VD_START_UNKNOWN);
        const bool term = b == p.T && (p.flags & VD_TERMINATED);
        for (int k = 0; k < NS / 32; ++k) {
            const int j = lane + 32 * k;
            lam[warp][0][j] = (known && j != 0) ? -(1 << 28) : 0;   // head start of the reset state
        }
        __syncwarp();
        int cur = 0;
        const int8_t *L = p.llr + a * p.beta;
        // stages that do not fill a whole step go first, as radix-2 steps
        for (int r = 0; r < rem; ++r) {
            step<K, 1>(p, lane, lam[warp][cur], lam[warp][cur ^ 1], sv + (size_t)r * NS, L);
            cur ^= 1;
            L += p.beta;
        }
        for (int q = 0; q < nsteps; ++q) {
            step<K, RHO>(p, lane, lam[warp][cur], lam[warp][cur ^ 1], sv + (size_t)(rem + q) * NS, L);
            cur ^= 1;
            L += RHO * p.beta;
        }
        // traceback start: state 0 at a terminated end, else the best state (lowest index on ties)
        int bv = lam[warp][cur][lane], bj = lane;
        for (int k = 1; k < NS / 32; ++k) {
            const int j = lane + 32 * k;
            if (lam[warp][cur][j] > bv) { bv = lam[warp][cur][j]; bj = j; }
        }
#pragma unroll
        for (int m = 1; m < 32; m <<= 1) {
            const int ov = __shfl_xor_sync(0xFFFFFFFFu, bv, m), oj = __shfl_xor_sync(0xFFFFFFFFu, bj, m);
            if (ov > bv || (ov == bv && oj < bj)) { bv = ov; bj = oj; }
        }
        __threadfence_block();
        if (lane == 0) {
            uint32_t j = term ? 0u : (uint32_t)bj;
            int64_t t = b - 1, wcur = -1;
            uint32_t word = 0;
            auto emit = [&](int64_t st, uint32_t bit) {
                if (st < o || st >= e) return;
                const int64_t w = st >> 5;
                if (w != wcur) {
                    if (wcur >= 0) p.out[wcur] = word;
                    wcur = w;
                    word = 0;
                }
                word |= bit << (st & 31);
            };
            for (int q = nsteps - 1; q >= 0; --q) {
                const uint32_t d = sv[(size_t)(rem + q) * NS + j];
#pragma unroll
                for (int k = 0; k < RHO; ++k) emit(t - k, (j >> (K - 2 - k)) & 1u);
                j = ((j << RHO) & MASK) | d;
                t -= RHO;
            }
            for (int r = rem - 1; r >= 0; --r) {
                const uint32_t d = sv[(size_t)r * NS + j];
                emit(t, j >> (K - 2));
                j = ((j << 1) & MASK) | d;
                t -= 1;
            }
            if (wcur >= 0) p.out[wcur] = word;
        }
        __syncwarp();
    }
}

template <int K, int RHO>
cudaError_t launch(const RadixParams &p, int blocks, cudaStream_t st) {
    radix_kernel<K, RHO><<<blocks, kRxWarps * 32, 0, st>>>(p);
    return cudaGetLastError();
}

vd_status fail(vd_status st, const char *msg) {
    vd_internal_set_error(msg);
    return st;
}

}  // namespace

extern "C" vd_status vd_decode_radix(const vd_code *c, const void *d_llr, int64_t n_info, int f, int v, int rho,
                                     uint32_t flags, uint32_t *d_out, void *stream) {
    if (!c) return fail(VD_EINVAL, "vd_decode_radix: code is NULL");
    if (n_info < 0 || f <= 0 || v < 0) return fail(VD_EINVAL, "vd_decode_radix: bad n_info, f or v");
    if (rho < 1 || rho > 3) return fail(VD_EINVAL, "vd_decode_radix: rho must be 1, 2 or 3");
    if (flags & ~(uint32_t)(VD_TERMINATED | VD_START_UNKNOWN)) return fail(VD_EINVAL, "vd_decode_radix: unknown flags");
    if (n_info == 0) return VD_OK;
    if (!d_llr || !d_out) return fail(VD_EINVAL, "vd_decode_radix: NULL device pointer");
    if (f < n_info && f % 32) return fail(VD_EINVAL, "vd_decode_radix: f must be a multiple of 32 (or >= n_info)");
    if ((c->K != 7 && c->K != 9) || c->punctured)
        return fail(VD_EUNSUPPORTED, "vd_decode_radix: unpunctured int8 LLRs of K=7 or K=9 codes");
    RadixParams p;
    memset(&p, 0, sizeof p);
    p.llr = (const int8_t *)d_llr;
    p.out = d_out;
    p.n_info = n_info;
    p.T = n_info + ((flags & VD_TERMINATED) ? c->K - 1 : 0);
    p.f = f;
    p.v = v;
    p.n_win = (n_info + f - 1) / f;
    p.flags = flags;
    p.beta = c->beta;
    for (int b = 0; b < c->beta; ++b) p.gens[b] = c->gens[b];
    const int64_t wmax = std::min<int64_t>(p.T, (int64_t)f + 2 * (int64_t)v);
    if (wmax > (1 << 16)) return fail(VD_EUNSUPPORTED, "vd_decode_radix: frames longer than 65536 stages");
    p.max_steps = (int32_t)(wmax / rho + rho);
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t warps = std::min<int64_t>(p.n_win, (int64_t)n_sm * kRxWarpsPerSm);
    const int blocks = (int)((warps + kRxWarps - 1) / kRxWarps);
    const size_t ns = (size_t)1 << (c->K - 1);
    void *surv = nullptr;
    const vd_status st = vd_internal_scratch(6, (size_t)blocks * kRxWarps * (size_t)p.max_steps * ns, (cudaStream_t)stream,
                                             &surv);
    if (st != VD_OK) return st;
    p.surv = (uint8_t *)surv;
    cudaError_t e;
    if (c->K == 7) e = rho == 1 ? launch<7, 1>(p, blocks, (cudaStream_t)stream)
                     : rho == 2 ? launch<7, 2>(p, blocks, (cudaStream_t)stream)
                                : launch<7, 3>(p, blocks, (cudaStream_t)stream);
    else e = rho == 1 ? launch<9, 1>(p, blocks, (cudaStream_t)stream)
           : rho == 2 ? launch<9, 2>(p, blocks, (cudaStream_t)stream)
                      : launch<9, 3>(p, blocks, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(VD_ECUDA, cudaGetErrorString(e));
    return VD_OK;
}
