// vd_decode_tc: the paper's tensor-core formulation of the radix-4 forward
// procedure (Sec. VIII, "Employing Tensor Cores For Radix-4"), as a measured
// variant of the CUDA-core decoder: for every stage pair (t-1, t) the 16
// candidates of each dragonfly are one column of
//
//     D = Theta_hat * L + Lambda                                   (Sec. VIII-B/C)
//
// where Theta_hat holds the +-1 outputs of the dragonfly's 16 super-branches
// over the 2 beta LLRs of the pair (Eq. radix4:BM), L those LLRs and Lambda
// the path metrics of the left states feeding each super-branch (Eq.
// radix4:PM).  Dragonflies whose Theta_hat are equal up to a permutation of
// their left states form a dragonfly group (Sec. VIII-D-2), so the A operand
// holds one Theta_hat per group side by side, B places the LLRs in the rows
// of the dragonfly's group, and C is filled through the group's left-state
// permutation: one mma.sync.m16n8k16 (f16 x f16 -> f32) covers 8 dragonflies,
// two cover the whole 64-state trellis of the (2,1,7) code.  Integer LLRs
// (|l| <= 127) and the f32 metrics are exact, so the decoded bits equal the
// CUDA-core decoder's.
//
// Per stage pair, a warp (one frame) then takes the maximum over the four
// rows of each right state (two shuffle rounds on keys 4 lambda + y, y the
// left index, so equal metrics go to the larger left index: the tie order
// of two radix-2 steps with ties to the odd predecessor), normalises by the
// minimum, and keeps the 2-bit survivor y of every state (Eq. radix4:SP0) in
// shared memory; one lane walks the traceback (Algorithm 2, two stages per
// step).  An odd number of stages starts with one radix-2 stage on the CUDA
// cores.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/vd.h"
#include "vd_code.h"

namespace {

constexpr int kTcK = 7;                 // the variant is built for K = 7, beta = 2 codes
constexpr int kTcNS = 64;               // states
constexpr int kTcDF = 16;               // dragonflies per stage pair
constexpr int kTcWarps = 4;             // frames (warps) per block
constexpr int kTcMaxW = 1024;           // longest frame (stages) the variant takes
constexpr float kTcHead = 1048576.0f;   // head start of state 0 at a known start: more than any
                                        // metric spread a frame of kTcMaxW stages can build

struct TcTables {
    uint8_t group[kTcDF];    // dragonfly -> group
    uint8_t perm[kTcDF][4];  // dragonfly, representative left index y -> the dragonfly's left index
    uint32_t a_frag[32][4];  // A fragment registers (f16x2) of each lane
};

struct TcParams {
    const int8_t *llr;       // [T][2] int8
    uint32_t *out;
    int64_t n_info, T, f, v, n_win;
    uint32_t flags;
    int32_t max_pairs;       // survivor rows per warp (longest frame / 2 + 1)
    int32_t per_warp;        // shared-memory bytes per warp
    int *status;
    TcTables tab;
};

__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1,
                                          const float (&c)[4]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%12,%13};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]), "f"(c[2]),
          "f"(c[3]));
}

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Branch output bits of the K=7 code (generators in c) for register r.
__device__ __forceinline__ int out_bit(uint32_t gen, uint32_t r) { return __popc(gen & r) & 1; }

__global__ void __launch_bounds__(kTcWarps * 32) tc_kernel(const TcParams p, uint32_t g0, uint32_t g1) {
    extern __shared__ __align__(16) unsigned char tc_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t s = (int64_t)blockIdx.x * kTcWarps + warp;   // frame
    if (s >= p.n_win) return;
    float *lam = reinterpret_cast<float *>(tc_smem + (size_t)p.per_warp * warp);       // [2][64] path metrics
    uint8_t *sv = tc_smem + (size_t)p.per_warp * warp + 2 * kTcNS * sizeof(float);    // [pairs + 1][64] survivors

    // frame geometry (Sec. III; v stages on each side, clipped)
    const int64_t o = s * p.f, e = min(p.n_info, (s + 1) * p.f);
    const int64_t a = max((int64_t)0, o - p.v), b = min(p.T, (s + 1) * p.f + p.v);
    const int W = (int)(b - a);
    if ((W >> 1) + 1 > p.max_pairs) {   // the host sizes max_pairs for the longest frame: never taken
        if (lane == 0) atomicOr(p.status, 1);
        return;
    }
    const bool known = a == 0 && !(p.flags & VD_START_UNKNOWN);
    const bool term = b == p.T && (p.flags & VD_TERMINATED);
    const int odd = W & 1;
    const int npairs = W >> 1;

    // lane constants: fragment rows g, g + 8 and columns 2q, 2q + 1 (C/D); B column g
    const int g = lane >> 2, q = lane & 3;
    uint32_t afr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) afr[i] = p.tab.a_frag[lane][i];
    int cst[2][2];          // left state whose metric fills C at (row g or g + 8, column 2q + c) of MMA h
    float yl[2][2];         // that left state's index y_l within its dragonfly (the survivor)
    bool bsel[2][2];        // B register k of MMA h carries the LLRs (the dragonfly g of MMA h is in that group)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int n = 8 * h + 2 * q + c;
            const int y = p.tab.perm[n][g & 3];
            cst[h][c] = 4 * n + y;
            yl[h][c] = (float)y;
        }
        const int nb = 8 * h + g;   // B column of this lane
        bsel[h][0] = p.tab.group[nb] == (q >> 1);
        bsel[h][1] = p.tab.group[nb] == 2 + (q >> 1);
    }

    // initial path metrics (Algorithm 1; a known start gives state 0 a head start)
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int j = 2 * lane + i;
        lam[j] = (known && j != 0) ? -kTcHead : 0.0f;
    }
    __syncwarp();
    int cur = 0;
    const int8_t *L = p.llr + a * 2;

    if (odd) {
        // one radix-2 stage (Eq. PM / Eq. SP0, ties to the odd predecessor)
        const float l0 = (float)L[0], l1 = (float)L[1];
        float *dst = lam + kTcNS;
        float mn = 3.0e38f;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int j = 2 * lane + i;
            const uint32_t u = (uint32_t)j >> 5, p0 = ((uint32_t)j << 1) & 63u, p1 = p0 | 1u;
            const uint32_t r0 = (u << 6) | p0, r1 = (u << 6) | p1;
            const float d0 = (out_bit(g0, r0) ? -l0 : l0) + (out_bit(g1, r0) ? -l1 : l1);
            const float d1 = (out_bit(g0, r1) ? -l0 : l0) + (out_bit(g1, r1) ? -l1 : l1);
            const float c0 = lam[p0] + d0, c1 = lam[p1] + d1;
            const bool odd_wins = c1 >= c0;
            dst[j] = odd_wins ? c1 : c0;
            sv[kTcNS * npairs + j] = odd_wins ? 1 : 0;   // the radix-2 stage's survivors
            mn = fminf(mn, dst[j]);
        }
#pragma unroll
        for (int m = 1; m < 32; m <<= 1) mn = fminf(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, m));
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 2; ++i) dst[2 * lane + i] -= mn;
        cur = 1;
        L += 2;
        __syncwarp();
    }

    for (int pr = 0; pr < npairs; ++pr) {
        const float *src = lam + cur * kTcNS;
        float *dst = lam + (cur ^ 1) * kTcNS;
        // the pair's LLRs: lanes with q even take stage t-1, odd ones stage t (rows 2(q&1), +1 of a group's block)
        const int sb = (q & 1) * 2;
        const uint32_t lpair = pack_h2((float)L[sb], (float)L[sb + 1]);
        float mn = 3.0e38f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float c0 = src[cst[h][0]], c1 = src[cst[h][1]];
            const float cin[4] = {c0, c1, c0, c1};   // rows g and g + 8 share the left state
            float dd[4];
            mma_16816(dd, afr, bsel[h][0] ? lpair : 0u, bsel[h][1] ? lpair : 0u, cin);
            // keys 4 D + y_l: the maximum over the four left states of a right state's block
            // (lanes l, l^4, l^8, l^12) is the new metric, ties to the larger y_l
            float key[4] = {fmaf(dd[0], 4.0f, yl[h][0]), fmaf(dd[1], 4.0f, yl[h][1]),
                            fmaf(dd[2], 4.0f, yl[h][0]), fmaf(dd[3], 4.0f, yl[h][1])};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                key[i] = fmaxf(key[i], __shfl_xor_sync(0xFFFFFFFFu, key[i], 4));
                key[i] = fmaxf(key[i], __shfl_xor_sync(0xFFFFFFFFu, key[i], 8));
            }
            // right state of (row block jp, dragonfly n): n + 16 jp (Eq. radix4:S)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int jp = (i < 2 ? 0 : 2) + (g >> 2);
                const int n = 8 * h + 2 * q + (i & 1);
                const float lamv = floorf(key[i] * 0.25f);
                const int y = (int)(key[i] - 4.0f * lamv);
                mn = fminf(mn, lamv);
                if ((g & 3) == 0) {
                    const int j = n + 16 * jp;
                    dst[j] = lamv;
                    sv[kTcNS * pr + j] = (uint8_t)y;
                }
            }
        }
#pragma unroll
        for (int m = 1; m < 32; m <<= 1) mn = fminf(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, m));
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 2; ++i) dst[2 * lane + i] -= mn;
        cur ^= 1;
        L += 4;
        __syncwarp();
    }

    // traceback start (Algorithm 2): state 0 at a terminated end, else the best state (lowest index on ties)
    const float *fin = lam + cur * kTcNS;
    int js = 0;
    if (!term) {
        float bv = fin[2 * lane];
        int bj = 2 * lane;
        if (fin[2 * lane + 1] > bv) { bv = fin[2 * lane + 1]; bj = 2 * lane + 1; }
#pragma unroll
        for (int m = 1; m < 32; m <<= 1) {
            const float ov = __shfl_xor_sync(0xFFFFFFFFu, bv, m);
            const int oj = __shfl_xor_sync(0xFFFFFFFFu, bj, m);
            if (ov > bv || (ov == bv && oj < bj)) { bv = ov; bj = oj; }
        }
        js = bj;
    }
    if (lane != 0) return;
    // walk back, two stages per step (Algorithm 2); the decoded bit of stage t
    // is the input bit of the state after it.  Stages arrive in decreasing
    // order; each output word is stored once it is complete.
    int64_t t = b - 1;
    uint32_t j = (uint32_t)js;
    int64_t wcur = -1;
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
    for (int pr = npairs - 1; pr >= 0; --pr) {
        const uint32_t y = sv[kTcNS * pr + j];
        emit(t, j >> 5);
        emit(t - 1, (j >> 4) & 1u);
        j = ((j << 2) & 63u) | y;
        t -= 2;
    }
    if (odd) {
        emit(t, j >> 5);
        j = ((j << 1) & 63u) | sv[kTcNS * npairs + j];
    }
    if (wcur >= 0) p.out[wcur] = word;
}

vd_status fail(vd_status st, const char *msg) {
    vd_internal_set_error(msg);
    return st;
}

int parity(uint32_t x) { return __builtin_popcount(x) & 1; }

// Host tables: the super-branch outputs of every dragonfly (Eq. radix4:S,
// Eq. radix4:BM), the dragonfly groups and left-state permutations (Sec.
// VIII-D-2) and the A fragments of each lane.  Returns false if the code
// needs more than four groups (A holds four Theta_hat side by side).
bool build_tables(const vd_code *c, TcTables *tab) {
    const uint32_t mask = kTcNS - 1;
    auto next = [&](uint32_t st, uint32_t u) { return (u << (kTcK - 2)) | (st >> 1); };
    auto outp = [&](uint32_t st, uint32_t u) {   // beta = 2 output bits of the branch (st, u)
        const uint32_t r = (u << (kTcK - 1)) | st;
        return (uint32_t)parity(c->gens[0] & r) | ((uint32_t)parity(c->gens[1] & r) << 1);
    };
    // pattern[n][jp][y]: 4 bits (stage t-1: b0, b1; stage t: b0, b1) of left 4n+y -> right n+16jp
    uint8_t pat[kTcDF][4][4];
    for (int n = 0; n < kTcDF; ++n)
        for (int jp = 0; jp < 4; ++jp)
            for (int y = 0; y < 4; ++y) {
                const uint32_t i = 4u * n + y, j = (uint32_t)n + 16u * jp;
                int found = 0;
                for (uint32_t u1 = 0; u1 < 2; ++u1)
                    for (uint32_t u2 = 0; u2 < 2; ++u2) {
                        const uint32_t m = next(i, u1);
                        if ((next(m, u2) & mask) == j) {
                            pat[n][jp][y] = (uint8_t)(outp(i, u1) | (outp(m, u2) << 2));
                            ++found;
                        }
                    }
                if (found != 1) return false;   // not a dragonfly of this trellis
            }
    int rep[4], n_groups = 0;
    for (int n = 0; n < kTcDF; ++n) {
        int gsel = -1;
        for (int gi = 0; gi < n_groups && gsel < 0; ++gi) {
            // a left permutation pi with pat[n][jp][pi[y]] == pat[rep][jp][y] for every jp, y
            int pi[4] = {0, 1, 2, 3};
            do {
                bool ok = true;
                for (int jp = 0; jp < 4 && ok; ++jp)
                    for (int y = 0; y < 4 && ok; ++y) ok = pat[n][jp][pi[y]] == pat[rep[gi]][jp][y];
                if (ok) {
                    gsel = gi;
                    for (int y = 0; y < 4; ++y) tab->perm[n][y] = (uint8_t)pi[y];
                    break;
                }
            } while (std::next_permutation(pi, pi + 4));
        }
        if (gsel < 0) {
            if (n_groups == 4) return false;
            gsel = n_groups;
            rep[n_groups++] = n;
            for (int y = 0; y < 4; ++y) tab->perm[n][y] = (uint8_t)y;
        }
        tab->group[n] = (uint8_t)gsel;
    }
    // A[row][k]: row 4 jp + y, k = 4 group + b: (-1)^(bit b of the representative's pattern)
    auto A = [&](int row, int k) -> float {
        const int gi = k >> 2, b = k & 3;
        if (gi >= n_groups) return 0.0f;
        return ((pat[rep[gi]][row >> 2][row & 3] >> b) & 1) ? -1.0f : 1.0f;
    };
    auto h2 = [](float lo, float hi) {
        const __half2 h = __floats2half2_rn(lo, hi);
        uint32_t u;
        memcpy(&u, &h, 4);
        return u;
    };
    for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, q = lane & 3;
        tab->a_frag[lane][0] = h2(A(g, 2 * q), A(g, 2 * q + 1));
        tab->a_frag[lane][1] = h2(A(g + 8, 2 * q), A(g + 8, 2 * q + 1));
        tab->a_frag[lane][2] = h2(A(g, 2 * q + 8), A(g, 2 * q + 9));
        tab->a_frag[lane][3] = h2(A(g + 8, 2 * q + 8), A(g + 8, 2 * q + 9));
    }
    return true;
}

}  // namespace

extern "C" vd_status vd_decode_tc(const vd_code *c, const void *d_llr, int64_t n_info, int f, int v,
                                  uint32_t flags, uint32_t *d_out, void *stream) {
    if (!c) return fail(VD_EINVAL, "vd_decode_tc: code is NULL");
    if (n_info < 0 || f <= 0 || v < 0) return fail(VD_EINVAL, "vd_decode_tc: bad n_info, f or v");
    if (flags & ~(uint32_t)(VD_TERMINATED | VD_START_UNKNOWN)) return fail(VD_EINVAL, "vd_decode_tc: unknown flags");
    if (n_info == 0) return VD_OK;
    if (!d_llr || !d_out) return fail(VD_EINVAL, "vd_decode_tc: NULL device pointer");
    if (f < n_info && f % 32) return fail(VD_EINVAL, "vd_decode_tc: f must be a multiple of 32 (or >= n_info)");
    if (c->K != kTcK || c->beta != 2 || c->punctured)
        return fail(VD_EUNSUPPORTED, "vd_decode_tc: K=7, beta=2, unpunctured int8 codes only");
    TcParams p;
    memset(&p, 0, sizeof p);
    if (!build_tables(c, &p.tab))
        return fail(VD_EUNSUPPORTED, "vd_decode_tc: the code's dragonflies need more than four groups");
    p.llr = (const int8_t *)d_llr;
    p.out = d_out;
    p.n_info = n_info;
    p.T = n_info + ((flags & VD_TERMINATED) ? kTcK - 1 : 0);
    p.f = f;
    p.v = v;
    p.n_win = (n_info + f - 1) / f;
    p.flags = flags;
    const int64_t wmax = std::min<int64_t>(p.T, (int64_t)f + 2 * (int64_t)v);
    if (wmax > kTcMaxW) return fail(VD_EUNSUPPORTED, "vd_decode_tc: frames longer than 1024 stages");
    p.max_pairs = (int32_t)(wmax / 2 + 1);
    p.per_warp = (int32_t)(2 * kTcNS * sizeof(float) + (size_t)p.max_pairs * kTcNS);
    p.per_warp = (p.per_warp + 15) & ~15;
    p.status = vd_internal_status_word();
    if (!p.status) return fail(VD_ENOMEM, "vd_decode_tc: no device status word");
    const size_t smem = (size_t)p.per_warp * kTcWarps;
    if (smem > 48u * 1024u &&
        cudaFuncSetAttribute(tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return fail(VD_ECUDA, "vd_decode_tc: shared memory opt-in failed");
    const int64_t blocks = (p.n_win + kTcWarps - 1) / kTcWarps;
    if (blocks > 0x7FFFFFFF) return fail(VD_EINVAL, "vd_decode_tc: stream too long");
    tc_kernel<<<(unsigned)blocks, kTcWarps * 32, smem, (cudaStream_t)stream>>>(p, c->gens[0], c->gens[1]);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(VD_ECUDA, cudaGetErrorString(e));
    return VD_OK;
}
