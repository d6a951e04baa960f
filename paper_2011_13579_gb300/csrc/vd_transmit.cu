// vd_transmit: the transmitter and channel of the paper's verification
// system (Sec. IX-B) on the GPU, so that a decoder (or the serving loop) can
// be fed without host-generated LLRs: information bits -> convolutional
// encoder (Sec. II-A) -> puncturing -> BPSK -> AWGN -> quantiser.
//
// One thread makes eight consecutive kept values (two Philox blocks).  For
// kept value k the stage t and output b come from the puncturing pattern
// (k-th kept position in stage-major, b-ascending order); the encoder output
// is the parity of g_b and the register of inputs t-K+1 .. t, read straight
// from the packed information bits (zero before the start and in the tail).
// The noise is the k-th standard normal of the stream: Philox4x64-10 (Salmon
// et al., SC 2011) with key (seed, stream_id) on counter block k / 4, turned
// into four normals by the Box-Muller transform in double precision.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "../../include/vd.h"
#include "vd_code.h"

namespace {

struct TxParams {
    const uint32_t *bits;   // packed information bits, LSB-first
    int64_t n_info, n_kept, n_words;
    int K, beta, period, kept_per_period;
    uint32_t gens[4];
    uint8_t pos_phase[32], pos_b[32];   // r-th kept position of a period: (phase, output)
    double sigma, inv_var2;             // sigma and 2 / sigma^2
    uint64_t seed, stream_id;
    int llr_type;
    void *out;
};

__device__ __forceinline__ void philox4x64(uint64_t (&c)[4], uint64_t k0, uint64_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t lo0 = 0xD2E7470EE14C6C93ull * c[0], hi0 = __umul64hi(0xD2E7470EE14C6C93ull, c[0]);
        const uint64_t lo1 = 0xCA5A826395121157ull * c[2], hi1 = __umul64hi(0xCA5A826395121157ull, c[2]);
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
}

__device__ __forceinline__ double unit53(uint64_t x) { return (double)((x >> 11) + 1ull) * 0x1.0p-53; }

// Bits [lo, lo + 16) of the information stream (zero outside [0, n_info)).
__device__ __forceinline__ uint32_t info_window(const TxParams &p, int64_t lo) {
    uint32_t v = 0;
#pragma unroll
    for (int w = 0; w < 2; ++w) {
        const int64_t base = (lo >> 5) + w;          // word holding bits base*32 ..
        uint32_t x = (base >= 0 && base < p.n_words) ? p.bits[base] : 0u;
        const int64_t first = base * 32;
        if (first + 32 > p.n_info) {                 // clear bits at or past n_info
            const int64_t keep = p.n_info - first;
            x = keep <= 0 ? 0u : (x & (0xFFFFFFFFu >> (32 - (int)keep)));
        }
        const int64_t sh = first - lo;               // position of bit `first` in the window
        if (sh >= 0 && sh < 32) v |= x << sh;
        else if (sh < 0 && sh > -32) v |= x >> (-sh);
    }
    return v;
}

__global__ void transmit_kernel(const TxParams p) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t k0 = 8 * j;
    if (k0 >= p.n_kept) return;
    double z[8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint64_t c[4] = {(uint64_t)(2 * j + h), 0ull, 0ull, 0ull};
        philox4x64(c, p.seed, p.stream_id);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const double u = unit53(c[2 * q]), v = unit53(c[2 * q + 1]);
            const double rad = sqrt(-2.0 * log(u)), ang = 2.0 * 3.14159265358979323846 * v;
            z[4 * h + 2 * q] = rad * cos(ang);
            z[4 * h + 2 * q + 1] = rad * sin(ang);
        }
    }
    uint32_t packed = 0;   // 4-bit and hard outputs of this thread's values
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t k = k0 + i;
        if (k >= p.n_kept) break;
        const int64_t g = k / p.kept_per_period;
        const int r = (int)(k - g * p.kept_per_period);
        const int64_t t = g * p.period + p.pos_phase[r];
        const int b = p.pos_b[r];
        const uint32_t reg = info_window(p, t - (p.K - 1)) & ((1u << p.K) - 1u);
        const uint32_t cbit = (uint32_t)__popc(p.gens[b] & reg) & 1u;
        const double y = (cbit ? -1.0 : 1.0) + p.sigma * z[i];
        switch (p.llr_type) {
        case VD_LLR_S8: {
            const double q = fmin(fmax(rint(32.0 * y), -127.0), 127.0);
            static_cast<int8_t *>(p.out)[k] = (int8_t)q;
            break;
        }
        case VD_LLR_S4: {
            const double q = fmin(fmax(rint(2.0 * y), -7.0), 7.0);
            packed |= ((uint32_t)(int)q & 0xFu) << (4 * i);
            break;
        }
        case VD_LLR_F16:
            static_cast<__half *>(p.out)[k] = __double2half(y * p.inv_var2);
            break;
        default:   // VD_LLR_HARD
            packed |= (y < 0.0 ? 1u : 0u) << i;
            break;
        }
    }
    if (p.llr_type == VD_LLR_S4) {
        // values k0 .. k0+7 are bytes 4j .. 4j+3; the last byte may be partial
        uint8_t *o = static_cast<uint8_t *>(p.out) + 4 * j;
        const int64_t nbytes = (p.n_kept + 1) / 2;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (4 * j + i < nbytes) o[i] = (uint8_t)(packed >> (8 * i));
    } else if (p.llr_type == VD_LLR_HARD) {
        static_cast<uint8_t *>(p.out)[j] = (uint8_t)packed;
    }
}

vd_status fail(vd_status st, const char *msg) {
    vd_internal_set_error(msg);
    return st;
}

}  // namespace

extern "C" int64_t vd_transmit_bytes(const vd_code *c, int64_t n_info, uint32_t flags, int llr_type) {
    if (!c || n_info < 0) return -1;
    const int64_t T = n_info + ((flags & VD_TERMINATED) ? c->K - 1 : 0);
    const int64_t kept = vd_num_kept(c, T);
    switch (llr_type) {
    case VD_LLR_S8: return kept;
    case VD_LLR_S4: return (kept + 1) / 2;
    case VD_LLR_F16: return 2 * kept;
    case VD_LLR_HARD: return (kept + 7) / 8;
    default: return -1;
    }
}

extern "C" vd_status vd_transmit(const vd_code *c, const uint32_t *d_bits, int64_t n_info, uint32_t flags,
                                 double sigma, uint64_t seed, uint64_t stream_id, int llr_type, void *d_out,
                                 void *stream) {
    if (!c) return fail(VD_EINVAL, "vd_transmit: code is NULL");
    if (n_info < 0 || n_info > ((int64_t)1 << 40)) return fail(VD_EINVAL, "vd_transmit: bad n_info");
    if (flags & ~(uint32_t)VD_TERMINATED) return fail(VD_EINVAL, "vd_transmit: flags other than VD_TERMINATED");
    if (!(sigma >= 0.0) || sigma > 1e6) return fail(VD_EINVAL, "vd_transmit: sigma must be in [0, 1e6]");
    if (llr_type == VD_LLR_F16 && sigma == 0.0)
        return fail(VD_EINVAL, "vd_transmit: fp16 LLRs (2 y / sigma^2) need sigma > 0");
    if (llr_type != VD_LLR_S8 && llr_type != VD_LLR_S4 && llr_type != VD_LLR_F16 && llr_type != VD_LLR_HARD)
        return fail(VD_EINVAL, "vd_transmit: unknown llr_type");
    const int64_t T = n_info + ((flags & VD_TERMINATED) ? c->K - 1 : 0);
    TxParams p;
    memset(&p, 0, sizeof p);
    p.n_kept = vd_num_kept(c, T);
    if (p.n_kept == 0) return VD_OK;
    if (!d_out || (n_info > 0 && !d_bits)) return fail(VD_EINVAL, "vd_transmit: NULL device pointer");
    p.bits = d_bits;
    p.n_info = n_info;
    p.n_words = (n_info + 31) / 32;
    p.K = c->K;
    p.beta = c->beta;
    p.period = c->period;
    p.kept_per_period = c->kept_per_period;
    for (int b = 0; b < c->beta; ++b) p.gens[b] = c->gens[b];
    int r = 0;
    for (int ph = 0; ph < c->period; ++ph)
        for (int b = 0; b < c->beta; ++b)
            if (c->punct[b][ph]) {
                p.pos_phase[r] = (uint8_t)ph;
                p.pos_b[r] = (uint8_t)b;
                ++r;
            }
    p.sigma = sigma;
    p.inv_var2 = sigma > 0.0 ? 2.0 / (sigma * sigma) : 0.0;
    p.seed = seed;
    p.stream_id = stream_id;
    p.llr_type = llr_type;
    p.out = d_out;
    const int64_t threads = (p.n_kept + 7) / 8;
    const int tb = 256;
    const int64_t blocks = (threads + tb - 1) / tb;
    if (blocks > 0x7FFFFFFF) return fail(VD_EINVAL, "vd_transmit: stream too long");
    transmit_kernel<<<(unsigned)blocks, tb, 0, (cudaStream_t)stream>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(VD_ECUDA, cudaGetErrorString(e));
    return VD_OK;
}
