// Integer-issue microbenchmark (measurement): the throughput, per SM and
// clock, of the instruction classes the decode kernels issue — 16x2 adds and
// maxima, the fused add-then-max of the butterfly, 32-bit multiply-adds,
// three-input logic, byte permutes and funnel shifts — alone and in the
// mixes the kernels use.  It supplies the peak that the decoder's integer
// roofline divides by: the paper's add-compare-select (Eq. PM) runs on these
// units, not on tensor cores or over HBM.
//
// Each thread runs CH dependency chains for `iters` iterations of an
// unrolled body, so the issue rate, not latency, limits it (a chain of maxima
// against a constant would be idempotent, and the compiler shortens it, so
// the max variants take the neighbouring chain as their second operand).  One block
// per SM; its first thread records the SM's clock64() span between two block
// barriers, so the result is in SM clocks whatever the clock frequency was.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/vd.h"
#include "vd_code.h"
#include "vd_device.cuh"

namespace {

constexpr int CH = 8;      // independent chains per thread
constexpr int UNR = 16;    // unrolled body repetitions per iteration

__device__ __forceinline__ uint32_t lop3_xor3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t shf_l(uint32_t a, uint32_t b, uint32_t s) {
    uint32_t d;
    asm("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(s));
    return d;
}

// One body of variant V on the chains x: 8 operations (16 for variant 10).
template <int V>
__device__ __forceinline__ void body(uint32_t (&x)[CH], uint32_t a, uint32_t b, uint32_t c, uint32_t m) {
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        if constexpr (V == 0) {          // 16x2 add
            x[k] = vd::add_u16x2(x[k], a);
        } else if constexpr (V == 1) {   // 16x2 max (of the neighbouring chain: not idempotent)
            x[k] = vd::max_u16x2(x[k], x[(k + 1) % CH]);
        } else if constexpr (V == 2) {   // fused add-then-max (the butterfly's second half)
            x[k] = vd::addmax_u16x2(x[k], a, b ^ (uint32_t)k);
        } else if constexpr (V == 3) {   // 32-bit multiply-add
            x[k] = vd::imad(x[k], m, c);
        } else if constexpr (V == 4) {   // three-input logic
            x[k] = lop3_xor3(x[k], a, b);
        } else if constexpr (V == 5) {   // byte permute
            x[k] = vd::prmt(x[k], a, c);
        } else if constexpr (V == 6) {   // funnel shift
            x[k] = shf_l(x[k], a, 3u);
        } else if constexpr (V == 7) {   // 16x2 add and multiply-add, 1:1
            x[k] = (k & 1) ? vd::imad(x[k], m, c) : vd::add_u16x2(x[k], a);
        } else if constexpr (V == 8) {   // fused add-max and multiply-add, 1:1
            x[k] = (k & 1) ? vd::imad(x[k], m, c) : vd::addmax_u16x2(x[k], a, b ^ (uint32_t)k);
        } else if constexpr (V == 9) {   // 16x2 max and three-input logic, 1:1
            // (both read the neighbouring chain, so no pair of steps folds away)
            x[k] = (k & 1) ? lop3_xor3(x[k], a, x[(k + 1) % CH]) : vd::max_u16x2(x[k], x[(k + 1) % CH]);
        }
    }
    if constexpr (V == 10) {
        // the radix-2 butterfly of the decoder on 4 register pairs: two 16x2
        // adds for the odd candidates and two fused add-max (4 instructions,
        // 12 algorithmic operations for two frames)
#pragma unroll
        for (int k = 0; k < CH; k += 2) {
            const uint32_t pa = x[k], pb = x[k + 1];
            const uint32_t cb0 = vd::add_u16x2(pb, a), cb1 = vd::add_u16x2(pb, b);
            x[k] = vd::addmax_u16x2(pa, c, cb0);
            x[k + 1] = vd::addmax_u16x2(pa, m, cb1);
        }
    }
}

template <int V>
__global__ void __launch_bounds__(1024) int_peak_kernel(int64_t iters, uint32_t one, long long *cycles,
                                                        uint32_t *sink) {
    uint32_t x[CH];
    const uint32_t t = threadIdx.x + 1u;
#pragma unroll
    for (int k = 0; k < CH; ++k) x[k] = t * 0x9E3779B9u + (uint32_t)k;
    // runtime operands the compiler cannot fold
    const uint32_t a = (t & 7u) * 0x00010001u, b = (t >> 3) * 0x00030003u, c = 0x3210u + (t & 1u);
    const uint32_t m = one;   // 1, from the host: a multiply-add the compiler must keep
    __syncthreads();
    const long long t0 = clock64();
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNR; ++u) body<V>(x, a, b, c, m);
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < CH; ++k) s ^= x[k];
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int V>
cudaError_t launch(int n_blocks, int64_t iters, long long *cycles, uint32_t *sink, cudaStream_t st) {
    int_peak_kernel<V><<<n_blocks, 1024, 0, st>>>(iters, 1u, cycles, sink);
    return cudaGetLastError();
}

}  // namespace

extern "C" vd_status vd_int_peak(int variant, int64_t iters, int n_blocks, int64_t *d_cycles,
                                 uint32_t *d_sink, void *stream) {
    if (iters <= 0 || n_blocks <= 0 || !d_cycles || !d_sink) {
        vd_internal_set_error("vd_int_peak: iters and n_blocks must be positive, buffers non-NULL");
        return VD_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    long long *cy = reinterpret_cast<long long *>(d_cycles);
    cudaError_t e;
    switch (variant) {
    case 0: e = launch<0>(n_blocks, iters, cy, d_sink, st); break;
    case 1: e = launch<1>(n_blocks, iters, cy, d_sink, st); break;
    case 2: e = launch<2>(n_blocks, iters, cy, d_sink, st); break;
    case 3: e = launch<3>(n_blocks, iters, cy, d_sink, st); break;
    case 4: e = launch<4>(n_blocks, iters, cy, d_sink, st); break;
    case 5: e = launch<5>(n_blocks, iters, cy, d_sink, st); break;
    case 6: e = launch<6>(n_blocks, iters, cy, d_sink, st); break;
    case 7: e = launch<7>(n_blocks, iters, cy, d_sink, st); break;
    case 8: e = launch<8>(n_blocks, iters, cy, d_sink, st); break;
    case 9: e = launch<9>(n_blocks, iters, cy, d_sink, st); break;
    case 10: e = launch<10>(n_blocks, iters, cy, d_sink, st); break;
    default:
        vd_internal_set_error("vd_int_peak: variant must be 0..10");
        return VD_EINVAL;
    }
    if (e != cudaSuccess) {
        vd_internal_set_error(cudaGetErrorString(e));
        return VD_ECUDA;
    }
    return VD_OK;
}
