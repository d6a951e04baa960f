// Branch-metric gate (measurement): the 2^beta branch metrics of Eq. BM for
// the (2,1,7) code, for a pair of frames per thread, computed two ways that
// deliver the same packed 16x2 values to every thread —
//
//   * CUDA cores: the decoder's own form (byte permutes with sign extension,
//     16x2 negation and adds);
//   * tensor cores: the paper's formulation (Sec. V, D = Theta L): the +-1
//     output patterns of the code (rows of Theta) times the LLR columns of 64
//     frames, as eight mma.sync m16n8k32 s8 -> s32 per stage and warp, then a
//     shared-memory transpose from the accumulator layout (a pattern's values
//     for eight frames across four lanes) to the decoder's layout (all
//     patterns of one frame pair in one lane).
//
// Both fold every metric into a per-thread checksum (and optionally write
// them out), so the two kernels do identical consumer work.  The decoder
// only adopts the tensor-core form if it is faster here.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/vd.h"
#include "vd_code.h"
#include "vd_device.cuh"

namespace {

// LLR layout: [n_stages][n_pairs] 32-bit words, bytes (l0, l1) of frame 0
// then (l0, l1) of frame 1.  Metric layout (optional out): [n_stages][4][n_pairs].

__device__ __forceinline__ void bm_cuda_core(uint32_t w, uint32_t (&A)[4]) {
    const uint32_t l0 = vd::prmt(w, 0u, 0xA280u);   // sign-extended bytes 0 | 2
    const uint32_t l1 = vd::prmt(w, 0u, 0xB391u);   // sign-extended bytes 1 | 3
    const uint32_t n0 = vd::neg_s16x2(l0), n1 = vd::neg_s16x2(l1);
    A[0] = vd::add_s16x2(l0, l1);   // pattern 00: +l0 +l1
    A[1] = vd::add_s16x2(n0, l1);   // pattern 01 (bit 0 set): -l0 +l1
    A[2] = vd::add_s16x2(l0, n1);   // pattern 10: +l0 -l1
    A[3] = vd::add_s16x2(n0, n1);   // pattern 11: -l0 -l1
}

__device__ __forceinline__ uint32_t fold(uint32_t cs, const uint32_t (&A)[4]) {
    return ((cs ^ A[0]) + A[1]) ^ (A[2] + A[3]);
}

__global__ void bm_kernel_cuda(const uint32_t *llr, int64_t n_pairs, int32_t n_stages, uint32_t *checksum,
                               uint32_t *out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    uint32_t cs = 0;
    for (int32_t s = 0; s < n_stages; ++s) {
        uint32_t A[4];
        bm_cuda_core(__ldg(llr + (int64_t)s * n_pairs + p), A);
        cs = fold(cs, A);
        if (out) {
#pragma unroll
            for (int x = 0; x < 4; ++x) out[((int64_t)s * 4 + x) * n_pairs + p] = A[x];
        }
    }
    checksum[p] = cs;
}

// One warp = 32 frame pairs (64 frames); n_pairs must be a multiple of 32.
__global__ void bm_kernel_mma(const uint32_t *llr, int64_t n_pairs, int32_t n_stages, uint32_t *checksum,
                              uint32_t *out) {
    __shared__ uint32_t tr[4][8][4][4];   // [warp in block][mma m][pattern][tid4]
    const int wib = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t p0 = warp * 32;
    if (p0 >= n_pairs) return;
    const int gid = lane >> 2, tid4 = lane & 3;
    // Theta fragment (rows = patterns 0..3, columns = outputs 0, 1): +1 / -1 bytes
    uint32_t a0 = 0;
    if (gid < 4 && tid4 == 0) a0 = ((gid & 1) ? 0xFFu : 0x01u) | ((gid & 2) ? 0xFF00u : 0x0100u);
    const uint32_t zero = 0;
    uint32_t cs = 0;
    for (int32_t s = 0; s < n_stages; ++s) {
        const uint32_t w = __ldg(llr + (int64_t)s * n_pairs + p0 + lane);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            // column gid of mma m = frame 8m + gid = half (gid & 1) of pair 4m + gid/2
            const uint32_t wp = __shfl_sync(0xFFFFFFFFu, w, 4 * m + (gid >> 1));
            const uint32_t b0 = tid4 == 0 ? ((gid & 1) ? (wp >> 16) : (wp & 0xFFFFu)) : 0u;
            int32_t d0 = 0, d1 = 0, d2 = 0, d3 = 0;
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 "
                "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
                : "+r"(d0), "+r"(d1), "+r"(d2), "+r"(d3)
                : "r"(a0), "r"(zero), "r"(zero), "r"(zero), "r"(b0), "r"(zero));
            // lane (gid < 4, tid4) holds pattern gid of pair 4m + tid4, both halves
            if (gid < 4) tr[wib][m][gid][tid4] = ((uint32_t)d0 & 0xFFFFu) | ((uint32_t)d1 << 16);
        }
        __syncwarp();
        uint32_t A[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) A[x] = tr[wib][lane >> 2][x][lane & 3];
        __syncwarp();
        cs = fold(cs, A);
        if (out) {
#pragma unroll
            for (int x = 0; x < 4; ++x) out[((int64_t)s * 4 + x) * n_pairs + p0 + lane] = A[x];
        }
    }
    checksum[p0 + lane] = cs;
}

}  // namespace

extern "C" vd_status vd_bm_gate(int variant, const void *d_llr, int64_t n_pairs, int32_t n_stages,
                                uint32_t *d_checksum, uint32_t *d_metrics, void *stream) {
    if (variant != 0 && variant != 1) {
        vd_internal_set_error("variant must be 0 (CUDA cores) or 1 (tensor cores)");
        return VD_EINVAL;
    }
    if (!d_llr || !d_checksum || n_pairs <= 0 || n_stages <= 0 || n_pairs % 32 != 0) {
        vd_internal_set_error("need device buffers, n_stages > 0 and n_pairs a positive multiple of 32");
        return VD_EINVAL;
    }
    const int threads = 128;
    const int64_t blocks = (n_pairs + threads - 1) / threads;
    if (blocks > 0x7FFFFFFF) {
        vd_internal_set_error("too many pairs for one launch");
        return VD_EINVAL;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    if (variant == 0)
        bm_kernel_cuda<<<(unsigned)blocks, threads, 0, cs>>>((const uint32_t *)d_llr, n_pairs, n_stages,
                                                              d_checksum, d_metrics);
    else
        bm_kernel_mma<<<(unsigned)blocks, threads, 0, cs>>>((const uint32_t *)d_llr, n_pairs, n_stages,
                                                             d_checksum, d_metrics);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        vd_internal_set_error(cudaGetErrorString(e));
        return VD_ECUDA;
    }
    return VD_OK;
}
