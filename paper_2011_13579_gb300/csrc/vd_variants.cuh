// Runtime dispatch from a lane count to the compiled kernel instantiations of
// one (code, radix) variant.  Each instantiation set lives in its own
// translation unit so the heavy kernels compile in parallel.
#pragma once
#include "vd_launch.h"
#include "vd_stream_f32.cuh"

namespace vd {

template <int K, int BETA, uint64_t GENS, bool R4, int... Ls>
struct Variants {
    template <int L>
    static cudaError_t stream_one(const StreamParams &p, int64_t blocks, cudaStream_t st) {
        stream_kernel<K, BETA, GENS, L, R4, kThreads><<<(unsigned)blocks, kThreads, 0, st>>>(p);
        return cudaGetLastError();
    }
    template <int L>
    static cudaError_t batch_one(const BatchParams &p, int64_t blocks, cudaStream_t st) {
        batch_kernel<K, BETA, GENS, L, R4, kThreads><<<(unsigned)blocks, kThreads, 0, st>>>(p);
        return cudaGetLastError();
    }
    template <int L>
    static cudaError_t occ_one(int *blocks_per_sm) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            blocks_per_sm, batch_kernel<K, BETA, GENS, L, R4, kThreads>, kThreads, 0);
    }

    static cudaError_t stream(int lanes, const StreamParams &p, int64_t blocks, cudaStream_t st) {
        cudaError_t e = cudaErrorInvalidValue;
        (void)((lanes == Ls && ((e = stream_one<Ls>(p, blocks, st)), true)) || ...);
        return e;
    }
    static cudaError_t batch(int lanes, const BatchParams &p, int64_t blocks, cudaStream_t st) {
        cudaError_t e = cudaErrorInvalidValue;
        (void)((lanes == Ls && ((e = batch_one<Ls>(p, blocks, st)), true)) || ...);
        return e;
    }
    static cudaError_t occupancy(int lanes, int *blocks_per_sm) {
        cudaError_t e = cudaErrorInvalidValue;
        (void)((lanes == Ls && ((e = occ_one<Ls>(blocks_per_sm)), true)) || ...);
        return e;
    }
};

// Per-variant entry points (defined in inst_k{7,9}_r{2,4}.cu).
cudaError_t launch_stream_k7_r2(int lanes, const StreamParams &p, int64_t blocks, cudaStream_t st);
cudaError_t launch_stream_k7_r4(int lanes, const StreamParams &p, int64_t blocks, cudaStream_t st);
cudaError_t launch_stream_k9_r2(int lanes, const StreamParams &p, int64_t blocks, cudaStream_t st);
cudaError_t launch_stream_k9_r4(int lanes, const StreamParams &p, int64_t blocks, cudaStream_t st);
cudaError_t launch_batch_k7_r2(int lanes, const BatchParams &p, int64_t blocks, cudaStream_t st);
cudaError_t launch_batch_k7_r4(int lanes, const BatchParams &p, int64_t blocks, cudaStream_t st);
cudaError_t launch_batch_k9_r2(int lanes, const BatchParams &p, int64_t blocks, cudaStream_t st);
cudaError_t launch_batch_k9_r4(int lanes, const BatchParams &p, int64_t blocks, cudaStream_t st);
cudaError_t occupancy_k7_r2(int lanes, int *blocks_per_sm);
cudaError_t occupancy_k7_r4(int lanes, int *blocks_per_sm);
cudaError_t occupancy_k9_r2(int lanes, int *blocks_per_sm);
cudaError_t occupancy_k9_r4(int lanes, int *blocks_per_sm);

}  // namespace vd
