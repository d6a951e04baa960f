// Compiled variants of the integer kernels: one (code, radix, lanes) triple
// per explicit instantiation.  Instantiation units include this header with
// the kernel definitions; the dispatch unit only needs the declarations, so
// the heavy kernels of different variants compile in parallel.
#pragma once
#include "vd_launch.h"

namespace vd {

template <int K> struct CodeOf;
template <> struct CodeOf<7> { static constexpr int BETA = 2; static constexpr uint64_t GENS = GENS_K7; };
template <> struct CodeOf<9> { static constexpr int BETA = 3; static constexpr uint64_t GENS = GENS_K9; };

template <int K, bool R4, int L>
cudaError_t launch_stream_v(const StreamParams &p, int64_t blocks, cudaStream_t st) {
    stream_kernel<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4, kThreads><<<(unsigned)blocks, kThreads, 0, st>>>(p);
    return cudaGetLastError();
}

template <int K, bool R4, int L>
cudaError_t launch_batch_v(const BatchParams &p, int64_t blocks, cudaStream_t st) {
    batch_kernel<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4, kThreads><<<(unsigned)blocks, kThreads, 0, st>>>(p);
    return cudaGetLastError();
}

template <int K, bool R4, int L>
cudaError_t occupancy_v(int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, batch_kernel<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4, kThreads>, kThreads, 0);
}

template <int K, bool R4, int L>
cudaError_t launch_stream_persistent_v(const StreamParams &p, int64_t blocks, cudaStream_t st) {
    stream_persistent_kernel<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4, kThreads>
        <<<(unsigned)blocks, kThreads, 0, st>>>(p);
    return cudaGetLastError();
}

template <int K, bool R4, int L>
cudaError_t occupancy_stream_v(int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, stream_persistent_kernel<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4, kThreads>,
        kThreads, 0);
}

// The instantiations that exist (each compiled in one inst_*.cu unit).
#define VD_VARIANT_LIST(X) \
    X(7, false, 1) X(7, false, 2) X(7, false, 4) X(7, true, 1) X(7, true, 2) X(7, true, 4) \
    X(9, false, 4) X(9, false, 8) X(9, true, 4) X(9, true, 8)

#define VD_DECLARE_VARIANT(K, R4, L)                                                           \
    extern template cudaError_t launch_stream_v<K, R4, L>(const StreamParams &, int64_t, cudaStream_t); \
    extern template cudaError_t launch_batch_v<K, R4, L>(const BatchParams &, int64_t, cudaStream_t);   \
    extern template cudaError_t occupancy_v<K, R4, L>(int *);                                   \
    extern template cudaError_t launch_stream_persistent_v<K, R4, L>(const StreamParams &, int64_t, \
                                                                     cudaStream_t);                 \
    extern template cudaError_t occupancy_stream_v<K, R4, L>(int *);
VD_VARIANT_LIST(VD_DECLARE_VARIANT)
#undef VD_DECLARE_VARIANT


}  // namespace vd
