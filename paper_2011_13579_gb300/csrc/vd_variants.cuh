// Compiled variants of the integer kernels: one (code, radix, lanes) triple
// per explicit instantiation.  Instantiation units include this header with
// the kernel definitions; the dispatch unit only needs the declarations, so
// the heavy kernels of different variants compile in parallel.
#pragma once
#include <atomic>
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

// Dynamic shared memory of the persistent kernels (PersistentSmem).  A
// block may use more than 48 KB only after the kernel opts in, once per
// device (the attribute belongs to the kernel in that device's context);
// the flags are per kernel instantiation, devices 0..63.
template <int K, bool R4, int L>
constexpr size_t persistent_smem_bytes() {
    return PersistentSmem<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4, kThreads>::BYTES;
}

template <typename Kern>
cudaError_t opt_in_smem(Kern kern, size_t bytes, std::atomic<uint64_t> &done) {
    if (bytes <= 48u * 1024u) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

template <int K, bool R4, int L>
cudaError_t batch_smem_opt_in() {
    static std::atomic<uint64_t> done{0};
    return opt_in_smem(batch_kernel<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4, kThreads>,
                       persistent_smem_bytes<K, R4, L>(), done);
}

template <int K, bool R4, int L>
cudaError_t stream_persistent_smem_opt_in() {
    static std::atomic<uint64_t> done{0};
    return opt_in_smem(stream_persistent_kernel<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4, kThreads>,
                       persistent_smem_bytes<K, R4, L>(), done);
}

template <int K, bool R4, int L>
cudaError_t launch_batch_v(const BatchParams &p, int64_t blocks, cudaStream_t st) {
    const cudaError_t e = batch_smem_opt_in<K, R4, L>();
    if (e != cudaSuccess) return e;
    if (!p.chained) {
        batch_kernel<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4, kThreads>
            <<<(unsigned)blocks, kThreads, persistent_smem_bytes<K, R4, L>(), st>>>(p);
        return cudaGetLastError();
    }
    // programmatic dependent launch: may start before the kernel before it
    // on the stream completes (the kernel's griddepcontrol waits order it)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = persistent_smem_bytes<K, R4, L>();
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_kernel<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4, kThreads>, p);
}

template <int K, bool R4, int L>
cudaError_t occupancy_v(int *blocks_per_sm) {
    const cudaError_t e = batch_smem_opt_in<K, R4, L>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, batch_kernel<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4, kThreads>, kThreads,
        persistent_smem_bytes<K, R4, L>());
}

template <int K, bool R4, int L>
cudaError_t launch_stream_persistent_v(const StreamParams &p, int64_t blocks, cudaStream_t st) {
    const cudaError_t e = stream_persistent_smem_opt_in<K, R4, L>();
    if (e != cudaSuccess) return e;
    stream_persistent_kernel<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4, kThreads>
        <<<(unsigned)blocks, kThreads, persistent_smem_bytes<K, R4, L>(), st>>>(p);
    return cudaGetLastError();
}

template <int K, bool R4, int L>
cudaError_t occupancy_stream_v(int *blocks_per_sm) {
    const cudaError_t e = stream_persistent_smem_opt_in<K, R4, L>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, stream_persistent_kernel<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4, kThreads>,
        kThreads, persistent_smem_bytes<K, R4, L>());
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
