// Runtime dispatch from (lanes, radix) to the compiled kernel variants, and
// the host-side geometry of each (no kernel code is instantiated here).
#include "vd_variants.cuh"

namespace vd {

cudaError_t launch_stream_k7(int lanes, bool radix4, const StreamParams &p, int64_t blocks,
                             cudaStream_t st) {
#define X(K, R4, L) if (K == 7 && radix4 == R4 && lanes == L) return launch_stream_v<K, R4, L>(p, blocks, st);
    VD_VARIANT_LIST(X)
#undef X
    return cudaErrorInvalidValue;
}
cudaError_t launch_stream_k9(int lanes, bool radix4, const StreamParams &p, int64_t blocks,
                             cudaStream_t st) {
#define X(K, R4, L) if (K == 9 && radix4 == R4 && lanes == L) return launch_stream_v<K, R4, L>(p, blocks, st);
    VD_VARIANT_LIST(X)
#undef X
    return cudaErrorInvalidValue;
}
cudaError_t launch_batch_k7(int lanes, bool radix4, const BatchParams &p, int64_t blocks,
                            cudaStream_t st) {
#define X(K, R4, L) if (K == 7 && radix4 == R4 && lanes == L) return launch_batch_v<K, R4, L>(p, blocks, st);
    VD_VARIANT_LIST(X)
#undef X
    return cudaErrorInvalidValue;
}
cudaError_t launch_batch_k9(int lanes, bool radix4, const BatchParams &p, int64_t blocks,
                            cudaStream_t st) {
#define X(K, R4, L) if (K == 9 && radix4 == R4 && lanes == L) return launch_batch_v<K, R4, L>(p, blocks, st);
    VD_VARIANT_LIST(X)
#undef X
    return cudaErrorInvalidValue;
}
cudaError_t batch_occupancy_k7(int lanes, bool radix4, int *blocks_per_sm) {
#define X(K, R4, L) if (K == 7 && radix4 == R4 && lanes == L) return occupancy_v<K, R4, L>(blocks_per_sm);
    VD_VARIANT_LIST(X)
#undef X
    return cudaErrorInvalidValue;
}
cudaError_t batch_occupancy_k9(int lanes, bool radix4, int *blocks_per_sm) {
#define X(K, R4, L) if (K == 9 && radix4 == R4 && lanes == L) return occupancy_v<K, R4, L>(blocks_per_sm);
    VD_VARIANT_LIST(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_stream_persistent(int K, int lanes, bool radix4, const StreamParams &p, int64_t blocks,
                                     cudaStream_t st) {
#define X(KK, R4, L) \
    if (K == KK && radix4 == R4 && lanes == L) return launch_stream_persistent_v<KK, R4, L>(p, blocks, st);
    VD_VARIANT_LIST(X)
#undef X
    return cudaErrorInvalidValue;
}
cudaError_t stream_persistent_occupancy(int K, int lanes, bool radix4, int *blocks_per_sm) {
#define X(KK, R4, L) if (K == KK && radix4 == R4 && lanes == L) return occupancy_stream_v<KK, R4, L>(blocks_per_sm);
    VD_VARIANT_LIST(X)
#undef X
    return cudaErrorInvalidValue;
}

bool geom_k7(int lanes, bool radix4, KernelGeom *g) {
#define X(K, R4, L)                                                        \
    if (K == 7 && radix4 == R4 && lanes == L) {                            \
        g->U = StreamCfg<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4>::U;   \
        g->NW = StreamCfg<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4>::SW; \
        return true;                                                       \
    }
    VD_VARIANT_LIST(X)
#undef X
    return false;
}
bool geom_k9(int lanes, bool radix4, KernelGeom *g) {
#define X(K, R4, L)                                                        \
    if (K == 9 && radix4 == R4 && lanes == L) {                            \
        g->U = StreamCfg<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4>::U;   \
        g->NW = StreamCfg<K, CodeOf<K>::BETA, CodeOf<K>::GENS, L, R4>::SW; \
        return true;                                                       \
    }
    VD_VARIANT_LIST(X)
#undef X
    return false;
}

}  // namespace vd
