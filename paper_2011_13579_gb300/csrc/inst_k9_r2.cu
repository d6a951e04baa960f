// Radix-2 kernel instantiations for the K=9 code (generators 557/663/711).
#include "vd_variants.cuh"

namespace vd {

using V_k9_r2 = Variants<9, 3, GENS_K9, false, 4, 8>;

cudaError_t launch_stream_k9_r2(int lanes, const StreamParams &p, int64_t blocks, cudaStream_t st) {
    return V_k9_r2::stream(lanes, p, blocks, st);
}
cudaError_t launch_batch_k9_r2(int lanes, const BatchParams &p, int64_t blocks, cudaStream_t st) {
    return V_k9_r2::batch(lanes, p, blocks, st);
}
cudaError_t occupancy_k9_r2(int lanes, int *blocks_per_sm) {
    return V_k9_r2::occupancy(lanes, blocks_per_sm);
}

}  // namespace vd
