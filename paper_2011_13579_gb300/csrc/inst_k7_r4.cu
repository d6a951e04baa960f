// Radix-4 kernel instantiations for the K=7 code (generators 171/133).
#include "vd_variants.cuh"

namespace vd {

using V_k7_r4 = Variants<7, 2, GENS_K7, true, 1, 2, 4>;

cudaError_t launch_stream_k7_r4(int lanes, const StreamParams &p, int64_t blocks, cudaStream_t st) {
    return V_k7_r4::stream(lanes, p, blocks, st);
}
cudaError_t launch_batch_k7_r4(int lanes, const BatchParams &p, int64_t blocks, cudaStream_t st) {
    return V_k7_r4::batch(lanes, p, blocks, st);
}
cudaError_t occupancy_k7_r4(int lanes, int *blocks_per_sm) {
    return V_k7_r4::occupancy(lanes, blocks_per_sm);
}

}  // namespace vd
