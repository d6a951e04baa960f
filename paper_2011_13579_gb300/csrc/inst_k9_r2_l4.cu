// Kernel instantiations: K=9 (557/663/711), radix 2, 4 lanes per frame pair.
#include "vd_variants.cuh"

namespace vd {

template cudaError_t launch_stream_v<9, false, 4>(const StreamParams &, int64_t, cudaStream_t);
template cudaError_t launch_batch_v<9, false, 4>(const BatchParams &, int64_t, cudaStream_t);
template cudaError_t occupancy_v<9, false, 4>(int *);
template cudaError_t launch_stream_persistent_v<9, false, 4>(const StreamParams &, int64_t, cudaStream_t);
template cudaError_t occupancy_stream_v<9, false, 4>(int *);

}  // namespace vd
