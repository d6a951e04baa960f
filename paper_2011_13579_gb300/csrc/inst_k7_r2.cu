// Kernel instantiations: K=7 (171/133), radix 2, 1/2/4 lanes per frame pair.
#include "vd_variants.cuh"

namespace vd {

template cudaError_t launch_stream_v<7, false, 1>(const StreamParams &, int64_t, cudaStream_t);
template cudaError_t launch_batch_v<7, false, 1>(const BatchParams &, int64_t, cudaStream_t);
template cudaError_t occupancy_v<7, false, 1>(int *);
template cudaError_t launch_stream_persistent_v<7, false, 1>(const StreamParams &, int64_t, cudaStream_t);
template cudaError_t occupancy_stream_v<7, false, 1>(int *);
template cudaError_t launch_stream_v<7, false, 2>(const StreamParams &, int64_t, cudaStream_t);
template cudaError_t launch_batch_v<7, false, 2>(const BatchParams &, int64_t, cudaStream_t);
template cudaError_t occupancy_v<7, false, 2>(int *);
template cudaError_t launch_stream_persistent_v<7, false, 2>(const StreamParams &, int64_t, cudaStream_t);
template cudaError_t occupancy_stream_v<7, false, 2>(int *);
template cudaError_t launch_stream_v<7, false, 4>(const StreamParams &, int64_t, cudaStream_t);
template cudaError_t launch_batch_v<7, false, 4>(const BatchParams &, int64_t, cudaStream_t);
template cudaError_t occupancy_v<7, false, 4>(int *);
template cudaError_t launch_stream_persistent_v<7, false, 4>(const StreamParams &, int64_t, cudaStream_t);
template cudaError_t occupancy_stream_v<7, false, 4>(int *);

}  // namespace vd
