// Launchers for the kernel instantiations compiled in separate translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "vd_batch.cuh"

namespace vd {

// Codes with compiled kernels.  Generators are packed 16 bits each.
constexpr uint64_t pack_gens(uint32_t g0, uint32_t g1, uint32_t g2 = 0, uint32_t g3 = 0) {
    return (uint64_t)g0 | ((uint64_t)g1 << 16) | ((uint64_t)g2 << 32) | ((uint64_t)g3 << 48);
}
constexpr uint64_t GENS_K7 = pack_gens(0171, 0133);
constexpr uint64_t GENS_K9 = pack_gens(0557, 0663, 0711);

enum CodeKind { KIND_NONE = 0, KIND_K7_R2 = 1, KIND_K9_R3 = 2 };

constexpr int kThreads = 128;

// Geometry of one instantiation, for scratch sizing on the host.
struct KernelGeom {
    int U;       // stages per chunk
    int NW;      // survivor scratch words per thread per stage (StreamCfg::SW)
};

// Returns cudaErrorInvalidValue if (kind, lanes, radix4) has no instantiation.
cudaError_t launch_stream_k7(int lanes, bool radix4, const StreamParams &p, int64_t blocks,
                             cudaStream_t st);
cudaError_t launch_stream_k9(int lanes, bool radix4, const StreamParams &p, int64_t blocks,
                             cudaStream_t st);
cudaError_t launch_batch_k7(int lanes, bool radix4, const BatchParams &p, int64_t blocks,
                            cudaStream_t st);
cudaError_t launch_batch_k9(int lanes, bool radix4, const BatchParams &p, int64_t blocks,
                            cudaStream_t st);
cudaError_t batch_occupancy_k7(int lanes, bool radix4, int *blocks_per_sm);
cudaError_t batch_occupancy_k9(int lanes, bool radix4, int *blocks_per_sm);
// Persistent stream decode (K = 7 or 9): p.counter must be zero at launch.
cudaError_t launch_stream_persistent(int K, int lanes, bool radix4, const StreamParams &p, int64_t blocks,
                                     cudaStream_t st);
cudaError_t stream_persistent_occupancy(int K, int lanes, bool radix4, int *blocks_per_sm);
cudaError_t launch_stream_f32_k7(int lanes, const StreamParams &p, int64_t blocks, cudaStream_t st);
cudaError_t launch_stream_f32_k9(int lanes, const StreamParams &p, int64_t blocks, cudaStream_t st);
bool geom_f32_k7(int lanes, KernelGeom *g);
bool geom_f32_k9(int lanes, KernelGeom *g);
bool geom_k7(int lanes, bool radix4, KernelGeom *g);
bool geom_k9(int lanes, bool radix4, KernelGeom *g);

}  // namespace vd
