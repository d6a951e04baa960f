// fp16-LLR / fp32-metric stream kernel instantiations: K=7 with 2 lanes per
// frame pair, K=9 with 8.
#include "vd_launch.h"
#include "vd_stream_f32.cuh"

namespace vd {

cudaError_t launch_stream_f32_k7(int lanes, const StreamParams &p, int64_t blocks, cudaStream_t st) {
    if (lanes != 2) return cudaErrorInvalidValue;
    stream_kernel_f32<7, 2, GENS_K7, 2, kThreads><<<(unsigned)blocks, kThreads, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_stream_f32_k9(int lanes, const StreamParams &p, int64_t blocks, cudaStream_t st) {
    if (lanes != 8) return cudaErrorInvalidValue;
    stream_kernel_f32<9, 3, GENS_K9, 8, kThreads><<<(unsigned)blocks, kThreads, 0, st>>>(p);
    return cudaGetLastError();
}

bool geom_f32_k7(int lanes, KernelGeom *g) {
    if (lanes != 2) return false;
    g->U = StreamCfgF32<7, 2, GENS_K7, 2>::U;
    g->NW = StreamCfgF32<7, 2, GENS_K7, 2>::NW;
    return true;
}

bool geom_f32_k9(int lanes, KernelGeom *g) {
    if (lanes != 8) return false;
    g->U = StreamCfgF32<9, 3, GENS_K9, 8>::U;
    g->NW = StreamCfgF32<9, 3, GENS_K9, 8>::NW;
    return true;
}

}  // namespace vd
