// Kernel instantiations for the K=9 code (generators 557/663/711).
#include "vd_launch.h"
#include "vd_stream_f32.cuh"

namespace vd {

template <int L, bool R4>
static cudaError_t launch_one(const StreamParams &p, int64_t blocks, cudaStream_t st) {
    stream_kernel<9, 3, GENS_K9, L, R4, kThreads><<<(unsigned)blocks, kThreads, 0, st>>>(p);
    return cudaGetLastError();
}

template <int L, bool R4>
static cudaError_t launch_batch(const BatchParams &p, int64_t blocks, cudaStream_t st) {
    batch_kernel<9, 3, GENS_K9, L, R4, kThreads><<<(unsigned)blocks, kThreads, 0, st>>>(p);
    return cudaGetLastError();
}

template <int L, bool R4>
static cudaError_t occ(int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, batch_kernel<9, 3, GENS_K9, L, R4, kThreads>, kThreads, 0);
}

cudaError_t launch_stream_k9(int lanes, bool radix4, const StreamParams &p, int64_t blocks,
                             cudaStream_t st) {
    if (radix4) {
        switch (lanes) {
        case 4: return launch_one<4, true>(p, blocks, st);
        case 8: return launch_one<8, true>(p, blocks, st);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (lanes) {
    case 4: return launch_one<4, false>(p, blocks, st);
    case 8: return launch_one<8, false>(p, blocks, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_k9(int lanes, bool radix4, const BatchParams &p, int64_t blocks,
                            cudaStream_t st) {
    if (radix4) {
        switch (lanes) {
        case 4: return launch_batch<4, true>(p, blocks, st);
        case 8: return launch_batch<8, true>(p, blocks, st);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (lanes) {
    case 4: return launch_batch<4, false>(p, blocks, st);
    case 8: return launch_batch<8, false>(p, blocks, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t batch_occupancy_k9(int lanes, bool radix4, int *blocks_per_sm) {
    if (radix4) {
        switch (lanes) {
        case 4: return occ<4, true>(blocks_per_sm);
        case 8: return occ<8, true>(blocks_per_sm);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (lanes) {
    case 4: return occ<4, false>(blocks_per_sm);
    case 8: return occ<8, false>(blocks_per_sm);
    default: return cudaErrorInvalidValue;
    }
}

bool geom_k9(int lanes, bool radix4, KernelGeom *g) {
    switch (lanes) {
    case 4:
        g->U = radix4 ? StreamCfg<9, 3, GENS_K9, 4, true>::U : StreamCfg<9, 3, GENS_K9, 4, false>::U;
        g->NW = radix4 ? StreamCfg<9, 3, GENS_K9, 4, true>::NW : StreamCfg<9, 3, GENS_K9, 4, false>::NW;
        return true;
    case 8:
        g->U = radix4 ? StreamCfg<9, 3, GENS_K9, 8, true>::U : StreamCfg<9, 3, GENS_K9, 8, false>::U;
        g->NW = radix4 ? StreamCfg<9, 3, GENS_K9, 8, true>::NW : StreamCfg<9, 3, GENS_K9, 8, false>::NW;
        return true;
    default: return false;
    }
}

cudaError_t launch_stream_f32_k9(int lanes, const StreamParams &p, int64_t blocks, cudaStream_t st) {
    switch (lanes) {
    case 8: stream_kernel_f32<9, 3, GENS_K9, 8, kThreads><<<(unsigned)blocks, kThreads, 0, st>>>(p); return cudaGetLastError();
    default: return cudaErrorInvalidValue;
    }
}

bool geom_f32_k9(int lanes, KernelGeom *g) {
    switch (lanes) {
    case 8: g->U = StreamCfgF32<9, 3, GENS_K9, 8>::U; g->NW = StreamCfgF32<9, 3, GENS_K9, 8>::NW; return true;
    default: return false;
    }
}

}  // namespace vd
