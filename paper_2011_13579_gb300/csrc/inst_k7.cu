// Kernel instantiations for the K=7 code (generators 171/133).
#include "vd_launch.h"
#include "vd_stream_f32.cuh"

namespace vd {

template <int L, bool R4>
static cudaError_t launch_one(const StreamParams &p, int64_t blocks, cudaStream_t st) {
    stream_kernel<7, 2, GENS_K7, L, R4, kThreads><<<(unsigned)blocks, kThreads, 0, st>>>(p);
    return cudaGetLastError();
}

template <int L, bool R4>
static cudaError_t launch_batch(const BatchParams &p, int64_t blocks, cudaStream_t st) {
    batch_kernel<7, 2, GENS_K7, L, R4, kThreads><<<(unsigned)blocks, kThreads, 0, st>>>(p);
    return cudaGetLastError();
}

template <int L, bool R4>
static cudaError_t occ(int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, batch_kernel<7, 2, GENS_K7, L, R4, kThreads>, kThreads, 0);
}

cudaError_t launch_stream_k7(int lanes, bool radix4, const StreamParams &p, int64_t blocks,
                             cudaStream_t st) {
    if (radix4) {
        switch (lanes) {
        case 1: return launch_one<1, true>(p, blocks, st);
        case 2: return launch_one<2, true>(p, blocks, st);
        case 4: return launch_one<4, true>(p, blocks, st);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (lanes) {
    case 1: return launch_one<1, false>(p, blocks, st);
    case 2: return launch_one<2, false>(p, blocks, st);
    case 4: return launch_one<4, false>(p, blocks, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_k7(int lanes, bool radix4, const BatchParams &p, int64_t blocks,
                            cudaStream_t st) {
    if (radix4) {
        switch (lanes) {
        case 1: return launch_batch<1, true>(p, blocks, st);
        case 2: return launch_batch<2, true>(p, blocks, st);
        case 4: return launch_batch<4, true>(p, blocks, st);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (lanes) {
    case 1: return launch_batch<1, false>(p, blocks, st);
    case 2: return launch_batch<2, false>(p, blocks, st);
    case 4: return launch_batch<4, false>(p, blocks, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t batch_occupancy_k7(int lanes, bool radix4, int *blocks_per_sm) {
    if (radix4) {
        switch (lanes) {
        case 1: return occ<1, true>(blocks_per_sm);
        case 2: return occ<2, true>(blocks_per_sm);
        case 4: return occ<4, true>(blocks_per_sm);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (lanes) {
    case 1: return occ<1, false>(blocks_per_sm);
    case 2: return occ<2, false>(blocks_per_sm);
    case 4: return occ<4, false>(blocks_per_sm);
    default: return cudaErrorInvalidValue;
    }
}

bool geom_k7(int lanes, bool radix4, KernelGeom *g) {
    switch (lanes) {
    case 1:
        g->U = radix4 ? StreamCfg<7, 2, GENS_K7, 1, true>::U : StreamCfg<7, 2, GENS_K7, 1, false>::U;
        g->NW = radix4 ? StreamCfg<7, 2, GENS_K7, 1, true>::NW : StreamCfg<7, 2, GENS_K7, 1, false>::NW;
        return true;
    case 2:
        g->U = radix4 ? StreamCfg<7, 2, GENS_K7, 2, true>::U : StreamCfg<7, 2, GENS_K7, 2, false>::U;
        g->NW = radix4 ? StreamCfg<7, 2, GENS_K7, 2, true>::NW : StreamCfg<7, 2, GENS_K7, 2, false>::NW;
        return true;
    case 4:
        g->U = radix4 ? StreamCfg<7, 2, GENS_K7, 4, true>::U : StreamCfg<7, 2, GENS_K7, 4, false>::U;
        g->NW = radix4 ? StreamCfg<7, 2, GENS_K7, 4, true>::NW : StreamCfg<7, 2, GENS_K7, 4, false>::NW;
        return true;
    default: return false;
    }
}

cudaError_t launch_stream_f32_k7(int lanes, const StreamParams &p, int64_t blocks, cudaStream_t st) {
    switch (lanes) {
    case 2: stream_kernel_f32<7, 2, GENS_K7, 2, kThreads><<<(unsigned)blocks, kThreads, 0, st>>>(p); return cudaGetLastError();
    default: return cudaErrorInvalidValue;
    }
}

bool geom_f32_k7(int lanes, KernelGeom *g) {
    switch (lanes) {
    case 2: g->U = StreamCfgF32<7, 2, GENS_K7, 2>::U; g->NW = StreamCfgF32<7, 2, GENS_K7, 2>::NW; return true;
    default: return false;
    }
}

}  // namespace vd
