// Radix dispatch and host-side geometry of the integer kernels (no kernel
// code is instantiated here).
#include "vd_variants.cuh"

namespace vd {

cudaError_t launch_stream_k7(int lanes, bool radix4, const StreamParams &p, int64_t blocks,
                             cudaStream_t st) {
    return radix4 ? launch_stream_k7_r4(lanes, p, blocks, st) : launch_stream_k7_r2(lanes, p, blocks, st);
}
cudaError_t launch_stream_k9(int lanes, bool radix4, const StreamParams &p, int64_t blocks,
                             cudaStream_t st) {
    return radix4 ? launch_stream_k9_r4(lanes, p, blocks, st) : launch_stream_k9_r2(lanes, p, blocks, st);
}
cudaError_t launch_batch_k7(int lanes, bool radix4, const BatchParams &p, int64_t blocks,
                            cudaStream_t st) {
    return radix4 ? launch_batch_k7_r4(lanes, p, blocks, st) : launch_batch_k7_r2(lanes, p, blocks, st);
}
cudaError_t launch_batch_k9(int lanes, bool radix4, const BatchParams &p, int64_t blocks,
                            cudaStream_t st) {
    return radix4 ? launch_batch_k9_r4(lanes, p, blocks, st) : launch_batch_k9_r2(lanes, p, blocks, st);
}
cudaError_t batch_occupancy_k7(int lanes, bool radix4, int *blocks_per_sm) {
    return radix4 ? occupancy_k7_r4(lanes, blocks_per_sm) : occupancy_k7_r2(lanes, blocks_per_sm);
}
cudaError_t batch_occupancy_k9(int lanes, bool radix4, int *blocks_per_sm) {
    return radix4 ? occupancy_k9_r4(lanes, blocks_per_sm) : occupancy_k9_r2(lanes, blocks_per_sm);
}

template <int K, int BETA, uint64_t GENS, int... Ls>
static bool geom_of(int lanes, bool radix4, KernelGeom *g) {
    bool ok = false;
    (void)((lanes == Ls && ((g->U = radix4 ? StreamCfg<K, BETA, GENS, Ls, true>::U
                                           : StreamCfg<K, BETA, GENS, Ls, false>::U),
                            (g->NW = radix4 ? StreamCfg<K, BETA, GENS, Ls, true>::NW
                                            : StreamCfg<K, BETA, GENS, Ls, false>::NW),
                            (ok = true))) || ...);
    return ok;
}

bool geom_k7(int lanes, bool radix4, KernelGeom *g) { return geom_of<7, 2, GENS_K7, 1, 2, 4>(lanes, radix4, g); }
bool geom_k9(int lanes, bool radix4, KernelGeom *g) { return geom_of<9, 3, GENS_K9, 4, 8>(lanes, radix4, g); }

}  // namespace vd
