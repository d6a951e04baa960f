// Internal definition of the opaque vd_code object (shared by the C-ABI sources).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/vd.h"
#include "vd_launch.h"

struct vd_code {
    int K, beta;
    uint32_t gens[4];
    int period;
    uint8_t punct[4][8];
    int kept_per_period;
    int kept_prefix[9];      // kept values before phase p within a period
    bool punctured;
    vd::CodeKind kind;
};

// Sets the calling thread's message returned by vd_last_error().
void vd_internal_set_error(const char *msg);

// Reads and clears the device status word of vd_decode_noalloc on the current
// device (VD_EBOUNDS if a kernel set it); called by vd_sync.
vd_status vd_internal_noalloc_status(void);

// The library's device status word of the current device (created on first
// use; NULL if it cannot be allocated), for kernels outside vd_api.cu.
int *vd_internal_status_word(void);

// A buffer of at least `bytes` from the library's scratch pool of the current
// device and `stream` (slots 0-5 belong to vd_api.cu; 6 = vd_decode_radix).
vd_status vd_internal_scratch(int slot, size_t bytes, cudaStream_t stream, void **out);

namespace vd {

// Input pre-pass shared by batches and the server: expands the transmitted
// values of each listed packet to int8 [T][beta] (0 at erased positions).
constexpr int kMaxBatchCodes = 16;

struct PrepCode {
    int beta, period, kept_per_period, pad;
    uint8_t punct[4][8];
    int kept_prefix[9];
};

struct PrepJob {
    const uint8_t *src;  // NULL: the launch's source arena; else the packet's own values (device)
    int64_t src_off;     // first kept value of the packet in the source (values)
    int64_t dst_off;     // byte offset of the packet's [T][beta] int8 in the destination
    int64_t T;
    int32_t code_slot;
    int32_t llr_type;
};

struct PrepBatchParams {
    const uint8_t *src;
    int8_t *dst;
    const PrepJob *jobs;
    int64_t n_jobs;
    PrepCode codes[kMaxBatchCodes];
};

cudaError_t launch_prep_batch(const PrepBatchParams &p, cudaStream_t st);
void fill_prep_code(const vd_code *c, PrepCode *pc);

}  // namespace vd
