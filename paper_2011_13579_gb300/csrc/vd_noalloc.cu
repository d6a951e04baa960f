// vd_decode_noalloc: the stream decode of vd_decode with its survivor scratch
// in a fixed, file-scope device array instead of memory the library
// allocates at run time.
//
// Who needs it: a caller that must not allocate device memory once it is
// running — for example a real-time receiver thread whose latency budget
// cannot absorb cudaMalloc (which can block and synchronise the whole
// device), an application whose device memory is reserved up front by
// another allocator or memory budget, or a process that must not grow its
// footprint after start-up.  This entry point makes no allocation of any
// kind: no cudaMalloc, no cudaFree, no allocating library call.  The
// caller still passes the input and output buffers.
//
// What it costs: the array below occupies kNoallocScratchBytes of device
// memory on every GPU where the library's device code is loaded, until the
// process exits.  Requests whose scratch would not fit are rejected.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/vd.h"
#include "vd_code.h"
#include "vd_launch.h"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)32 << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

// Survivor scratch shared by every call on a device; contents persist between
// calls and nothing in it needs to start at zero (every word the traceback
// reads is written earlier in the same launch).
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoallocScratchBytes / 4];
// Device status word of these launches: a kernel ORs bit 0 into it if it
// refuses a frame pair that would overrun the scratch.  Zero at load; read
// and cleared by vd_sync (vd_internal_noalloc_status), never by a decode
// call, so an error is reported even when several calls ran before it.
static __device__ __align__(256) int g_noalloc_status[1];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices];
void *g_status_addr[kMaxDevices];

vd_status fail(vd_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    vd_internal_set_error(buf);   // readable through vd_last_error()
    return st;
}

// Once per device, with that device current: the device addresses of the
// arrays (in host code their names are host-side stand-ins, not device
// addresses, so a kernel must never be given them directly).
vd_status device_arrays(void **scratch, int **status) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(VD_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(VD_EUNSUPPORTED, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *a = nullptr, *b = nullptr;
        e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(VD_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        e = cudaGetSymbolAddress(&b, g_noalloc_status);
        if (e != cudaSuccess)
            return fail(VD_ECUDA, "cudaGetSymbolAddress(status): %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = a;
        g_status_addr[dev] = b;
    }
    *scratch = g_scratch_addr[dev];
    *status = (int *)g_status_addr[dev];
    return VD_OK;
}

}  // namespace

// Reads and clears this device's noalloc status word, if a noalloc call has
// set up this device (otherwise no kernel can have written it).  Called by
// vd_sync after it has waited for the stream; no allocation.
vd_status vd_internal_noalloc_status(void) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(VD_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return VD_OK;
    void *addr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        addr = g_status_addr[dev];
    }
    if (!addr) return VD_OK;
    int h = 0;
    e = cudaMemcpy(&h, addr, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(VD_ECUDA, "cudaMemcpy (noalloc status): %s", cudaGetErrorString(e));
    if (h) {
        e = cudaMemset(addr, 0, sizeof h);
        if (e != cudaSuccess) return fail(VD_ECUDA, "cudaMemset (noalloc status): %s", cudaGetErrorString(e));
        return fail(VD_EBOUNDS, "a vd_decode_noalloc kernel refused a frame pair that would overrun "
                                "its scratch (status 0x%x); its outputs were not written", h);
    }
    return VD_OK;
}

extern "C" int64_t vd_noalloc_scratch_limit(void) { return (int64_t)kNoallocScratchBytes; }

extern "C" vd_status vd_decode_noalloc(const vd_code *c, const void *d_llr, int64_t n_info, int f,
                                       int v, int radix, uint32_t flags, uint32_t *d_out,
                                       void *stream) {
    if (!c) return fail(VD_EINVAL, "code is NULL");
    if (n_info < 0) return fail(VD_EINVAL, "n_info < 0");
    if (f <= 0 || v < 0) return fail(VD_EINVAL, "f must be positive and v >= 0");
    if (radix != 2 && radix != 4) return fail(VD_EINVAL, "radix must be 2 or 4");
    if (flags & ~(uint32_t)(VD_TERMINATED | VD_START_UNKNOWN))
        return fail(VD_EINVAL, "unknown flag bits 0x%x", flags);
    if (n_info == 0) {
        // a zero-length call only sets the device up (module load, symbol lookup)
        void *scratch = nullptr;
        int *status = nullptr;
        return device_arrays(&scratch, &status);
    }
    if (!d_llr || !d_out) return fail(VD_EINVAL, "NULL device pointer");
    if (f < n_info && f % 32 != 0)
        return fail(VD_EINVAL, "f=%d must be a multiple of 32 when the stream has several frames", f);
    if (n_info > ((int64_t)1 << 40)) return fail(VD_EINVAL, "n_info too large");
    if (c->punctured)
        return fail(VD_EUNSUPPORTED, "vd_decode_noalloc takes unpunctured int8 LLRs only");

    int lanes = 0;
    vd::KernelGeom g;
    bool ok = false;
    if (c->kind == vd::KIND_K7_R2) { lanes = 1; ok = vd::geom_k7(lanes, radix == 4, &g); }
    if (c->kind == vd::KIND_K9_R3) { lanes = 4; ok = vd::geom_k9(lanes, radix == 4, &g); }
    if (!ok) return fail(VD_EUNSUPPORTED, "no kernel for this code");

    const int64_t T = n_info + ((flags & VD_TERMINATED) ? c->K - 1 : 0);
    const int64_t n_win = (n_info + f - 1) / f;
    const int64_t n_pairs = (n_win + 1) / 2;
    const int64_t wmax = T < (int64_t)f + 2 * (int64_t)v ? T : (int64_t)f + 2 * (int64_t)v;
    const int64_t wpad = ((wmax + g.U - 1) / g.U) * g.U;
    const int64_t blocks = (n_pairs * lanes + vd::kThreads - 1) / vd::kThreads;
    const double need = (double)blocks * vd::kThreads * (double)wpad * g.NW * 4.0;
    if (need > (double)kNoallocScratchBytes)
        return fail(VD_EINVAL,
                    "stream needs %.0f bytes of survivor scratch; vd_decode_noalloc has %zu "
                    "(use vd_decode, or shorter streams)", need, kNoallocScratchBytes);

    void *scratch = nullptr;
    int *status = nullptr;
    vd_status st = device_arrays(&scratch, &status);
    if (st != VD_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e;

    vd::StreamParams p;
    p.llr = (const int8_t *)d_llr;
    p.llr_bytes = T * c->beta;
    p.n_info = n_info;
    p.T = T;
    p.f = f;
    p.v = v;
    p.n_win = n_win;
    p.n_pairs = n_pairs;
    p.flags = flags;
    p.wpad_max = (int32_t)wpad;
    p.out = d_out;
    p.surv = (uint32_t *)scratch;
    p.pm_out = nullptr;
    p.status = status;
    p.counter = nullptr;   // the non-persistent kernel takes no task counter
    p.n_tasks = 0;
    e = (c->kind == vd::KIND_K7_R2) ? vd::launch_stream_k7(lanes, radix == 4, p, blocks, cs)
                                    : vd::launch_stream_k9(lanes, radix == 4, p, blocks, cs);
    if (e != cudaSuccess) return fail(VD_ECUDA, "decode launch: %s", cudaGetErrorString(e));
    return VD_OK;
}
