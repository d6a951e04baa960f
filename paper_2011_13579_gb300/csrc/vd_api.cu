// C ABI of the decoder: code objects, argument checks, scratch management and
// kernel dispatch.  See include/vd.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/vd.h"
#include "vd_code.h"
#include "vd_prep.cuh"
#include "vd_launch.h"

namespace {

thread_local std::string g_err;

vd_status fail(vd_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

vd_status cuda_fail(cudaError_t e, const char *what) {
    return fail(VD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

// ------------------------------------------------------------------ codes


namespace {

vd::CodeKind code_kind(int K, int beta, const uint32_t *g) {
    if (K == 7 && beta == 2 && g[0] == 0171 && g[1] == 0133) return vd::KIND_K7_R2;
    if (K == 9 && beta == 3 && g[0] == 0557 && g[1] == 0663 && g[2] == 0711) return vd::KIND_K9_R3;
    return vd::KIND_NONE;
}

vd_status check_gens(int K, int beta, const uint32_t *g) {
    if (K < 3 || K > 9) return fail(VD_EINVAL, "K=%d outside [3, 9]", K);
    if (beta < 2 || beta > 4) return fail(VD_EINVAL, "beta=%d outside [2, 4]", beta);
    if (!g) return fail(VD_EINVAL, "generator array is NULL");
    for (int b = 0; b < beta; ++b) {
        if (g[b] >= (1u << K)) return fail(VD_EINVAL, "generator %d (0%o) has more than K=%d bits", b, g[b], K);
        if (!(g[b] >> (K - 1) & 1u))
            return fail(VD_EINVAL, "generator %d (0%o) does not tap the current input (bit K-1)", b, g[b]);
    }
    return VD_OK;
}

}  // namespace

extern "C" int vd_code_supported(int K, int beta, const uint32_t *gens_octal) {
    if (!gens_octal || beta < 2 || beta > 4) return 0;
    return code_kind(K, beta, gens_octal) != vd::KIND_NONE;
}

extern "C" vd_status vd_code_create(vd_code **out, int K, int beta, const uint32_t *gens_octal,
                                    int rate_num, int rate_den, const uint8_t *puncture, int period) {
    if (!out) return fail(VD_EINVAL, "out is NULL");
    *out = nullptr;
    vd_status st = check_gens(K, beta, gens_octal);
    if (st != VD_OK) return st;
    vd_code c;
    memset(&c, 0, sizeof c);
    c.K = K;
    c.beta = beta;
    for (int b = 0; b < beta; ++b) c.gens[b] = gens_octal[b];
    if (puncture) {
        if (period < 1 || period > 8) return fail(VD_EINVAL, "puncture period %d outside [1, 8]", period);
        for (int ph = 0; ph < period; ++ph) {
            int col = 0;
            for (int b = 0; b < beta; ++b) {
                const uint8_t x = puncture[b * period + ph];
                if (x > 1) return fail(VD_EINVAL, "puncture entry (%d,%d) is not 0/1", b, ph);
                c.punct[b][ph] = x;
                col += x;
            }
            if (!col) return fail(VD_EINVAL, "puncture column %d transmits nothing", ph);
        }
        c.period = period;
    } else {
        c.period = 1;
        for (int b = 0; b < beta; ++b) c.punct[b][0] = 1;
    }
    c.kept_prefix[0] = 0;
    for (int ph = 0; ph < c.period; ++ph) {
        int col = 0;
        for (int b = 0; b < beta; ++b) col += c.punct[b][ph];
        c.kept_prefix[ph + 1] = c.kept_prefix[ph] + col;
    }
    c.kept_per_period = c.kept_prefix[c.period];
    c.punctured = c.kept_per_period != beta * c.period;
    // nominal rate = period / kept
    if (rate_num <= 0 || rate_den <= 0 ||
        (int64_t)rate_num * c.kept_per_period != (int64_t)rate_den * c.period)
        return fail(VD_EINVAL, "rate %d/%d does not match the pattern (%d/%d)", rate_num, rate_den,
                    c.period, c.kept_per_period);
    c.kind = code_kind(K, beta, c.gens);
    if (c.kind == vd::KIND_NONE)
        return fail(VD_EUNSUPPORTED, "no decode kernel for K=%d beta=%d with these generators", K, beta);
    vd_code *p = new (std::nothrow) vd_code(c);
    if (!p) return fail(VD_ENOMEM, "out of host memory");
    *out = p;
    return VD_OK;
}

extern "C" void vd_code_destroy(vd_code *code) { delete code; }

extern "C" int64_t vd_num_frames(int64_t n_info, int f) {
    if (n_info <= 0 || f <= 0) return 0;
    return (n_info + f - 1) / f;
}

extern "C" int64_t vd_num_kept(const vd_code *c, int64_t T) {
    if (!c || T < 0) return -1;
    return (T / c->period) * c->kept_per_period + c->kept_prefix[T % c->period];
}

// ---------------------------------------------------------------- scratch

namespace {

struct Scratch {
    void *ptr = nullptr;
    size_t bytes = 0;
};

std::mutex g_scratch_mu;
// (device, stream, slot) -> buffer; slot 0 = survivors, 1 = depunctured LLRs,
// 2 = the status word (stream 0), 3 = the persistent kernel's task counter,
// 4 / 5 = vd_decode_host's device copies of the LLRs / decoded words,
// 6 = vd_decode_radix's survivors
std::map<std::tuple<int, uintptr_t, int>, Scratch> g_scratch;

vd_status get_scratch(int slot, size_t bytes, cudaStream_t st, void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    Scratch &s = g_scratch[std::make_tuple(dev, (uintptr_t)st, slot)];
    if (s.bytes < bytes) {
        if (s.ptr) {
            // earlier launches on this stream may still read the old buffer
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
            cudaFree(s.ptr);
            s.ptr = nullptr;
            s.bytes = 0;
        }
        size_t want = bytes + bytes / 8;   // headroom against small growth steps
        e = cudaMalloc(&s.ptr, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s.ptr = nullptr;
            return fail(VD_ENOMEM, "cannot allocate %zu bytes of scratch: %s", want, cudaGetErrorString(e));
        }
        s.bytes = want;
    }
    *out = s.ptr;
    return VD_OK;
}

// Library-owned device status word (per device): kernels OR error bits into it.
vd_status device_status_word(cudaStream_t st, int **out) {
    void *p = nullptr;
    bool fresh = false;
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        Scratch &s = g_scratch[std::make_tuple(dev, (uintptr_t)0, 2)];
        if (!s.ptr) {
            e = cudaMalloc(&s.ptr, 256);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(VD_ENOMEM, "cannot allocate the device status word");
            }
            s.bytes = 256;
            fresh = true;
        }
        p = s.ptr;
    }
    if (fresh) {
        cudaError_t e = cudaMemset(p, 0, 256);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
    }
    (void)st;
    *out = (int *)p;
    return VD_OK;
}

// The library's status word of the current device, or NULL if no call has
// created it yet (then no kernel can have written it).
int *existing_status_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    auto it = g_scratch.find(std::make_tuple(dev, (uintptr_t)0, 2));
    return it == g_scratch.end() ? nullptr : (int *)it->second.ptr;
}

}  // namespace

extern "C" vd_status vd_sync(void *stream) {
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    // the no-allocation entry point's own status word first (it allocates nothing)
    const vd_status na = vd_internal_noalloc_status();
    if (na != VD_OK) return na;
    int *status = existing_status_word();
    if (!status) return VD_OK;
    int h = 0;
    e = cudaMemcpy(&h, status, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    if (h) {
        cudaMemset(status, 0, sizeof h);
        return fail(VD_EBOUNDS, "a device-side bounds check fired (status 0x%x)", h);
    }
    return VD_OK;
}

extern "C" vd_status vd_release_scratch(void) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    for (auto it = g_scratch.begin(); it != g_scratch.end();) {
        if (std::get<0>(it->first) == dev) {
            cudaFree(it->second.ptr);
            it = g_scratch.erase(it);
        } else {
            ++it;
        }
    }
    return VD_OK;
}

// ------------------------------------------------------- input pre-pass

namespace {

struct PrepParams {
    const uint8_t *src;       // kept values: int8, or 4-bit packed (two per byte)
    int64_t n_kept;           // number of kept values available
    int64_t T;                // stages to produce
    int beta, period, kept_per_period, llr_type;
    uint8_t punct[4][8];
    int kept_prefix[9];
    int8_t *dst;              // [T][beta]
};

// Expands the transmitted values of each stage to beta int8 LLRs, with 0 at
// erased positions (depuncturing) and 4-bit values sign-extended
// (vd_prep.cuh); a grid-stride loop over whole puncturing periods.
__global__ void prep_kernel(const PrepParams p) {
    vd::prep_expand(p.src, 0, p.n_kept, p.llr_type, p.T, p.beta, p.period, p.kept_per_period, p.punct, p.dst,
                    (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

}  // namespace

// ----------------------------------------------------------------- decode

namespace {

bool default_lanes(vd::CodeKind kind, int *lanes) {
    switch (kind) {
    case vd::KIND_K7_R2: *lanes = 1; return true;
    case vd::KIND_K9_R3: *lanes = 4; return true;
    default: return false;
    }
}

bool geometry(vd::CodeKind kind, int lanes, bool r4, vd::KernelGeom *g) {
    switch (kind) {
    case vd::KIND_K7_R2: return vd::geom_k7(lanes, r4, g);
    case vd::KIND_K9_R3: return vd::geom_k9(lanes, r4, g);
    default: return false;
    }
}

struct Plan {
    int lanes;
    bool r4;
    bool persistent;   // integer LLRs: the persistent kernel with interleaved traceback
    vd::KernelGeom geom;
    int64_t T, n_win, n_pairs, n_tasks, blocks;
    int32_t wpad_max;
    size_t surv_bytes;
};

// Streams with at least this many tasks per resident warp take the persistent
// form (measured on GB300: below one wave the one-pair-per-lane-group kernel
// is faster, from one wave up the persistent one, for K=7 and K=9).
constexpr int64_t kPersistentWaves = 1;

// Resident blocks per SM of the persistent stream kernel, per device and shape.
int persistent_blocks_per_sm(int K, int lanes, bool r4) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(dev, K, lanes, (int)r4);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int bps = 0;
    if (vd::stream_persistent_occupancy(K, lanes, r4, &bps) != cudaSuccess) {
        cudaGetLastError();
        bps = 0;
    }
    cache[key] = bps;
    return bps;
}

vd_status make_plan(const vd_code *c, int64_t n_info, int f, int v, int radix, uint32_t flags,
                    const vd_tune *tune, Plan *pl, bool f32 = false) {
    pl->r4 = radix == 4 && !f32;
    if (tune && (tune->form < 0 || tune->form > 2)) return fail(VD_EINVAL, "tune.form must be 0, 1 or 2");
    if (tune && tune->lanes > 0) {
        pl->lanes = tune->lanes;
    } else if (f32) {
        pl->lanes = c->kind == vd::KIND_K7_R2 ? 2 : 8;
    } else if (!default_lanes(c->kind, &pl->lanes)) {
        return fail(VD_EUNSUPPORTED, "no kernel for this code");
    }
    const bool have = f32 ? (c->kind == vd::KIND_K7_R2 ? vd::geom_f32_k7(pl->lanes, &pl->geom)
                                                       : vd::geom_f32_k9(pl->lanes, &pl->geom))
                          : geometry(c->kind, pl->lanes, pl->r4, &pl->geom);
    if (!have)
        return fail(VD_EUNSUPPORTED, "no kernel with %d lanes per frame pair (radix %d) for K=%d",
                    pl->lanes, radix, c->K);
    pl->T = n_info + ((flags & VD_TERMINATED) ? c->K - 1 : 0);
    pl->n_win = vd_num_frames(n_info, f);
    pl->n_pairs = (pl->n_win + 1) / 2;
    const int64_t wmax = std::min<int64_t>(pl->T, (int64_t)f + 2 * (int64_t)v);
    const int64_t wpad = ((wmax + pl->geom.U - 1) / pl->geom.U) * pl->geom.U;
    if (wpad > (1 << 30)) return fail(VD_EINVAL, "frame too long (%lld stages)", (long long)wmax);
    pl->wpad_max = (int32_t)wpad;
    const int64_t threads = pl->n_pairs * pl->lanes;
    pl->n_tasks = (pl->n_pairs + 32 / pl->lanes - 1) / (32 / pl->lanes);
    pl->persistent = false;
    if (!f32) {
        // Long streams (a task per resident warp or more): resident warps
        // pull tasks and hide each task's traceback behind the next task's
        // forward pass; each owns two survivor buffers.  Shorter streams are
        // less than one wave of warps, for which the one-pair-per-lane-group
        // kernel is faster.
        int n_sm = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        const int bps = persistent_blocks_per_sm(c->K, pl->lanes, pl->r4);
        const int64_t resident_warps = (int64_t)n_sm * bps * (vd::kThreads / 32);
        const int form = tune ? tune->form : 0;
        if (bps >= 1 && (form == 1 || (form == 0 && pl->n_tasks >= kPersistentWaves * resident_warps))) {
            pl->persistent = true;
            pl->blocks = (int64_t)n_sm * bps;
            pl->surv_bytes = 2u * (size_t)pl->blocks * vd::kThreads * (size_t)wpad * pl->geom.NW * 4u;
        }
    }
    if (!pl->persistent) {
        pl->blocks = (threads + vd::kThreads - 1) / vd::kThreads;
        pl->surv_bytes = (size_t)pl->blocks * vd::kThreads * (size_t)wpad * pl->geom.NW * 4u;
    }
    return VD_OK;
}

vd_status check_decode_args(const vd_code *c, const void *d_llr, int llr_type, int64_t n_info, int f,
                            int v, int radix, uint32_t flags, const uint32_t *d_out) {
    if (!c) return fail(VD_EINVAL, "code is NULL");
    if (n_info < 0) return fail(VD_EINVAL, "n_info < 0");
    if (f <= 0) return fail(VD_EINVAL, "f must be positive");
    if (v < 0) return fail(VD_EINVAL, "v must be >= 0");
    if (radix != 2 && radix != 4) return fail(VD_EINVAL, "radix must be 2 or 4");
    if (flags & ~(uint32_t)(VD_TERMINATED | VD_START_UNKNOWN))
        return fail(VD_EINVAL, "unknown flag bits 0x%x", flags);
    if (llr_type != VD_LLR_S8 && llr_type != VD_LLR_S4 && llr_type != VD_LLR_F16 && llr_type != VD_LLR_HARD)
        return fail(VD_EINVAL, "unknown llr_type %d", llr_type);
    if (n_info > 0 && (!d_llr || !d_out)) return fail(VD_EINVAL, "NULL device pointer");
    if (n_info > 0 && f < n_info && f % 32 != 0)
        return fail(VD_EINVAL, "f=%d must be a multiple of 32 when the stream has several frames", f);
    if (n_info > ((int64_t)1 << 40)) return fail(VD_EINVAL, "n_info too large");
    return VD_OK;
}

}  // namespace

extern "C" int64_t vd_scratch_bytes(const vd_code *c, int64_t n_info, int f, int v, int radix,
                                    const vd_tune *tune) {
    if (!c || n_info <= 0 || f <= 0 || v < 0) return 0;
    Plan pl;
    if (make_plan(c, n_info, f, v, radix, 0, tune, &pl) != VD_OK) return -1;
    int64_t extra = 0;
    if (c->punctured) extra = pl.T * c->beta;
    return (int64_t)pl.surv_bytes + extra;
}

extern "C" vd_status vd_decode(const vd_code *c, const void *d_llr, int llr_type, int64_t n_info,
                               int f, int v, int radix, uint32_t flags, uint32_t *d_out, int32_t *d_pm,
                               const vd_tune *tune, void *stream) {
    vd_status st = check_decode_args(c, d_llr, llr_type, n_info, f, v, radix, flags, d_out);
    if (st != VD_OK) return st;
    if (n_info == 0) return VD_OK;
    const bool f32 = llr_type == VD_LLR_F16;
    if (f32 && c->punctured) return fail(VD_EUNSUPPORTED, "fp16 LLRs of punctured codes are not supported");
    if (f32 && d_pm) return fail(VD_EUNSUPPORTED, "metric output is for integer LLRs only");
    cudaStream_t cs = (cudaStream_t)stream;
    Plan pl;
    st = make_plan(c, n_info, f, v, radix, flags, tune, &pl, f32);
    if (st != VD_OK) return st;

    const int8_t *llr = (const int8_t *)d_llr;
    if (!f32 && (c->punctured || llr_type == VD_LLR_S4 || llr_type == VD_LLR_HARD)) {
        void *buf = nullptr;
        st = get_scratch(1, (size_t)pl.T * c->beta, cs, &buf);
        if (st != VD_OK) return st;
        PrepParams pp;
        memset(&pp, 0, sizeof pp);
        pp.src = (const uint8_t *)d_llr;
        pp.n_kept = vd_num_kept(c, pl.T);
        pp.T = pl.T;
        pp.beta = c->beta;
        pp.period = c->period;
        pp.kept_per_period = c->kept_per_period;
        pp.llr_type = llr_type;
        memcpy(pp.punct, c->punct, sizeof pp.punct);
        memcpy(pp.kept_prefix, c->kept_prefix, sizeof pp.kept_prefix);
        pp.dst = (int8_t *)buf;
        const int tb = 256;
        const int64_t groups = (pl.T + c->period - 1) / c->period;
        const int64_t blocks = std::min<int64_t>((groups + tb - 1) / tb, 4096);
        prep_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), tb, 0, cs>>>(pp);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "input pre-pass launch");
        llr = (const int8_t *)buf;
    }

    void *surv = nullptr;
    st = get_scratch(0, pl.surv_bytes, cs, &surv);
    if (st != VD_OK) return st;

    vd::StreamParams p;
    p.llr = llr;
    p.llr_bytes = pl.T * c->beta;
    p.n_info = n_info;
    p.T = pl.T;
    p.f = f;
    p.v = v;
    p.n_win = pl.n_win;
    p.n_pairs = pl.n_pairs;
    p.flags = flags;
    p.wpad_max = pl.wpad_max;
    p.out = d_out;
    p.surv = (uint32_t *)surv;
    p.pm_out = d_pm;
    int *status = nullptr;
    st = device_status_word(cs, &status);
    if (st != VD_OK) return st;
    p.status = status;
    p.counter = nullptr;
    p.n_tasks = pl.n_tasks;
    if (pl.blocks > 0x7FFFFFFF) return fail(VD_EINVAL, "stream too long for one launch");
    cudaError_t e;
    p.llr_bytes = pl.T * c->beta * (f32 ? 2 : 1);
    if (pl.persistent) {
        void *ctr = nullptr;
        st = get_scratch(3, 256, cs, &ctr);
        if (st != VD_OK) return st;
        e = cudaMemsetAsync(ctr, 0, sizeof(int), cs);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (task counter)");
        p.counter = (int *)ctr;
        e = vd::launch_stream_persistent(c->K, pl.lanes, pl.r4, p, pl.blocks, cs);
        if (e != cudaSuccess) return cuda_fail(e, "decode launch");
        return VD_OK;
    }
    switch (c->kind) {
    case vd::KIND_K7_R2:
        e = f32 ? vd::launch_stream_f32_k7(pl.lanes, p, pl.blocks, cs)
                : vd::launch_stream_k7(pl.lanes, pl.r4, p, pl.blocks, cs);
        break;
    case vd::KIND_K9_R3:
        e = f32 ? vd::launch_stream_f32_k9(pl.lanes, p, pl.blocks, cs)
                : vd::launch_stream_k9(pl.lanes, pl.r4, p, pl.blocks, cs);
        break;
    default: return fail(VD_EUNSUPPORTED, "no kernel for this code");
    }
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    return VD_OK;
}

extern "C" vd_status vd_decode_each(const vd_code *const *codes, int n_codes, const vd_packet *packets,
                                    int64_t n_packets, const void *d_llr_arena, uint32_t *d_out_arena, int radix,
                                    void *const *streams, int n_streams) {
    if (!codes || n_codes <= 0 || (n_packets > 0 && !packets) || n_packets < 0)
        return fail(VD_EINVAL, "vd_decode_each: bad code or packet arrays");
    if (!streams || n_streams <= 0) return fail(VD_EINVAL, "vd_decode_each: no streams");
    for (int64_t i = 0; i < n_packets; ++i) {
        const vd_packet &p = packets[i];
        if (p.code_id < 0 || p.code_id >= n_codes || !codes[p.code_id])
            return fail(VD_EINVAL, "vd_decode_each: packet %lld has a bad code_id", (long long)i);
        if (p.f <= 0) return fail(VD_EINVAL, "vd_decode_each: packet %lld needs f > 0", (long long)i);
        int64_t byte_off = p.llr_offset;
        if (p.llr_type == VD_LLR_S4) {
            if (p.llr_offset & 1) return fail(VD_EINVAL, "vd_decode_each: 4-bit packet %lld not on a byte", (long long)i);
            byte_off = p.llr_offset / 2;
        } else if (p.llr_type == VD_LLR_HARD) {
            if (p.llr_offset & 7) return fail(VD_EINVAL, "vd_decode_each: hard packet %lld not on a byte", (long long)i);
            byte_off = p.llr_offset / 8;
        } else if (p.llr_type == VD_LLR_F16) {
            byte_off = p.llr_offset * 2;
        }
        const vd_status st = vd_decode(codes[p.code_id], (const uint8_t *)d_llr_arena + byte_off, p.llr_type,
                                       p.n_info, p.f, p.v, radix, p.flags, d_out_arena + p.out_word_offset,
                                       nullptr, nullptr, streams[i % n_streams]);
        if (st != VD_OK) return st;
    }
    return VD_OK;
}

// ------------------------------------------------ decode from host memory

namespace {

constexpr int kHostComp = 2;   // decode streams of vd_decode_host

// Copy and decode streams, events and the two single-stream batch plans of
// vd_decode_host, per (device, caller stream), rebuilt when the stream
// configuration changes.
struct HostPipe {
    cudaStream_t in = nullptr, out = nullptr, comp[kHostComp] = {nullptr, nullptr};
    std::vector<cudaEvent_t> ev;
    vd_batch_plan *plan[kHostComp] = {nullptr, nullptr};
    const vd_code *code = nullptr;
    int64_t n_info = -1;
    int f = 0, v = 0, radix = 0;
    uint32_t flags = 0;
};
std::mutex g_pipe_mu;
std::map<std::pair<int, uintptr_t>, HostPipe> g_pipes;

vd_status host_pipe(const vd_code *c, int64_t n_info, int f, int v, int radix, uint32_t flags, cudaStream_t cs,
                    size_t n_events, HostPipe **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    HostPipe &hp = g_pipes[std::make_pair(dev, (uintptr_t)cs)];
    if (!hp.in) {
        if ((e = cudaStreamCreateWithFlags(&hp.in, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&hp.out, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&hp.comp[0], cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&hp.comp[1], cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreate (host pipeline)");
    }
    while (hp.ev.size() < n_events) {
        cudaEvent_t ev;
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate (host pipeline)");
        hp.ev.push_back(ev);
    }
    if (hp.code != c || hp.n_info != n_info || hp.f != f || hp.v != v || hp.radix != radix || hp.flags != flags) {
        for (auto &pl : hp.plan) {
            if (pl) {
                cudaDeviceSynchronize();
                vd_batch_plan_destroy(pl);
                pl = nullptr;
            }
        }
        // one packet: a whole stream at offset 0 of the arenas given at launch
        vd_packet pk;
        memset(&pk, 0, sizeof pk);
        pk.code_id = 0;
        pk.llr_type = VD_LLR_S8;
        pk.n_info = n_info;
        pk.flags = flags;
        pk.f = f;
        pk.v = v;
        vd_tune tune;
        memset(&tune, 0, sizeof tune);
        tune.radix = radix;
        if (!default_lanes(c->kind, &tune.lanes)) return fail(VD_EUNSUPPORTED, "no kernel for this code");
        const vd_code *codes[1] = {c};
        for (int k = 0; k < kHostComp; ++k) {
            const vd_status st = vd_batch_plan_create(&hp.plan[k], codes, 1, &pk, 1, &tune, hp.comp[k]);
            if (st != VD_OK) return st;
        }
        hp.code = c;
        hp.n_info = n_info;
        hp.f = f;
        hp.v = v;
        hp.radix = radix;
        hp.flags = flags;
    }
    *out = &hp;
    return VD_OK;
}

}  // namespace

extern "C" vd_status vd_decode_host(const vd_code *c, int n_streams, const void *const *h_llr, int llr_type,
                                    int64_t n_info, int f, int v, int radix, uint32_t flags,
                                    uint32_t *const *h_out, void *stream) {
    if (n_streams < 1 || !h_llr || !h_out) return fail(VD_EINVAL, "vd_decode_host: bad stream arrays");
    for (int i = 0; i < n_streams; ++i)
        if (!h_llr[i] || !h_out[i]) return fail(VD_EINVAL, "vd_decode_host: NULL host buffer %d", i);
    vd_status st = check_decode_args(c, h_llr[0], llr_type, n_info, f, v, radix, flags, h_out[0]);
    if (st != VD_OK) return st;
    if (llr_type != VD_LLR_S8 || c->punctured)
        return fail(VD_EUNSUPPORTED, "vd_decode_host: unpunctured int8 LLRs only");
    if (n_info == 0) return VD_OK;
    const cudaStream_t cs = (cudaStream_t)stream;
    const int64_t T = n_info + ((flags & VD_TERMINATED) ? c->K - 1 : 0);
    const size_t llr_bytes = (size_t)T * c->beta, llr_stride = (llr_bytes + 255) & ~(size_t)255;
    const int64_t n_words = (n_info + 31) / 32;
    const size_t out_stride = ((size_t)n_words * 4 + 255) & ~(size_t)255;

    std::lock_guard<std::mutex> lk(g_pipe_mu);
    HostPipe *hp = nullptr;
    st = host_pipe(c, n_info, f, v, radix, flags, cs, 2 * (size_t)n_streams + 2, &hp);
    if (st != VD_OK) return st;
    void *d_llr = nullptr, *d_out = nullptr;
    if ((st = get_scratch(4, llr_stride * n_streams, cs, &d_llr)) != VD_OK) return st;
    if ((st = get_scratch(5, out_stride * n_streams, cs, &d_out)) != VD_OK) return st;
    cudaError_t e;
    // everything below starts after earlier work on the caller's stream (which
    // may still read the device copies)
    size_t evi = 0;
    cudaEvent_t entry = hp->ev[evi++];
    if ((e = cudaEventRecord(entry, cs)) != cudaSuccess) return cuda_fail(e, "vd_decode_host: ordering");
    for (cudaStream_t x : {hp->in, hp->out, hp->comp[0], hp->comp[1]})
        if ((e = cudaStreamWaitEvent(x, entry, 0)) != cudaSuccess) return cuda_fail(e, "vd_decode_host: ordering");
    // stream i: upload (copy stream), decode (decode stream i mod 2) once its
    // bytes are on the device, download its words (download stream)
    for (int i = 0; i < n_streams; ++i) {
        uint8_t *dllr = (uint8_t *)d_llr + llr_stride * i;
        uint32_t *dout = (uint32_t *)((uint8_t *)d_out + out_stride * i);
        const int k = i % kHostComp;
        cudaEvent_t up = hp->ev[evi++], dec = hp->ev[evi++];
        if ((e = cudaMemcpyAsync(dllr, h_llr[i], llr_bytes, cudaMemcpyHostToDevice, hp->in)) != cudaSuccess ||
            (e = cudaEventRecord(up, hp->in)) != cudaSuccess || (e = cudaStreamWaitEvent(hp->comp[k], up, 0)) != cudaSuccess)
            return cuda_fail(e, "vd_decode_host: upload");
        if ((st = vd_batch_plan_launch(hp->plan[k], dllr, dout, hp->comp[k])) != VD_OK) return st;
        if ((e = cudaEventRecord(dec, hp->comp[k])) != cudaSuccess || (e = cudaStreamWaitEvent(hp->out, dec, 0)) != cudaSuccess ||
            (e = cudaMemcpyAsync(h_out[i], dout, (size_t)n_words * 4, cudaMemcpyDeviceToHost, hp->out)) != cudaSuccess)
            return cuda_fail(e, "vd_decode_host: download");
    }
    cudaEvent_t done = hp->ev[evi++];
    if ((e = cudaEventRecord(done, hp->out)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, done, 0)) != cudaSuccess)
        return cuda_fail(e, "vd_decode_host: ordering");
    return VD_OK;
}

extern "C" vd_status vd_get_tune(const vd_code *c, int llr_type, int f, int v, int radix, vd_tune *out) {
    if (!c || !out) return fail(VD_EINVAL, "NULL argument");
    if (f <= 0 || v < 0) return fail(VD_EINVAL, "f must be positive and v >= 0");
    if (radix != 2 && radix != 4) return fail(VD_EINVAL, "radix must be 2 or 4");
    if (llr_type != VD_LLR_S8 && llr_type != VD_LLR_S4 && llr_type != VD_LLR_F16 && llr_type != VD_LLR_HARD)
        return fail(VD_EINVAL, "unknown llr_type %d", llr_type);
    memset(out, 0, sizeof *out);
    const bool f32 = llr_type == VD_LLR_F16;
    int lanes = 0;
    if (f32) lanes = c->kind == vd::KIND_K7_R2 ? 2 : 8;
    else if (!default_lanes(c->kind, &lanes)) return fail(VD_EUNSUPPORTED, "no kernel for this code");
    out->f = f;
    out->v = v;
    out->radix = f32 ? 2 : radix;   // the fp32 form runs radix-2 steps
    out->lanes = lanes;
    out->threads = vd::kThreads;
    return VD_OK;
}

vd_status vd_internal_scratch(int slot, size_t bytes, cudaStream_t stream, void **out) {
    return get_scratch(slot, bytes, stream, out);
}

int *vd_internal_status_word(void) {
    int *w = nullptr;
    return device_status_word(nullptr, &w) == VD_OK ? w : nullptr;
}

extern "C" const char *vd_last_error(void) { return g_err.c_str(); }

void vd_internal_set_error(const char *msg) { g_err = msg; }

extern "C" int vd_version(void) { return 100; }
