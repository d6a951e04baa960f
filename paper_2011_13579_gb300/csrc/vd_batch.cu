// Batched decode of many packets in one persistent launch per code kind:
// plan construction (argument checks, frame-length tuning, work list),
// the input pre-pass (depuncturing, 4-bit unpacking), launches and CUDA-graph
// replay.  See include/vd.h (vd_batch_plan_*, vd_decode_batch).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <functional>
#include <queue>
#include <vector>

#include "../../include/vd.h"
#include "vd_code.h"
#include "vd_launch.h"
#include "vd_prep.cuh"

namespace {

vd_status fail(vd_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    vd_internal_set_error(buf);
    return st;
}

vd_status cuda_fail(cudaError_t e, const char *what) {
    return fail(VD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

using vd::kMaxBatchCodes;
using vd::PrepBatchParams;
using vd::PrepCode;
using vd::PrepJob;

// One block per packet: expand its transmitted values to beta int8 LLRs per
// stage, 0 at erased positions (vd_prep.cuh).
__global__ void prep_batch_kernel(const PrepBatchParams p) {
    const int64_t j = blockIdx.x;
    if (j >= p.n_jobs) return;
    const PrepJob jb = p.jobs[j];
    const PrepCode &c = p.codes[jb.code_slot];
    // the packet's last kept value bounds every read (steps past T read nothing)
    const int64_t kept_end = jb.src_off + (jb.T / c.period) * c.kept_per_period + c.kept_prefix[jb.T % c.period];
    vd::prep_expand(jb.src ? jb.src : p.src, jb.src_off, kept_end, jb.llr_type, jb.T, c.beta, c.period,
                    c.kept_per_period, c.punct, p.dst + jb.dst_off, threadIdx.x, blockDim.x);
}

// ----------------------------------------------------------------- tuner

int default_v(int K) { return K >= 9 ? 64 : 7 * (K - 1); }

int default_lanes(vd::CodeKind kind) { return kind == vd::KIND_K9_R3 ? 4 : 1; }

bool kind_geom(vd::CodeKind kind, int lanes, bool r4, vd::KernelGeom *g) {
    return kind == vd::KIND_K7_R2 ? vd::geom_k7(lanes, r4, g) : vd::geom_k9(lanes, r4, g);
}

int64_t frame_len(int64_t s, int64_t n_info, int64_t T, int64_t f, int64_t v) {
    const vd::Frame w = vd::frame_of(s, n_info, T, f, v, 0);
    return w.b - w.a;
}

// Predicted makespan (in padded stages) of one persistent launch: frames sorted
// by length, paired, grouped into warp tasks of ppw pairs, longest task first
// onto `slots` resident warps.
double predict_makespan(std::vector<int64_t> wpads, int ppw, int64_t slots) {
    if (wpads.empty()) return 0.0;
    std::sort(wpads.begin(), wpads.end(), std::greater<int64_t>());
    const int64_t per_task = 2 * (int64_t)ppw;
    std::priority_queue<double, std::vector<double>, std::greater<double>> q;
    for (int64_t i = 0; i < std::max<int64_t>(1, slots); ++i) q.push(0.0);
    for (size_t i = 0; i < wpads.size(); i += (size_t)per_task) {
        const double cost = (double)wpads[i];
        const double t = q.top();
        q.pop();
        q.push(t + cost);
    }
    double mk = 0.0;
    while (!q.empty()) { mk = std::max(mk, q.top()); q.pop(); }
    return mk;
}

}  // namespace

// ------------------------------------------------------------------- plan

struct vd_batch_group {
    vd::CodeKind kind;
    int K, lanes;
    bool r4;
    vd::KernelGeom geom;
    int64_t n_pairs, n_tasks;
    int32_t wpad_cap;
    int64_t blocks;
    int32_t threads;      // block size
    vd::PacketDesc *d_pk;
    vd::PairRef *d_pairs;
    uint32_t *d_surv;
    size_t surv_bytes;
    uint32_t *d_surv2;    // second scratch of chained launches (allocated by the first one)
};

struct vd_batch_plan {
    int device;
    int64_t n_packets;
    std::vector<int32_t> f, v;             // chosen per packet
    std::vector<vd_batch_group> groups;
    PrepBatchParams prep;                   // pointers filled at launch
    PrepJob *d_jobs;
    int64_t n_jobs;
    int8_t *d_llr_int;
    size_t llr_int_bytes;
    int *d_counters;                        // one per group
    int *d_status;
    // CUDA graph of the launch sequence for (llr arena, out arena)
    cudaGraphExec_t graph;
    const void *graph_llr;
    uint32_t *graph_out;
    int64_t frames;
    int last_parity;      // scratch and counters of the last launch: 0 (d_surv, counters + 0) or 1
};

namespace {

void free_plan(vd_batch_plan *pl) {
    if (!pl) return;
    for (auto &g : pl->groups) {
        cudaFree(g.d_pk);
        cudaFree(g.d_pairs);
        cudaFree(g.d_surv);
        cudaFree(g.d_surv2);
    }
    cudaFree(pl->d_jobs);
    cudaFree(pl->d_llr_int);
    cudaFree(pl->d_counters);
    cudaFree(pl->d_status);
    if (pl->graph) cudaGraphExecDestroy(pl->graph);
    delete pl;
}

template <typename T>
vd_status upload(T **dst, const std::vector<T> &src, cudaStream_t st) {
    *dst = nullptr;
    if (src.empty()) return VD_OK;
    cudaError_t e = cudaMalloc((void **)dst, src.size() * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(VD_ENOMEM, "cannot allocate %zu bytes for the batch plan", src.size() * sizeof(T));
    }
    e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (plan upload)");
    return VD_OK;
}

// Kernel shape of a group: geometry, resident blocks and scratch for
// (lanes, radix); the pairs and descriptors do not depend on it.
bool shape_group(vd_batch_group &g, int lanes, bool r4, int n_sm) {
    g.lanes = lanes;
    g.r4 = r4;
    g.threads = vd::kThreads;
    if (!kind_geom(g.kind, lanes, r4, &g.geom)) return false;
    int bps = 0;
    const cudaError_t e = g.kind == vd::KIND_K7_R2 ? vd::batch_occupancy_k7(lanes, r4, &bps)
                                                   : vd::batch_occupancy_k9(lanes, r4, &bps);
    if (e != cudaSuccess || bps < 1) { cudaGetLastError(); return false; }
    const int ppw = 32 / lanes;
    g.n_tasks = (g.n_pairs + ppw - 1) / ppw;
    const int64_t tasks_blocks = (g.n_tasks * 32 + g.threads - 1) / g.threads;
    g.blocks = std::max<int64_t>(1, std::min<int64_t>((int64_t)n_sm * bps, tasks_blocks));
    // two survivor buffers per resident warp: one being written, one being traced back
    g.surv_bytes = 2u * (size_t)g.blocks * g.threads * (size_t)g.wpad_cap * g.geom.NW * 4u;
    return true;
}

vd_status launch_group(const vd_batch_group &g, const int8_t *llr_user, const int8_t *llr_int, uint32_t *out,
                       int *counter, int *status, cudaStream_t cs, int parity = 0, bool chained = false) {
    vd::BatchParams p;
    p.pk = g.d_pk;
    p.pairs = g.d_pairs;
    p.n_pairs = g.n_pairs;
    p.n_tasks = g.n_tasks;
    p.llr_user = llr_user;
    p.llr_int = llr_int;
    p.out = out;
    p.counter = counter;
    p.surv = parity ? g.d_surv2 : g.d_surv;
    p.wpad_cap = g.wpad_cap;
    p.status = status;
    p.chained = chained ? 1 : 0;
    const cudaError_t e = g.kind == vd::KIND_K7_R2 ? vd::launch_batch_k7(g.lanes, g.r4, p, g.blocks, cs)
                                                   : vd::launch_batch_k9(g.lanes, g.r4, p, g.blocks, cs);
    return e == cudaSuccess ? VD_OK : cuda_fail(e, "batch launch");
}

// Measured choice of radix and lanes per code kind: every candidate shape
// runs the plan's own work list twice on zero LLRs (the kernels' control flow
// and memory traffic do not depend on the values), and the fastest stays.
vd_status autotune_shapes(vd_batch_plan *pl, const vd_code *const *codes, const vd_packet *packets,
                          int64_t n_packets, bool tune_radix, bool tune_lanes, int n_sm, cudaStream_t cs) {
    int64_t user_bytes = 16, out_words = 1;
    for (int64_t i = 0; i < n_packets; ++i) {
        const vd_packet &p = packets[i];
        const vd_code *c = codes[p.code_id];
        const int64_t T = p.n_info + ((p.flags & VD_TERMINATED) ? c->K - 1 : 0);
        if (!c->punctured && p.llr_type == VD_LLR_S8) user_bytes = std::max(user_bytes, p.llr_offset + T * c->beta);
        out_words = std::max(out_words, p.out_word_offset + (p.n_info + 31) / 32);
    }
    int8_t *d_user = nullptr;
    uint32_t *d_out = nullptr;
    uint32_t *d_surv = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    vd_status st = VD_OK;
    auto cleanup = [&] {
        cudaFree(d_user);
        cudaFree(d_out);
        cudaFree(d_surv);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc((void **)&d_user, (size_t)user_bytes) != cudaSuccess ||
        cudaMalloc((void **)&d_out, (size_t)out_words * 4u) != cudaSuccess ||
        cudaMemsetAsync(d_user, 0, (size_t)user_bytes, cs) != cudaSuccess ||
        (pl->d_llr_int && cudaMemsetAsync(pl->d_llr_int, 0, pl->llr_int_bytes, cs) != cudaSuccess) ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(VD_ENOMEM, "cannot allocate the autotuner's scratch");
    }
    size_t surv_cap = 0;
    for (size_t gi = 0; gi < pl->groups.size(); ++gi) {
        vd_batch_group &g = pl->groups[gi];
        struct Shape { int lanes; bool r4; };
        std::vector<Shape> cands;
        const int lane_opts[2] = {g.kind == vd::KIND_K7_R2 ? 1 : 4, g.kind == vd::KIND_K7_R2 ? 2 : 8};
        for (int L : lane_opts)
            for (bool r4 : {false, true})
                if ((tune_lanes || L == g.lanes) && (tune_radix || r4 == g.r4)) cands.push_back({L, r4});
        float best_ms = 1e30f;
        Shape best = {g.lanes, g.r4};
        for (const Shape &sh : cands) {
            vd_batch_group c = g;
            if (!shape_group(c, sh.lanes, sh.r4, n_sm)) continue;
            if (c.surv_bytes > surv_cap) {
                cudaFree(d_surv);
                d_surv = nullptr;
                if (cudaMalloc((void **)&d_surv, c.surv_bytes) != cudaSuccess) {
                    cudaGetLastError();
                    surv_cap = 0;
                    continue;   // this shape does not fit in memory now: skip it
                }
                surv_cap = c.surv_bytes;
            }
            c.d_surv = d_surv;
            int *counter = pl->d_counters + 16 * (int)gi;
            float ms = 0.f;
            for (int rep = 0; rep < 3 && st == VD_OK; ++rep) {
                if (rep == 1 && cudaEventRecord(e0, cs) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "event");
                if (cudaMemsetAsync(counter, 0, sizeof(int), cs) != cudaSuccess)
                    st = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
                if (st == VD_OK) st = launch_group(c, d_user, pl->d_llr_int, d_out, counter, pl->d_status, cs);
            }
            if (st == VD_OK && cudaEventRecord(e1, cs) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "event");
            if (st == VD_OK && cudaEventSynchronize(e1) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "sync");
            if (st != VD_OK) { cleanup(); return st; }
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) { best_ms = ms; best = sh; }
        }
        if (best.lanes != g.lanes || best.r4 != g.r4) {
            cudaFree(g.d_surv);
            g.d_surv = nullptr;
            if (!shape_group(g, best.lanes, best.r4, n_sm) ||
                cudaMalloc((void **)&g.d_surv, g.surv_bytes) != cudaSuccess) {
                cudaGetLastError();
                cleanup();
                return fail(VD_ENOMEM, "cannot allocate %zu bytes of survivor scratch", g.surv_bytes);
            }
        }
    }
    cleanup();
    // the tuning launches leave no trace: clear the status word
    if (cudaMemsetAsync(pl->d_status, 0, 64 * sizeof(int), cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "autotuner clean-up");
    return VD_OK;
}

}  // namespace

extern "C" vd_status vd_batch_plan_create(vd_batch_plan **out, const vd_code *const *codes, int n_codes,
                                          const vd_packet *packets, int64_t n_packets,
                                          const vd_tune *tune, void *stream) {
    if (!out) return fail(VD_EINVAL, "out is NULL");
    *out = nullptr;
    if (!codes || n_codes < 1 || n_codes > kMaxBatchCodes)
        return fail(VD_EINVAL, "need 1..%d codes", kMaxBatchCodes);
    for (int i = 0; i < n_codes; ++i)
        if (!codes[i]) return fail(VD_EINVAL, "codes[%d] is NULL", i);
    if (n_packets < 0 || (n_packets > 0 && !packets)) return fail(VD_EINVAL, "bad packet array");
    if (n_packets > ((int64_t)1 << 31)) return fail(VD_EINVAL, "too many packets");
    if (tune && tune->radix != 0 && tune->radix != 2 && tune->radix != 4)
        return fail(VD_EINVAL, "tune.radix must be 0, 2 or 4");
    cudaStream_t cs = (cudaStream_t)stream;

    for (int64_t i = 0; i < n_packets; ++i) {
        const vd_packet &p = packets[i];
        if (p.code_id < 0 || p.code_id >= n_codes) return fail(VD_EINVAL, "packet %lld: bad code_id", (long long)i);
        if (p.llr_type != VD_LLR_S8 && p.llr_type != VD_LLR_S4 && p.llr_type != VD_LLR_HARD)
            return fail(VD_EUNSUPPORTED, "packet %lld: batches take int8, 4-bit or hard-decision input",
                        (long long)i);
        if (p.n_info <= 0) return fail(VD_EINVAL, "packet %lld: n_info must be positive", (long long)i);
        if (p.f < 0 || p.v < 0) return fail(VD_EINVAL, "packet %lld: negative f or v", (long long)i);
        if (p.f > 0 && p.f < p.n_info && p.f % 32)
            return fail(VD_EINVAL, "packet %lld: f must be a multiple of 32 (or >= n_info)", (long long)i);
        if (p.llr_offset < 0 || p.out_word_offset < 0)
            return fail(VD_EINVAL, "packet %lld: negative offset", (long long)i);
        if (p.llr_type == VD_LLR_S4 && (p.llr_offset & 1))
            return fail(VD_EINVAL, "packet %lld: 4-bit packets must start on a byte", (long long)i);
        if (p.llr_type == VD_LLR_HARD && (p.llr_offset & 7))
            return fail(VD_EINVAL, "packet %lld: hard-decision packets must start on a byte", (long long)i);
        if (p.flags & ~(uint32_t)(VD_TERMINATED | VD_START_UNKNOWN))
            return fail(VD_EINVAL, "packet %lld: unknown flags", (long long)i);
    }

    vd_batch_plan *pl = new (std::nothrow) vd_batch_plan();
    if (!pl) return fail(VD_ENOMEM, "out of host memory");
    cudaGetDevice(&pl->device);
    pl->n_packets = n_packets;
    pl->f.assign((size_t)n_packets, 0);
    pl->v.assign((size_t)n_packets, 0);
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, pl->device);

    // internal arena for packets that need depuncturing / unpacking
    std::vector<PrepJob> jobs;
    std::vector<int64_t> int_off((size_t)n_packets, -1);
    int64_t int_bytes = 0;
    memset(&pl->prep, 0, sizeof pl->prep);
    for (int i = 0; i < n_codes; ++i) {
        PrepCode &pc = pl->prep.codes[i];
        pc.beta = codes[i]->beta;
        pc.period = codes[i]->period;
        pc.kept_per_period = codes[i]->kept_per_period;
        memcpy(pc.punct, codes[i]->punct, sizeof pc.punct);
        memcpy(pc.kept_prefix, codes[i]->kept_prefix, sizeof pc.kept_prefix);
    }
    for (int64_t i = 0; i < n_packets; ++i) {
        const vd_packet &p = packets[i];
        const vd_code *c = codes[p.code_id];
        if (c->punctured || p.llr_type == VD_LLR_S4 || p.llr_type == VD_LLR_HARD) {
            const int64_t T = p.n_info + ((p.flags & VD_TERMINATED) ? c->K - 1 : 0);
            PrepJob j;
            j.src = nullptr;
            j.src_off = p.llr_offset;
            j.dst_off = int_bytes;
            j.T = T;
            j.code_slot = p.code_id;
            j.llr_type = p.llr_type;
            jobs.push_back(j);
            int_off[(size_t)i] = int_bytes;
            int_bytes += (T * c->beta + 15) & ~(int64_t)15;
        }
    }

    vd_status st = VD_OK;
    for (vd::CodeKind kind : {vd::KIND_K7_R2, vd::KIND_K9_R3}) {
        std::vector<int64_t> members;
        int K = 0;
        for (int64_t i = 0; i < n_packets; ++i) {
            const vd_code *c = codes[packets[i].code_id];
            if (c->kind == kind) { members.push_back(i); K = c->K; }
        }
        if (members.empty()) continue;
        vd_batch_group g;
        memset(&g, 0, sizeof g);
        g.kind = kind;
        g.K = K;
        g.lanes = (tune && tune->lanes > 0) ? tune->lanes : default_lanes(kind);
        g.r4 = tune && tune->radix == 4;
        if (!kind_geom(kind, g.lanes, g.r4, &g.geom)) {
            free_plan(pl);
            return fail(VD_EUNSUPPORTED, "no batch kernel with %d lanes for K=%d", g.lanes, K);
        }
        g.threads = vd::kThreads;
        int bps = 0;
        cudaError_t e = kind == vd::KIND_K7_R2 ? vd::batch_occupancy_k7(g.lanes, g.r4, &bps)
                                               : vd::batch_occupancy_k9(g.lanes, g.r4, &bps);
        if (e != cudaSuccess || bps < 1) { free_plan(pl); return cuda_fail(e, "occupancy query"); }
        g.blocks = (int64_t)n_sm * bps;
        const int ppw = 32 / g.lanes;
        const int64_t slots = g.blocks * (g.threads / 32);
        const int U = g.geom.U;
        auto wpad_of = [&](int64_t W) { return ((W + U - 1) / U) * U; };

        // frame length: the caller's, or the tuner's choice for this group
        const int v_def = (tune && tune->v > 0) ? tune->v : default_v(K);
        int f_tuned = (tune && tune->f > 0) ? tune->f : 0;
        bool need_tune = false;
        for (int64_t i : members) need_tune |= packets[i].f == 0;
        if (need_tune && f_tuned == 0) {
            static const int cands[] = {128, 192, 256, 384, 512, 768, 1024, 1536, 2048};
            double best = 1e300;
            for (int F : cands) {
                std::vector<int64_t> wp;
                for (int64_t i : members) {
                    const vd_packet &p = packets[i];
                    const int64_t T = p.n_info + ((p.flags & VD_TERMINATED) ? K - 1 : 0);
                    const int64_t f = p.f > 0 ? p.f : (p.n_info <= F ? p.n_info : F);
                    const int64_t v = p.f > 0 ? p.v : v_def;
                    const int64_t nw = (p.n_info + f - 1) / f;
                    for (int64_t s = 0; s < nw; ++s) wp.push_back(wpad_of(frame_len(s, p.n_info, T, f, v)));
                }
                const double mk = predict_makespan(wp, ppw, slots);
                if (mk < best * 0.98) { best = mk; f_tuned = F; }
            }
        }
        // frames of every member packet
        struct Fr { int64_t wpad; uint32_t pk, s; };
        std::vector<Fr> frs;
        std::vector<vd::PacketDesc> pds;
        std::vector<uint32_t> local_of(members.size());
        for (size_t m = 0; m < members.size(); ++m) {
            const int64_t i = members[m];
            const vd_packet &p = packets[i];
            const int64_t T = p.n_info + ((p.flags & VD_TERMINATED) ? K - 1 : 0);
            int64_t f = p.f, v = p.v;
            if (f == 0) {
                f = p.n_info <= f_tuned ? p.n_info : f_tuned;
                v = v_def;
            }
            pl->f[(size_t)i] = (int32_t)f;
            pl->v[(size_t)i] = (int32_t)v;
            vd::PacketDesc d;
            memset(&d, 0, sizeof d);
            if (int_off[(size_t)i] >= 0) {
                d.llr_off = int_off[(size_t)i];
                d.flags = p.flags | vd::PKT_INTERNAL_LLR;
            } else {
                d.llr_off = p.llr_offset;
                d.flags = p.flags;
            }
            d.out_word_off = p.out_word_offset;
            d.n_info = p.n_info;
            d.f = (int32_t)f;
            d.v = (int32_t)v;
            pds.push_back(d);
            const int64_t nw = (p.n_info + f - 1) / f;
            for (int64_t s = 0; s < nw; ++s)
                frs.push_back({wpad_of(frame_len(s, p.n_info, T, f, v)), (uint32_t)m, (uint32_t)s});
        }
        std::stable_sort(frs.begin(), frs.end(), [](const Fr &a, const Fr &b) { return a.wpad > b.wpad; });
        std::vector<vd::PairRef> pairs;
        for (size_t k = 0; k < frs.size(); k += 2) {
            vd::PairRef r;
            r.p0 = frs[k].pk;
            r.s0 = frs[k].s;
            if (k + 1 < frs.size()) { r.p1 = frs[k + 1].pk; r.s1 = frs[k + 1].s; }
            else { r.p1 = 0xFFFFFFFFu; r.s1 = 0; }
            pairs.push_back(r);
        }
        pl->frames += (int64_t)frs.size();
        g.n_pairs = (int64_t)pairs.size();
        g.wpad_cap = frs.empty() ? U : (int32_t)frs.front().wpad;
        if (!shape_group(g, g.lanes, g.r4, n_sm)) { free_plan(pl); return fail(VD_ECUDA, "occupancy query"); }
        if ((st = upload(&g.d_pk, pds, cs)) != VD_OK || (st = upload(&g.d_pairs, pairs, cs)) != VD_OK) {
            pl->groups.push_back(g);
            free_plan(pl);
            return st;
        }
        e = cudaMalloc((void **)&g.d_surv, g.surv_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            pl->groups.push_back(g);
            free_plan(pl);
            return fail(VD_ENOMEM, "cannot allocate %zu bytes of survivor scratch", g.surv_bytes);
        }
        pl->groups.push_back(g);
    }
    pl->n_jobs = (int64_t)jobs.size();
    if ((st = upload(&pl->d_jobs, jobs, cs)) != VD_OK) { free_plan(pl); return st; }
    if (int_bytes > 0) {
        cudaError_t e = cudaMalloc((void **)&pl->d_llr_int, (size_t)int_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_plan(pl);
            return fail(VD_ENOMEM, "cannot allocate %lld bytes for depunctured LLRs", (long long)int_bytes);
        }
        pl->llr_int_bytes = (size_t)int_bytes;
    }
    cudaError_t e = cudaMalloc((void **)&pl->d_counters, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&pl->d_status, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_status, 0, 64 * sizeof(int), cs);
    if (e != cudaSuccess) { free_plan(pl); return cuda_fail(e, "plan counters"); }
    e = cudaStreamSynchronize(cs);   // host vectors above go out of scope
    if (e != cudaSuccess) { free_plan(pl); return cuda_fail(e, "cudaStreamSynchronize"); }
    const bool tune_radix = !tune || tune->radix == 0, tune_lanes = !tune || tune->lanes == 0;
    if ((tune_radix || tune_lanes) && (st = autotune_shapes(pl, codes, packets, n_packets, tune_radix,
                                                            tune_lanes, n_sm, cs)) != VD_OK) {
        free_plan(pl);
        return st;
    }
    *out = pl;
    return VD_OK;
}

extern "C" void vd_batch_plan_destroy(vd_batch_plan *plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    free_plan(plan);
}

extern "C" vd_status vd_batch_plan_launch(vd_batch_plan *pl, const void *d_llr_arena, uint32_t *d_out_arena,
                                          void *stream) {
    if (!pl) return fail(VD_EINVAL, "plan is NULL");
    if (pl->n_packets == 0) return VD_OK;
    if (!d_llr_arena || !d_out_arena) return fail(VD_EINVAL, "NULL arena");
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e;
    if (pl->n_jobs > 0) {
        PrepBatchParams pp = pl->prep;
        pp.src = (const uint8_t *)d_llr_arena;
        pp.dst = pl->d_llr_int;
        pp.jobs = pl->d_jobs;
        pp.n_jobs = pl->n_jobs;
        prep_batch_kernel<<<(unsigned)pl->n_jobs, 128, 0, cs>>>(pp);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch pre-pass launch");
    }
    e = cudaMemsetAsync(pl->d_counters, 0, 64 * sizeof(int), cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    pl->last_parity = 0;
    int gi = 0;
    for (auto &g : pl->groups) {
        // separate cache lines per group for the task counters
        const vd_status st = launch_group(g, (const int8_t *)d_llr_arena, pl->d_llr_int, d_out_arena,
                                          pl->d_counters + 16 * gi, pl->d_status, cs);
        if (st != VD_OK) return st;
        ++gi;
        if (gi >= 4) break;
    }
    return VD_OK;
}

extern "C" vd_status vd_batch_plan_launch_chained(vd_batch_plan *pl, const void *d_llr_arena,
                                                  uint32_t *d_out_arena, void *stream) {
    if (!pl) return fail(VD_EINVAL, "plan is NULL");
    if (pl->n_packets == 0) return VD_OK;
    if (!d_llr_arena || !d_out_arena) return fail(VD_EINVAL, "NULL arena");
    // a pre-pass writes what the decode kernels read: no overlap then
    if (pl->n_jobs > 0) return vd_batch_plan_launch(pl, d_llr_arena, d_out_arena, stream);
    cudaStream_t cs = (cudaStream_t)stream;
    const int parity = pl->last_parity ^ 1;   // never the scratch of the launch before
    if (parity == 1) {
        for (auto &g : pl->groups) {
            if (g.d_surv2) continue;
            const cudaError_t e = cudaMalloc((void **)&g.d_surv2, g.surv_bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                g.d_surv2 = nullptr;
                return fail(VD_ENOMEM, "cannot allocate %zu bytes of survivor scratch", g.surv_bytes);
            }
        }
    }
    // counters: zero at plan creation and after every launch (the kernel's
    // last warp zeroes them); no memset, which would end the overlap
    int gi = 0;
    for (auto &g : pl->groups) {
        const vd_status st = launch_group(g, (const int8_t *)d_llr_arena, pl->d_llr_int, d_out_arena,
                                          pl->d_counters + 16 * gi + 8 * parity, pl->d_status, cs, parity, true);
        if (st != VD_OK) return st;
        ++gi;
        if (gi >= 4) break;
    }
    pl->last_parity = parity;
    return VD_OK;
}

extern "C" vd_status vd_batch_plan_launch_graph(vd_batch_plan *pl, const void *d_llr_arena,
                                                uint32_t *d_out_arena, void *stream) {
    if (!pl) return fail(VD_EINVAL, "plan is NULL");
    cudaStream_t cs = (cudaStream_t)stream;
    if (!cs) return fail(VD_EINVAL, "graph replay needs a non-default stream");
    if (!pl->graph || pl->graph_llr != d_llr_arena || pl->graph_out != d_out_arena) {
        if (pl->graph) { cudaGraphExecDestroy(pl->graph); pl->graph = nullptr; }
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        vd_status st = vd_batch_plan_launch(pl, d_llr_arena, d_out_arena, stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cs, &graph);
        if (st != VD_OK) { if (graph) cudaGraphDestroy(graph); return st; }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&pl->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { pl->graph = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
        pl->graph_llr = d_llr_arena;
        pl->graph_out = d_out_arena;
    }
    cudaError_t e = cudaGraphLaunch(pl->graph, cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return VD_OK;
}

extern "C" vd_status vd_batch_plan_info(const vd_batch_plan *pl, vd_batch_info *info) {
    if (!pl || !info) return fail(VD_EINVAL, "NULL argument");
    memset(info, 0, sizeof *info);
    info->n_packets = pl->n_packets;
    info->n_frames = pl->frames;
    info->n_launches = (int32_t)pl->groups.size() + (pl->n_jobs > 0 ? 1 : 0);
    for (const auto &g : pl->groups) {
        info->n_pairs += g.n_pairs;
        info->scratch_bytes += (int64_t)g.surv_bytes * (g.d_surv2 ? 2 : 1);
        info->lanes = g.lanes;
        info->radix = g.r4 ? 4 : 2;
        info->resident_warps += g.blocks * (g.threads / 32);
    }
    info->scratch_bytes += (int64_t)pl->llr_int_bytes;
    return VD_OK;
}

extern "C" vd_status vd_batch_plan_packet_tune(const vd_batch_plan *pl, int32_t *f_out, int32_t *v_out) {
    if (!pl || !f_out || !v_out) return fail(VD_EINVAL, "NULL argument");
    for (int64_t i = 0; i < pl->n_packets; ++i) {
        f_out[i] = pl->f[(size_t)i];
        v_out[i] = pl->v[(size_t)i];
    }
    return VD_OK;
}

extern "C" vd_status vd_batch_plan_status(vd_batch_plan *pl, void *stream) {
    if (!pl) return fail(VD_EINVAL, "plan is NULL");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int h = 0;
    e = cudaMemcpy(&h, pl->d_status, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    if (h) {
        cudaMemset(pl->d_status, 0, sizeof h);
        return fail(VD_EBOUNDS, "a device-side bounds check fired in a batch launch (0x%x)", h);
    }
    return VD_OK;
}

extern "C" vd_status vd_decode_batch(const vd_code *const *codes, int n_codes, const vd_packet *packets,
                                     int64_t n_packets, const void *d_llr_arena, uint32_t *d_out_arena,
                                     const vd_tune *tune, void *stream) {
    vd_batch_plan *pl = nullptr;
    vd_status st = vd_batch_plan_create(&pl, codes, n_codes, packets, n_packets, tune, stream);
    if (st != VD_OK) return st;
    st = vd_batch_plan_launch(pl, d_llr_arena, d_out_arena, stream);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    free_plan(pl);
    if (st != VD_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return VD_OK;
}

namespace vd {

cudaError_t launch_prep_batch(const PrepBatchParams &p, cudaStream_t st) {
    if (p.n_jobs <= 0) return cudaSuccess;
    prep_batch_kernel<<<(unsigned)p.n_jobs, 128, 0, st>>>(p);
    return cudaGetLastError();
}

void fill_prep_code(const vd_code *c, PrepCode *pc) {
    pc->beta = c->beta;
    pc->period = c->period;
    pc->kept_per_period = c->kept_per_period;
    memcpy(pc->punct, c->punct, sizeof pc->punct);
    memcpy(pc->kept_prefix, c->kept_prefix, sizeof pc->kept_prefix);
}

}  // namespace vd
