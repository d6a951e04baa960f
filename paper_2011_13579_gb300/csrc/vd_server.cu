// Continuous-batching decode server (vd_server_*): packets from many sources
// are queued on the host, admitted while the device arena has room, and
// decoded in micro-batches — one persistent launch per code kind, on a small
// pool of CUDA streams so that batches formed while earlier ones still run
// overlap on the device.  See include/vd.h.
//
// Memory: one device arena (LLRs, depunctured LLRs and outputs of admitted
// packets) with a pinned host mirror at the same offsets.  Each micro-batch
// takes one contiguous arena region (first fit, freed on completion).  Host
// packets are copied once, at submit, into a pinned staging area; a batch's
// staged packets keep their staging layout in the region, so each run of
// packets that are contiguous in staging goes down in one copy (and those
// that did not fit in staging in one more, from the mirror); the kernels
// read device memory only.  The outputs come back in one copy.  Every
// per-stream buffer (descriptors, work list, survivor scratch) is allocated
// once, when the server is created.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/vd.h"
#include "vd_code.h"
#include "vd_launch.h"

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

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr int kMaxKinds = 2;
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Req {
    uint64_t tag;
    int code_id, llr_type;
    int64_t n_info, T;
    uint32_t flags;
    int32_t f, v;
    std::vector<uint8_t> llr;      // received values as submitted (host packets that did not fit in staging)
    const uint8_t *dev_llr;        // device packets: the caller's buffer, read in place; else NULL
    size_t stage_off, stage_bytes; // the packet's staging region (stage_bytes 0: none)
    size_t in_bytes, prep_bytes, out_words;
    int64_t submit_ns, admit_ns, done_ns;
    size_t in_off, prep_off, out_off;   // arena offsets (relative to the batch region)
};

// First-fit allocator over [0, cap) with coalescing frees.
struct Arena {
    std::map<size_t, size_t> free_;    // offset -> size
    size_t cap = 0, used = 0;
    void init(size_t c) { cap = c; free_.clear(); free_[0] = c; used = 0; }
    bool alloc(size_t n, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used += n;
                return true;
            }
        }
        return false;
    }
    size_t largest() const {
        size_t m = 0;
        for (auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
    void release(size_t off, size_t n) {
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct KindRes {
    vd::CodeKind kind;
    int K, lanes, f, v;
    bool r4;
    vd::KernelGeom geom;
    int64_t blocks;
    int32_t wpad_cap;
    vd::PacketDesc *d_pk;
    vd::PairRef *d_pairs;
    uint32_t *d_surv;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Req *> reqs;
    size_t region_off = 0, region_bytes = 0;
    struct Run { size_t stage_off, region_off, bytes; };
    std::vector<Run> runs;         // staged inputs: one copy per run contiguous in staging
    std::vector<uint32_t> members;       // work lists of one launch, kept for their capacity
    std::vector<int64_t> sort_start;
    std::vector<uint64_t> sorted;
    size_t mirror_lo = 0, mirror_hi = 0;   // region bytes of the inputs that come from the mirror
    KindRes kinds[kMaxKinds];
    vd::PrepJob *d_jobs = nullptr;
    int *d_counters = nullptr;
    // pinned staging of descriptors
    vd::PacketDesc *h_pk[kMaxKinds] = {nullptr, nullptr};
    vd::PairRef *h_pairs[kMaxKinds] = {nullptr, nullptr};
    vd::PrepJob *h_jobs = nullptr;
};

}  // namespace

struct vd_server {
    std::vector<const vd_code *> codes;
    vd_server_config cfg;
    int device = 0, n_sm = 0;
    uint8_t *d_arena = nullptr, *h_arena = nullptr;
    Arena arena;
    // pinned staging for host packets: submit copies the values there once,
    // and each batch uploads its staged packets from there in a few copies
    uint8_t *h_stage = nullptr;
    Arena stage;
    std::mutex stage_mu;
    std::vector<Slot> slots;
    int *d_status = nullptr;
    int64_t max_pairs = 0;
    vd::PrepBatchParams prep_tmpl;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req *> pending;
    std::deque<Req *> done_q;
    std::thread worker;
    std::atomic<bool> stop{false};
    std::atomic<int64_t> in_system{0};
    vd_server_stats stats;
    std::atomic<int> error{0};
};

namespace {

int kind_index(vd::CodeKind k) { return k == vd::KIND_K7_R2 ? 0 : 1; }

void free_server(vd_server *s) {
    if (!s) return;
    for (auto &sl : s->slots) {
        for (auto &kr : sl.kinds) {
            cudaFree(kr.d_pk);
            cudaFree(kr.d_pairs);
            cudaFree(kr.d_surv);
        }
        cudaFree(sl.d_jobs);
        cudaFree(sl.d_counters);
        for (int k = 0; k < kMaxKinds; ++k) {
            cudaFreeHost(sl.h_pk[k]);
            cudaFreeHost(sl.h_pairs[k]);
        }
        cudaFreeHost(sl.h_jobs);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    cudaFree(s->d_arena);
    cudaFreeHost(s->h_arena);
    cudaFreeHost(s->h_stage);
    cudaFree(s->d_status);
    for (Req *r : s->pending) delete r;
    for (Req *r : s->done_q) delete r;
    delete s;
}

// Frames of one packet: (padded length, frame index)
int64_t frame_len_of(int64_t s, int64_t n_info, int64_t T, int64_t f, int64_t v) {
    const vd::Frame w = vd::frame_of(s, n_info, T, f, v, 0);
    return w.b - w.a;
}

// Launches one micro-batch on a slot: copies, pre-pass, one persistent launch
// per code kind, output copy, completion event.
bool launch_batch(vd_server *s, Slot &sl) {
    const cudaStream_t st = sl.st;
    uint8_t *dbase = s->d_arena + sl.region_off;
    uint8_t *hbase = s->h_arena + sl.region_off;
    // inputs: one copy per run of staged packets, one of the rest from the mirror
    for (const Slot::Run &run : sl.runs)
        if (cudaMemcpyAsync(dbase + run.region_off, s->h_stage + run.stage_off, run.bytes, cudaMemcpyHostToDevice,
                            st) != cudaSuccess)
            return false;
    if (sl.mirror_hi > sl.mirror_lo &&
        cudaMemcpyAsync(dbase + sl.mirror_lo, hbase + sl.mirror_lo, sl.mirror_hi - sl.mirror_lo,
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return false;
    // pre-pass for punctured / 4-bit packets
    int64_t n_jobs = 0;
    for (Req *r : sl.reqs) {
        if (!r->prep_bytes) continue;
        vd::PrepJob &j = sl.h_jobs[n_jobs++];
        j.src = r->dev_llr;   // NULL: the values came up with the batch, into the region
        j.src_off = r->dev_llr ? 0
                    : r->llr_type == VD_LLR_S4   ? (int64_t)(r->in_off * 2)
                    : r->llr_type == VD_LLR_HARD ? (int64_t)(r->in_off * 8)
                                                 : (int64_t)r->in_off;
        j.dst_off = (int64_t)r->prep_off;
        j.T = r->T;
        j.code_slot = r->code_id;
        j.llr_type = r->llr_type;
    }
    if (n_jobs) {
        if (cudaMemcpyAsync(sl.d_jobs, sl.h_jobs, n_jobs * sizeof(vd::PrepJob), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return false;
        vd::PrepBatchParams pp = s->prep_tmpl;
        pp.src = dbase;
        pp.dst = (int8_t *)dbase;
        pp.jobs = sl.d_jobs;
        pp.n_jobs = n_jobs;
        if (vd::launch_prep_batch(pp, st) != cudaSuccess) return false;
    }
    if (cudaMemsetAsync(sl.d_counters, 0, 64 * sizeof(int), st) != cudaSuccess) return false;
    for (int ki = 0; ki < kMaxKinds; ++ki) {
        KindRes &kr = sl.kinds[ki];
        if (!kr.d_pk) continue;
        std::vector<uint32_t> &members = sl.members;
        members.clear();
        for (uint32_t i = 0; i < sl.reqs.size(); ++i)
            if (s->codes[sl.reqs[i]->code_id]->kind == kr.kind) members.push_back(i);
        if (members.empty()) continue;
        // Frames longest first, stable (packet, then frame order): a counting
        // sort over the padded lengths (multiples of U up to wpad_cap).  Only
        // a packet's first frame and its last two can be shorter than f + 2v
        // when f >= v (so with the default frame lengths), so such a packet
        // costs four length computations, and the frames between are placed
        // as a run; other packets have every frame's length computed.
        const int U = kr.geom.U;
        const int nb = kr.wpad_cap / U + 1;
        auto bucket_of = [&](int64_t W) {   // a longer frame (never built) goes first; the kernel refuses it
            const int64_t wpad = ((W + U - 1) / U) * U;
            return (size_t)std::max<int64_t>(0, nb - 1 - wpad / U);
        };
        struct Lens { int64_t nf; bool run; size_t b0, bm, bp, bl; };   // buckets: first, middle run, last two
        auto lens_of = [&](const Req *r) {
            Lens L;
            L.nf = (r->n_info + r->f - 1) / r->f;
            const int64_t nf = L.nf;
            L.run = nf > 4 && r->f >= r->v;
            L.b0 = bucket_of(frame_len_of(0, r->n_info, r->T, r->f, r->v));
            L.bm = L.run ? bucket_of(frame_len_of(1, r->n_info, r->T, r->f, r->v)) : 0;
            L.bp = L.run ? bucket_of(frame_len_of(nf - 2, r->n_info, r->T, r->f, r->v)) : 0;
            L.bl = L.run ? bucket_of(frame_len_of(nf - 1, r->n_info, r->T, r->f, r->v)) : 0;
            return L;
        };
        std::vector<int64_t> &start = sl.sort_start;
        start.assign((size_t)nb + 1, 0);
        int64_t n_frames = 0;
        for (uint32_t m = 0; m < members.size(); ++m) {
            Req *r = sl.reqs[members[m]];
            vd::PacketDesc &d = sl.h_pk[ki][m];
            memset(&d, 0, sizeof d);
            d.out_word_off = (int64_t)(r->out_off / 4);
            d.n_info = r->n_info;
            d.f = r->f;
            d.v = r->v;
            if (r->dev_llr && !r->prep_bytes) {
                // unpunctured int8 device packet: decoded straight from the caller's buffer
                d.llr_off = (int64_t)(uintptr_t)r->dev_llr;
                d.flags = r->flags | vd::PKT_ABS_LLR;
            } else {
                d.llr_off = (int64_t)(r->prep_bytes ? r->prep_off : r->in_off);
                d.flags = r->flags;   // LLRs are in the arena: "user" arena of this launch
            }
            const Lens L = lens_of(r);
            n_frames += L.nf;
            if (!L.run) {
                for (int64_t f = 0; f < L.nf; ++f)
                    ++start[bucket_of(frame_len_of(f, r->n_info, r->T, r->f, r->v)) + 1];
            } else {
                ++start[L.b0 + 1];
                start[L.bm + 1] += L.nf - 3;
                ++start[L.bp + 1];
                ++start[L.bl + 1];
            }
        }
        for (int b = 0; b < nb; ++b) start[(size_t)b + 1] += start[(size_t)b];
        std::vector<uint64_t> &sorted = sl.sorted;   // (packet << 32) | frame
        sorted.resize((size_t)n_frames);
        for (uint32_t m = 0; m < members.size(); ++m) {
            const Req *r = sl.reqs[members[m]];
            const Lens L = lens_of(r);
            const uint64_t pk = (uint64_t)m << 32;
            if (!L.run) {
                for (int64_t f = 0; f < L.nf; ++f)
                    sorted[(size_t)start[bucket_of(frame_len_of(f, r->n_info, r->T, r->f, r->v))]++] = pk | (uint64_t)f;
            } else {
                sorted[(size_t)start[L.b0]++] = pk;
                int64_t &at = start[L.bm];
                for (int64_t f = 1; f < L.nf - 2; ++f) sorted[(size_t)at++] = pk | (uint64_t)f;
                sorted[(size_t)start[L.bp]++] = pk | (uint64_t)(L.nf - 2);
                sorted[(size_t)start[L.bl]++] = pk | (uint64_t)(L.nf - 1);
            }
        }
        int64_t np = 0;
        for (size_t k = 0; k < sorted.size(); k += 2) {
            vd::PairRef &pr = sl.h_pairs[ki][np++];
            pr.p0 = (uint32_t)(sorted[k] >> 32);
            pr.s0 = (uint32_t)sorted[k];
            if (k + 1 < sorted.size()) { pr.p1 = (uint32_t)(sorted[k + 1] >> 32); pr.s1 = (uint32_t)sorted[k + 1]; }
            else { pr.p1 = 0xFFFFFFFFu; pr.s1 = 0; }
        }
        if (cudaMemcpyAsync(kr.d_pk, sl.h_pk[ki], members.size() * sizeof(vd::PacketDesc),
                            cudaMemcpyHostToDevice, st) != cudaSuccess)
            return false;
        if (cudaMemcpyAsync(kr.d_pairs, sl.h_pairs[ki], np * sizeof(vd::PairRef), cudaMemcpyHostToDevice,
                            st) != cudaSuccess)
            return false;
        vd::BatchParams p;
        p.chained = 0;
        const int ppw = 32 / kr.lanes;
        p.pk = kr.d_pk;
        p.pairs = kr.d_pairs;
        p.n_pairs = np;
        p.n_tasks = (np + ppw - 1) / ppw;
        p.llr_user = (const int8_t *)dbase;
        p.llr_int = (const int8_t *)dbase;
        p.out = (uint32_t *)dbase;
        p.counter = sl.d_counters + 16 * ki;
        p.surv = kr.d_surv;
        p.wpad_cap = kr.wpad_cap;
        p.status = s->d_status;
        const int64_t blocks = std::max<int64_t>(1, std::min(kr.blocks, (p.n_tasks * 32 + vd::kThreads - 1) / vd::kThreads));
        const cudaError_t e = kr.kind == vd::KIND_K7_R2 ? vd::launch_batch_k7(kr.lanes, kr.r4, p, blocks, st)
                                                        : vd::launch_batch_k9(kr.lanes, kr.r4, p, blocks, st);
        if (e != cudaSuccess) return false;
    }
    // outputs back to the pinned mirror
    size_t out_lo = SIZE_MAX, out_hi = 0;
    for (Req *r : sl.reqs) {
        out_lo = std::min(out_lo, r->out_off);
        out_hi = std::max(out_hi, r->out_off + r->out_words * 4);
    }
    if (out_hi > out_lo &&
        cudaMemcpyAsync(hbase + out_lo, dbase + out_lo, out_hi - out_lo, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return false;
    return cudaEventRecord(sl.done, st) == cudaSuccess;
}

void worker_main(vd_server *s) {
    cudaSetDevice(s->device);
    const int64_t max_batch = s->cfg.max_batch;
    while (!s->stop.load()) {
        bool did = false;
        // 1. completions
        for (auto &sl : s->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            const int64_t t = now_ns();
            std::lock_guard<std::mutex> lk(s->mu);
            for (Req *r : sl.reqs) {
                r->done_ns = t;
                // the decoded words move into the request (the region is released now)
                r->llr.assign(s->h_arena + sl.region_off + r->out_off,
                              s->h_arena + sl.region_off + r->out_off + r->out_words * 4);
                s->done_q.push_back(r);
                s->stats.completed += 1;
                s->stats.bits_decoded += r->n_info;
            }
            if (q != cudaSuccess) s->error.store((int)q);
            s->arena.release(sl.region_off, sl.region_bytes);
            {
                // the batch's staged packets form the runs of its layout
                std::lock_guard<std::mutex> sk(s->stage_mu);
                for (const Slot::Run &run : sl.runs) s->stage.release(run.stage_off, run.bytes);
            }
            sl.reqs.clear();
            sl.busy = false;
            did = true;
            s->cv.notify_all();
        }
        // 2. admission + launch on a free slot
        Slot *free_slot = nullptr;
        for (auto &sl : s->slots)
            if (!sl.busy) { free_slot = &sl; break; }
        if (free_slot) {
            std::vector<Req *> batch;
            size_t region = 0, off = 0;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                const size_t room = s->arena.largest();
                int64_t frames[kMaxKinds] = {0, 0};
                while (!s->pending.empty() && (int64_t)batch.size() < max_batch) {
                    Req *r = s->pending.front();
                    const size_t need = align_up(r->in_bytes) + align_up(r->prep_bytes) + align_up(r->out_words * 4);
                    const int ki = kind_index(s->codes[r->code_id]->kind);
                    const int64_t fr = (r->n_info + r->f - 1) / r->f;
                    if (region + need > room) break;
                    if ((frames[ki] + fr + 1) / 2 > s->max_pairs) break;
                    frames[ki] += fr;
                    region += need;
                    batch.push_back(r);
                    s->pending.pop_front();
                }
                if (!batch.empty() && !s->arena.alloc(region, &off)) {
                    // not reachable: region <= the largest free range
                    for (auto it = batch.rbegin(); it != batch.rend(); ++it) s->pending.push_front(*it);
                    batch.clear();
                }
            }
            if (!batch.empty()) {
                {
                    // lay out: staged inputs (runs contiguous in staging keep their
                    // layout), the other host inputs, pre-pass outputs, decoded words
                    size_t cur = 0;
                    const int64_t t = now_ns();
                    std::vector<Slot::Run> &runs = free_slot->runs;
                    runs.clear();
                    for (Req *r : batch) {
                        r->admit_ns = t;
                        if (!r->stage_bytes) continue;
                        if (!runs.empty() && runs.back().stage_off + runs.back().bytes == r->stage_off) {
                            r->in_off = runs.back().region_off + runs.back().bytes;
                            runs.back().bytes += r->stage_bytes;
                        } else {
                            r->in_off = cur;
                            runs.push_back({r->stage_off, cur, r->stage_bytes});
                        }
                        cur = r->in_off + r->stage_bytes;
                    }
                    free_slot->mirror_lo = cur;
                    for (Req *r : batch)
                        if (!r->stage_bytes && r->in_bytes) { r->in_off = cur; cur += align_up(r->in_bytes); }
                    free_slot->mirror_hi = cur;
                    for (Req *r : batch) { r->prep_off = cur; cur += align_up(r->prep_bytes); }
                    for (Req *r : batch) { r->out_off = cur; cur += align_up(r->out_words * 4); }
                    for (Req *r : batch)
                        if (!r->stage_bytes && r->in_bytes)
                            memcpy(s->h_arena + off + r->in_off, r->llr.data(), r->in_bytes);
                    free_slot->reqs = batch;
                    free_slot->region_off = off;
                    free_slot->region_bytes = region;
                    free_slot->busy = true;
                    if (!launch_batch(s, *free_slot)) s->error.store(-1);
                    s->stats.batches += 1;
                    did = true;
                }
            }
        }
        if (!did) {
            std::unique_lock<std::mutex> lk(s->mu);
            bool busy = false;
            for (auto &sl : s->slots) busy |= sl.busy;
            if (busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(5));
            } else {
                s->cv.wait_for(lk, std::chrono::microseconds(200),
                               [&] { return s->stop.load() || !s->pending.empty(); });
            }
        }
    }
}

}  // namespace

extern "C" vd_status vd_server_create(vd_server **out, const vd_code *const *codes, int n_codes,
                                      const vd_server_config *cfg) {
    if (!out) return fail(VD_EINVAL, "out is NULL");
    *out = nullptr;
    if (!codes || n_codes < 1 || n_codes > vd::kMaxBatchCodes) return fail(VD_EINVAL, "need 1..16 codes");
    for (int i = 0; i < n_codes; ++i) if (!codes[i]) return fail(VD_EINVAL, "codes[%d] is NULL", i);
    vd_server_config c;
    memset(&c, 0, sizeof c);
    if (cfg) c = *cfg;
    if (c.device_bytes <= 0) c.device_bytes = (int64_t)256 << 20;
    if (c.max_batch <= 0) c.max_batch = 4096;
    if (c.n_streams <= 0) c.n_streams = 3;
    if (c.n_streams > 8) return fail(VD_EINVAL, "at most 8 streams");
    if (c.max_packet_bits <= 0) c.max_packet_bits = 12000;
    vd_server *s = new (std::nothrow) vd_server();
    if (!s) return fail(VD_ENOMEM, "out of host memory");
    s->codes.assign(codes, codes + n_codes);
    s->cfg = c;
    memset(&s->stats, 0, sizeof s->stats);
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, s->device);
    memset(&s->prep_tmpl, 0, sizeof s->prep_tmpl);
    for (int i = 0; i < n_codes; ++i) vd::fill_prep_code(codes[i], &s->prep_tmpl.codes[i]);

    auto bail = [&](vd_status st, const char *what) {
        free_server(s);
        return fail(st, "%s", what);
    };
    if (cudaMalloc((void **)&s->d_arena, (size_t)c.device_bytes) != cudaSuccess ||
        cudaHostAlloc((void **)&s->h_arena, (size_t)c.device_bytes, cudaHostAllocDefault) != cudaSuccess ||
        cudaMalloc((void **)&s->d_status, 256) != cudaSuccess) {
        cudaGetLastError();
        return bail(VD_ENOMEM, "cannot allocate the server arena");
    }
    cudaMemset(s->d_status, 0, 256);
    s->arena.init((size_t)c.device_bytes);
    // the staging area is optional: without it host packets go through the arena
    if (cudaHostAlloc((void **)&s->h_stage, (size_t)c.device_bytes, cudaHostAllocDefault) == cudaSuccess) {
        s->stage.init((size_t)c.device_bytes);
    } else {
        cudaGetLastError();
        cudaFreeHost(s->h_stage);
        s->h_stage = nullptr;
    }

    // which kinds are present, with their frame shape
    bool has[kMaxKinds] = {false, false};
    int Kof[kMaxKinds] = {7, 9};
    for (int i = 0; i < n_codes; ++i) has[kind_index(codes[i]->kind)] = true;
    const int64_t max_frames = (int64_t)c.max_batch * 4 + 64;
    s->max_pairs = max_frames;
    s->slots.resize((size_t)c.n_streams);
    for (auto &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc((void **)&sl.d_jobs, (size_t)c.max_batch * sizeof(vd::PrepJob)) != cudaSuccess ||
            cudaMalloc((void **)&sl.d_counters, 64 * sizeof(int)) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_jobs, (size_t)c.max_batch * sizeof(vd::PrepJob), 0) != cudaSuccess) {
            cudaGetLastError();
            return bail(VD_ENOMEM, "cannot allocate server stream resources");
        }
        for (int k = 0; k < kMaxKinds; ++k) {
            KindRes &kr = sl.kinds[k];
            memset(&kr, 0, sizeof kr);
            if (!has[k]) continue;
            kr.kind = k == 0 ? vd::KIND_K7_R2 : vd::KIND_K9_R3;
            kr.K = Kof[k];
            kr.lanes = c.lanes > 0 ? c.lanes : (k == 0 ? 1 : 4);
            kr.r4 = c.radix == 4;
            kr.f = k == 0 ? (c.f7 > 0 ? c.f7 : 256) : (c.f9 > 0 ? c.f9 : 512);
            kr.v = k == 0 ? (c.v7 > 0 ? c.v7 : 42) : (c.v9 > 0 ? c.v9 : 64);
            const bool ok = k == 0 ? vd::geom_k7(kr.lanes, kr.r4, &kr.geom) : vd::geom_k9(kr.lanes, kr.r4, &kr.geom);
            if (!ok) return bail(VD_EUNSUPPORTED, "no batch kernel for this lane count");
            int bps = 0;
            if ((k == 0 ? vd::batch_occupancy_k7(kr.lanes, kr.r4, &bps) : vd::batch_occupancy_k9(kr.lanes, kr.r4, &bps)) != cudaSuccess || bps < 1)
                return bail(VD_ECUDA, "occupancy query failed");
            kr.blocks = (int64_t)s->n_sm * bps;
            const int64_t wmax = (int64_t)kr.f + std::max(2 * kr.v, kr.K - 1);
            kr.wpad_cap = (int32_t)(((wmax + kr.geom.U - 1) / kr.geom.U) * kr.geom.U);
            const size_t surv = 2u * (size_t)kr.blocks * vd::kThreads * (size_t)kr.wpad_cap * kr.geom.NW * 4u;
            if (cudaMalloc((void **)&kr.d_pk, (size_t)c.max_batch * sizeof(vd::PacketDesc)) != cudaSuccess ||
                cudaMalloc((void **)&kr.d_pairs, (size_t)max_frames * sizeof(vd::PairRef)) != cudaSuccess ||
                cudaMalloc((void **)&kr.d_surv, surv) != cudaSuccess ||
                cudaHostAlloc((void **)&sl.h_pk[k], (size_t)c.max_batch * sizeof(vd::PacketDesc), 0) != cudaSuccess ||
                cudaHostAlloc((void **)&sl.h_pairs[k], (size_t)max_frames * sizeof(vd::PairRef), 0) != cudaSuccess) {
                cudaGetLastError();
                return bail(VD_ENOMEM, "cannot allocate server kernel resources");
            }
        }
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return VD_OK;
}

namespace {

// Checks one packet and builds its request (nothing staged or queued yet).
vd_status make_req(vd_server *s, int code_id, int llr_type, const void *llr, bool device, int64_t n_values,
                   int64_t n_info, uint32_t flags, uint64_t tag, Req **out, size_t *value_bytes_out) {
    if (!s) return fail(VD_EINVAL, "server is NULL");
    if (code_id < 0 || code_id >= (int)s->codes.size()) return fail(VD_EINVAL, "bad code_id");
    if (llr_type != VD_LLR_S8 && llr_type != VD_LLR_S4 && llr_type != VD_LLR_HARD)
        return fail(VD_EUNSUPPORTED, "server takes int8, 4-bit or hard-decision input");
    if (n_info <= 0 || n_info > s->cfg.max_packet_bits) return fail(VD_EINVAL, "n_info outside (0, max_packet_bits]");
    if (flags & ~(uint32_t)(VD_TERMINATED | VD_START_UNKNOWN)) return fail(VD_EINVAL, "unknown flags");
    const vd_code *c = s->codes[(size_t)code_id];
    const int64_t T = n_info + ((flags & VD_TERMINATED) ? c->K - 1 : 0);
    const int64_t kept = vd_num_kept(c, T);
    if (n_values != kept) return fail(VD_EINVAL, "packet has %lld values, the code sends %lld", (long long)n_values, (long long)kept);
    if (!llr) return fail(VD_EINVAL, "the LLR pointer is NULL");
    Req *r = new (std::nothrow) Req();
    if (!r) return fail(VD_ENOMEM, "out of host memory");
    r->tag = tag;
    r->code_id = code_id;
    r->llr_type = llr_type;
    r->n_info = n_info;
    r->T = T;
    r->flags = flags;
    const bool k7 = c->kind == vd::KIND_K7_R2;
    const int32_t F = k7 ? (s->cfg.f7 > 0 ? s->cfg.f7 : 256) : (s->cfg.f9 > 0 ? s->cfg.f9 : 512);
    r->f = n_info <= F ? (int32_t)n_info : F;
    r->v = k7 ? (s->cfg.v7 > 0 ? s->cfg.v7 : 42) : (s->cfg.v9 > 0 ? s->cfg.v9 : 64);
    const size_t value_bytes = llr_type == VD_LLR_S4     ? (size_t)((kept + 1) / 2)
                               : llr_type == VD_LLR_HARD ? (size_t)((kept + 7) / 8)
                                                         : (size_t)kept;
    r->prep_bytes = (c->punctured || llr_type != VD_LLR_S8) ? (size_t)(T * c->beta) : 0;
    r->out_words = (size_t)((n_info + 31) / 32);
    r->stage_off = r->stage_bytes = 0;
    r->dev_llr = device ? (const uint8_t *)llr : nullptr;
    r->in_bytes = device ? 0 : value_bytes;   // device packets: nothing to upload, read in place
    const size_t need = align_up(r->in_bytes) + align_up(r->prep_bytes) + align_up(r->out_words * 4);
    if (need > s->arena.cap) { delete r; return fail(VD_ENOMEM, "packet larger than the device arena"); }
    *out = r;
    *value_bytes_out = value_bytes;
    return VD_OK;
}

// Reserves staging for a host packet's values (the caller holds stage_mu);
// false when staging is full.
bool reserve_stage(vd_server *s, Req *r, size_t value_bytes) {
    size_t off = 0;
    if (!s->h_stage || !s->stage.alloc(align_up(value_bytes), &off)) return false;
    r->stage_off = off;
    r->stage_bytes = align_up(value_bytes);
    return true;
}

// Copies a host packet's values into its reserved staging, or, when staging
// was full, into the request itself (they then travel through the arena's
// mirror).  Runs without stage_mu: the range is this request's until its
// batch has been uploaded, and the request is queued only after the copy, so
// several submitting threads copy at once.
void fill_stage(vd_server *s, Req *r, const void *llr, size_t value_bytes) {
    if (r->stage_bytes) memcpy(s->h_stage + r->stage_off, llr, value_bytes);
    else r->llr.assign((const uint8_t *)llr, (const uint8_t *)llr + value_bytes);
}

// Queues built requests (one lock) and wakes the worker.
void enqueue(vd_server *s, Req *const *rs, int64_t n) {
    const int64_t t = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int64_t i = 0; i < n; ++i) {
            rs[i]->submit_ns = t;
            s->pending.push_back(rs[i]);
        }
        s->stats.submitted += n;
    }
    s->cv.notify_all();
}

vd_status submit_common(vd_server *s, int code_id, int llr_type, const void *llr, bool device,
                        int64_t n_values, int64_t n_info, uint32_t flags, uint64_t tag) {
    Req *r = nullptr;
    size_t vb = 0;
    const vd_status st = make_req(s, code_id, llr_type, llr, device, n_values, n_info, flags, tag, &r, &vb);
    if (st != VD_OK) return st;
    if (!device) {
        {
            std::lock_guard<std::mutex> lk(s->stage_mu);
            reserve_stage(s, r, vb);
        }
        fill_stage(s, r, llr, vb);
    }
    enqueue(s, &r, 1);
    return VD_OK;
}

// n packets (values at llr + llr_offset[i] bytes; host memory, or device
// memory read in place) with one staging lock and one queue lock; packet k
// is index[k] of the arrays (k without an index).  Checks every packet
// first: on an error nothing is queued.
vd_status submit_many(vd_server *s, bool device, int64_t n, const int32_t *code_id, const int32_t *llr_type,
                      const void *host_llr, const int64_t *llr_offset, const int64_t *n_values,
                      const int64_t *n_info, const uint32_t *flags, const uint64_t *tags, const int64_t *index) {
    std::vector<Req *> rs((size_t)n, nullptr);
    std::vector<size_t> vb((size_t)n, 0);
    const uint8_t *base = (const uint8_t *)host_llr;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t i = index ? index[k] : k;
        const vd_status st = make_req(s, code_id[i], llr_type[i], base + llr_offset[i], device, n_values[i],
                                      n_info[i], flags[i], tags ? tags[i] : (uint64_t)i, &rs[(size_t)k],
                                      &vb[(size_t)k]);
        if (st != VD_OK) {
            for (int64_t j = 0; j < k; ++j) delete rs[(size_t)j];
            return st;
        }
    }
    if (!device) {
        {
            std::lock_guard<std::mutex> lk(s->stage_mu);
            for (int64_t k = 0; k < n; ++k) reserve_stage(s, rs[(size_t)k], vb[(size_t)k]);
        }
        for (int64_t k = 0; k < n; ++k) {
            const int64_t i = index ? index[k] : k;
            fill_stage(s, rs[(size_t)k], base + llr_offset[i], vb[(size_t)k]);
        }
    }
    enqueue(s, rs.data(), n);
    return VD_OK;
}

}  // namespace

extern "C" vd_status vd_server_submit(vd_server *s, int code_id, int llr_type, const void *host_llr,
                                      int64_t n_values, int64_t n_info, uint32_t flags, uint64_t tag) {
    return submit_common(s, code_id, llr_type, host_llr, false, n_values, n_info, flags, tag);
}

extern "C" vd_status vd_server_submit_many(vd_server *s, int64_t n, const int32_t *code_id,
                                           const int32_t *llr_type, const void *host_llr,
                                           const int64_t *llr_offset, const int64_t *n_values,
                                           const int64_t *n_info, const uint32_t *flags, const uint64_t *tags) {
    if (!s) return fail(VD_EINVAL, "server is NULL");
    if (n < 0) return fail(VD_EINVAL, "n < 0");
    if (n == 0) return VD_OK;
    if (!code_id || !llr_type || !host_llr || !llr_offset || !n_values || !n_info || !flags || !tags)
        return fail(VD_EINVAL, "a packet array is NULL");
    return submit_many(s, false, n, code_id, llr_type, host_llr, llr_offset, n_values, n_info, flags, tags,
                       nullptr);
}

extern "C" vd_status vd_server_submit_device(vd_server *s, int code_id, int llr_type, const void *d_llr,
                                             int64_t n_values, int64_t n_info, uint32_t flags, uint64_t tag) {
    return submit_common(s, code_id, llr_type, d_llr, true, n_values, n_info, flags, tag);
}

extern "C" int64_t vd_server_poll(vd_server *s, vd_completion *comp, int64_t max_completions,
                                  uint32_t *words, int64_t words_cap) {
    if (!s || !comp || max_completions <= 0) return 0;
    int64_t n = 0, w = 0;
    std::lock_guard<std::mutex> lk(s->mu);
    while (!s->done_q.empty() && n < max_completions) {
        Req *r = s->done_q.front();
        const int64_t nw = (int64_t)r->out_words;
        if (words && w + nw > words_cap) break;
        vd_completion &c = comp[n++];
        c.tag = r->tag;
        c.status = s->error.load() ? VD_ECUDA : VD_OK;
        c.n_words = (int32_t)nw;
        c.word_offset = w;
        c.submit_ns = r->submit_ns;
        c.admit_ns = r->admit_ns;
        c.done_ns = r->done_ns;
        if (words) memcpy(words + w, r->llr.data(), (size_t)nw * 4);
        w += nw;
        s->done_q.pop_front();
        delete r;
    }
    return n;
}

extern "C" vd_status vd_server_stats_get(vd_server *s, vd_server_stats *out) {
    if (!s || !out) return fail(VD_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->pending = (int64_t)s->pending.size();
    out->arena_used = (int64_t)s->arena.used;
    out->error = s->error.load();
    return VD_OK;
}

extern "C" void vd_server_destroy(vd_server *s) {
    if (!s) return;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (auto &sl : s->slots)
        if (sl.st) cudaStreamSynchronize(sl.st);
    for (auto &sl : s->slots)
        for (Req *r : sl.reqs) delete r;
    free_server(s);
}

namespace {

constexpr int kReplayProducers = 4;   // submitting threads of a long replay
constexpr int kReplayGather = 256;    // packets a producer submits in one call at most

vd_status replay_core(vd_server *s, bool device, int64_t n, const int32_t *code_id, const int32_t *llr_type,
                      const void *host_llr, const int64_t *llr_offset, const int64_t *n_values,
                      const int64_t *n_info, const uint32_t *flags, const int64_t *arrival_ns,
                      int64_t timeout_ms, int64_t *latency_ns, uint32_t *words,
                      const int64_t *word_offset, int64_t *span_ns) {
    if (!s) return fail(VD_EINVAL, "server is NULL");
    if (n < 0) return fail(VD_EINVAL, "n < 0");
    if (n > 0 && (!code_id || !llr_type || !host_llr || !llr_offset || !n_values || !n_info || !flags ||
                  !arrival_ns || !latency_ns))
        return fail(VD_EINVAL, "a packet array is NULL");
    if (words && !word_offset) return fail(VD_EINVAL, "words given without word_offset");
    for (int64_t i = 1; i < n; ++i)
        if (arrival_ns[i] < arrival_ns[i - 1]) return fail(VD_EINVAL, "arrival_ns must be nondecreasing");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stats.submitted != s->stats.completed || !s->done_q.empty())
            return fail(VD_EINVAL, "replay needs an idle server (packets in flight or not polled)");
    }
    const int64_t cap_comp = 4096;
    const int64_t cap_words = cap_comp * ((int64_t)s->cfg.max_packet_bits + 31) / 32;
    std::vector<vd_completion> comp((size_t)cap_comp);
    std::vector<uint32_t> wbuf((size_t)cap_words);
    for (int64_t i = 0; i < n; ++i) latency_ns[i] = -1;
    const uint8_t *base = (const uint8_t *)host_llr;
    const int64_t t0 = now_ns();
    const int64_t deadline = timeout_ms > 0 ? t0 + timeout_ms * 1000000 : INT64_MAX;

    // Producers: packet i is submitted by thread i mod n_prod at its arrival
    // time.  Host packets are copied at submit, which several producers (as
    // from several receivers) share; device packets cost only the queue
    // insertion, which one producer does faster than several contending for
    // the queue lock.  This thread collects completions.
    const int n_prod = (!device && n >= 4096) ? kReplayProducers : 1;
    std::atomic<bool> abort{false};
    std::atomic<int> err{VD_OK};
    std::string err_msg;
    std::mutex err_mu;
    // Each producer submits, in one call, every packet of its share that has
    // arrived (up to kReplayGather at a time).
    auto producer = [&](int tid) {
        std::vector<int64_t> due;
        for (int64_t i = tid; i < n && !abort.load(std::memory_order_relaxed);) {
            for (;;) {
                const int64_t now = now_ns();
                const int64_t wait = arrival_ns[i] - (now - t0);
                if (wait <= 0) break;
                if (now > deadline || abort.load(std::memory_order_relaxed)) return;
                if (wait > 50000) std::this_thread::sleep_for(std::chrono::microseconds(20));
                else std::this_thread::yield();
            }
            due.clear();
            const int64_t now_rel = now_ns() - t0;
            while (i < n && arrival_ns[i] <= now_rel && (int64_t)due.size() < kReplayGather) {
                due.push_back(i);
                i += n_prod;
            }
            const vd_status st = submit_many(s, device, (int64_t)due.size(), code_id, llr_type, base, llr_offset,
                                             n_values, n_info, flags, nullptr, due.data());
            if (st != VD_OK) {
                std::lock_guard<std::mutex> lk(err_mu);
                if (err.load() == VD_OK) err_msg = vd_last_error();
                err.store(st);
                abort.store(true);
                return;
            }
        }
    };
    std::vector<std::thread> prods;
    for (int t = 0; t < n_prod; ++t) prods.emplace_back(producer, t);
    auto finish = [&](vd_status st) {
        abort.store(true);
        for (auto &th : prods) th.join();
        return st;
    };

    int64_t done = 0, first_submit = INT64_MAX, last_done = t0;
    while (done < n) {
        if (err.load() != VD_OK) {
            finish(VD_OK);
            return fail((vd_status)err.load(), "replay: submit failed: %s", err_msg.c_str());
        }
        if (now_ns() > deadline) {
            finish(VD_OK);
            if (span_ns) *span_ns = last_done - (first_submit == INT64_MAX ? t0 : first_submit);
            return fail(VD_ETIMEOUT, "replay: %lld of %lld packets done after %lld ms", (long long)done,
                        (long long)n, (long long)timeout_ms);
        }
        const int64_t k = vd_server_poll(s, comp.data(), cap_comp, wbuf.data(), cap_words);
        for (int64_t j = 0; j < k; ++j) {
            const vd_completion &c = comp[(size_t)j];
            const int64_t i = (int64_t)c.tag;
            if (i < 0 || i >= n) continue;
            if (c.status != VD_OK) {
                finish(VD_OK);
                return fail(VD_ECUDA, "replay: the device reported an error");
            }
            latency_ns[i] = c.done_ns - (t0 + arrival_ns[i]);   // from the scheduled arrival
            first_submit = std::min(first_submit, c.submit_ns);
            last_done = std::max(last_done, c.done_ns);
            if (words) memcpy(words + word_offset[i], wbuf.data() + c.word_offset, (size_t)c.n_words * 4);
            ++done;
        }
        if (k == 0) std::this_thread::sleep_for(std::chrono::microseconds(10));
    }
    finish(VD_OK);
    if (span_ns) *span_ns = n ? last_done - first_submit : 0;
    return VD_OK;
}

}  // namespace

extern "C" vd_status vd_server_replay(vd_server *s, int64_t n, const int32_t *code_id, const int32_t *llr_type,
                                      const void *host_llr, const int64_t *llr_offset, const int64_t *n_values,
                                      const int64_t *n_info, const uint32_t *flags, const int64_t *arrival_ns,
                                      int64_t timeout_ms, int64_t *latency_ns, uint32_t *words,
                                      const int64_t *word_offset, int64_t *span_ns) {
    return replay_core(s, false, n, code_id, llr_type, host_llr, llr_offset, n_values, n_info, flags, arrival_ns,
                       timeout_ms, latency_ns, words, word_offset, span_ns);
}

extern "C" vd_status vd_server_replay_device(vd_server *s, int64_t n, const int32_t *code_id,
                                             const int32_t *llr_type, const void *d_llr, const int64_t *llr_offset,
                                             const int64_t *n_values, const int64_t *n_info, const uint32_t *flags,
                                             const int64_t *arrival_ns, int64_t timeout_ms, int64_t *latency_ns,
                                             uint32_t *words, const int64_t *word_offset, int64_t *span_ns) {
    return replay_core(s, true, n, code_id, llr_type, d_llr, llr_offset, n_values, n_info, flags, arrival_ns,
                       timeout_ms, latency_ns, words, word_offset, span_ns);
}
