// Persistent decode: resident warps pull tasks of 32/L frame pairs from a
// global counter and run the stream kernel's frame-pair forward procedure on
// each, while tracing the previous task back.  Batches (many packets of one
// code kind in one launch): the host sorts every frame of every packet by
// length and pairs neighbours, longest first.  Long single streams
// (vd_decode): pair q is frames 2q and 2q+1.
#pragma once
#include "vd_stream.cuh"

namespace vd {

// Device-side packet descriptor (offsets are relative to the launch's arenas).
struct PacketDesc {
    int64_t llr_off;        // byte offset of the packet's int8 [T][beta] LLRs
    int64_t out_word_off;   // word offset of the packet's decoded bits
    int64_t n_info;
    int32_t f, v;
    uint32_t flags;         // VD_TERMINATED / VD_START_UNKNOWN; bit 31: LLRs in the internal arena;
                            // bit 30: llr_off is an absolute device address
    int32_t reserved;
};

constexpr uint32_t PKT_INTERNAL_LLR = 0x80000000u;
constexpr uint32_t PKT_ABS_LLR = 0x40000000u;   // llr_off is a device address (caller-owned LLRs)

// One frame pair: packet and frame index of each half (packet ~0u: no frame).
struct PairRef {
    uint32_t p0, s0, p1, s1;
};

struct BatchParams {
    const PacketDesc *pk;
    const PairRef *pairs;     // sorted; warp task t covers pairs [t * 32/L, (t+1) * 32/L)
    int64_t n_pairs, n_tasks;
    const int8_t *llr_user;   // the caller's arena (unpunctured int8 packets)
    const int8_t *llr_int;    // the internal arena (depunctured / unpacked packets)
    uint32_t *out;            // the caller's output arena
    int *counter;             // [0] task counter, [1] finished warps: zero at launch, zeroed by the last warp
    uint32_t *surv;           // per resident warp: 2 x wpad_cap x 32 x SW words
    int32_t wpad_cap;
    int *status;
    int32_t chained;          // host side: launched to overlap the kernel before it on the stream
};

template <int K>
__device__ __forceinline__ FrameTask packet_frame(const BatchParams &p, uint32_t pk, uint32_t s) {
    FrameTask t;
    if (pk == 0xFFFFFFFFu) {
        t = frame_task(p.llr_user, p.out, nullptr, 1, 0, 1, 1, 1, 0, 0);   // invalid frame
        return t;
    }
    const PacketDesc d = p.pk[pk];
    const uint32_t fl = d.flags & ~(PKT_INTERNAL_LLR | PKT_ABS_LLR);
    const int64_t T = d.n_info + ((fl & 1u) ? K - 1 : 0);
    const int64_t n_win = (d.n_info + d.f - 1) / d.f;
    const int8_t *llr = (d.flags & PKT_ABS_LLR) ? reinterpret_cast<const int8_t *>(d.llr_off)
                        : ((d.flags & PKT_INTERNAL_LLR) ? p.llr_int : p.llr_user) + d.llr_off;
    return frame_task(llr, p.out + d.out_word_off, nullptr, (int64_t)s, n_win, d.n_info, T, d.f, d.v, fl);
}

// Shared memory of the persistent kernels, in dynamic shared memory: the
// per-warp traceback staging (16-byte aligned, first), then NREC traceback
// records per thread.  Two records per thread when they fit the budget: the
// forward pass writes the next pair's record in place while the hook walks
// the previous one, so neither occupies registers.  The three-stage record
// form (ES = 3) stages 8 KB per warp and needs more than the 48 KB a block
// gets without opting in; the launchers opt in (cudaFuncSetAttribute).
template <int K, int BETA, uint64_t GENS, int L, bool RADIX4, int NT>
struct PersistentSmem {
    using Cfg = StreamCfg<K, BETA, GENS, L, RADIX4>;
    using Tb = Traceback<K, L, RADIX4, Cfg::NR, Cfg::NW, Cfg::ES>;
    static constexpr size_t STG_BYTES = (size_t)(NT / 32) * Tb::STAGE_WORDS * 4u;
    static constexpr size_t TB_BYTES = (size_t)NT * sizeof(TbState);
    static constexpr size_t BUDGET = (Cfg::ES == 3 ? 64u : 48u) * 1024u;
    static constexpr int NREC = (2 * TB_BYTES + STG_BYTES <= BUDGET) ? 2 : 1;
    static constexpr size_t BYTES = STG_BYTES + (size_t)NREC * TB_BYTES;
    static_assert(STG_BYTES % 16 == 0, "records follow the staging at a 16-byte boundary");
};

// The persistent decode loop.  Each resident warp pulls tasks of 32/L frame
// pairs from *counter; pair_of(pair index, ft) gives the two frames of a pair.
// While it runs the forward procedure of a task, the warp walks the previous
// task's traceback one group per chunk (the two tasks' survivors live in the
// two halves of the warp's scratch), so the traceback's latency hides behind
// forward work.  surv: per resident warp 2 x wpad_cap x 32 x SW words.
template <int K, int BETA, uint64_t GENS, int L, bool RADIX4, int NT, typename PairOf>
__device__ __forceinline__ void persistent_decode(int *counter, int64_t n_tasks, uint32_t *surv_all,
                                                  int32_t wpad_cap, int *status, PairOf &&pair_of) {
    constexpr int PPW = 32 / L;
    using Cfg = StreamCfg<K, BETA, GENS, L, RADIX4>;
    constexpr int SW = Cfg::SW;
    using Sm = PersistentSmem<K, BETA, GENS, L, RADIX4, NT>;
    using Tb = typename Sm::Tb;
    constexpr int NREC = Sm::NREC;
    extern __shared__ __align__(16) uint4 vd_dyn_smem[];
    auto stg = reinterpret_cast<uint32_t (*)[Tb::STAGE_WORDS]>(vd_dyn_smem);
    auto tbs = reinterpret_cast<TbState (*)[NT]>(reinterpret_cast<unsigned char *>(vd_dyn_smem) + Sm::STG_BYTES);
    const int wlane = (int)(threadIdx.x & 31u);
    const int group = wlane / L;
    const int lane = wlane % L;
    const unsigned gmask = (L == 32) ? 0xFFFFFFFFu : (((1u << L) - 1u) << (wlane & ~(L - 1)));
    const int grp_base = wlane & ~(L - 1);
    const int64_t gwarp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const size_t buf_words = (size_t)wpad_cap * 32u * (size_t)SW;
    uint32_t *surv = surv_all + (size_t)gwarp * 2u * buf_words;
    uint32_t *my_stg = stg[threadIdx.x >> 5];
    int cur = 0;   // record of the pair being traced back
    tbs[0][threadIdx.x].t0 = -1;
    tbs[0][threadIdx.x].tau_store = 0;
    tbs[0][threadIdx.x].slot = 0;
    tbs[0][threadIdx.x].R[0] = tbs[0][threadIdx.x].R[1] = 0;
    int buf = 0;
    while (true) {
        int t = 0;
        if (wlane == 0) t = atomicAdd(counter, 1);
        t = __shfl_sync(0xFFFFFFFFu, t, 0);
        if (t >= n_tasks) break;
        FrameTask ft[2];
        pair_of((int64_t)t * PPW + group, ft);
        TbState &pend = tbs[cur][threadIdx.x];
        typename Tb::Live live;
        if constexpr (NREC == 2) {
            TbState &next = tbs[cur ^ 1][threadIdx.x];
            forward_pair<K, BETA, GENS, L, RADIX4>(
                ft, surv + (size_t)buf * buf_words, wpad_cap, wlane, lane, gmask, grp_base, status, next,
                [&](auto Sc, int c) {
                    Tb::template sub<decltype(Sc)::value, Cfg::U>(pend, my_stg, live, wlane, lane, gmask,
                                                                  grp_base, c);
                });
            Tb::drain(pend, my_stg, wlane, lane, gmask, grp_base);
            cur ^= 1;
        } else {
            TbState tb;
            forward_pair<K, BETA, GENS, L, RADIX4>(
                ft, surv + (size_t)buf * buf_words, wpad_cap, wlane, lane, gmask, grp_base, status, tb,
                [&](auto Sc, int c) {
                    Tb::template sub<decltype(Sc)::value, Cfg::U>(pend, my_stg, live, wlane, lane, gmask,
                                                                  grp_base, c);
                });
            Tb::drain(pend, my_stg, wlane, lane, gmask, grp_base);
            pend = tb;
        }
        TbState &now = tbs[cur][threadIdx.x];
        if (Tb::active(now)) Tb::begin(now, my_stg, wlane);
        buf ^= 1;
        __syncwarp();
    }
    Tb::drain(tbs[cur][threadIdx.x], my_stg, wlane, lane, gmask, grp_base);
}

// Batches: pairs come from the plan's sorted work list of packet frames.  The
// loop is spelled out here rather than through persistent_decode: the two
// forms decode identically, and this one compiles to fewer spills.
template <int K, int BETA, uint64_t GENS, int L, bool RADIX4, int NT>
__global__ void __launch_bounds__(NT, (K <= 7 ? 3 : 2)) batch_kernel(const BatchParams p) {
    constexpr int PPW = 32 / L;
    using Cfg = StreamCfg<K, BETA, GENS, L, RADIX4>;
    constexpr int SW = Cfg::SW;
    using Sm = PersistentSmem<K, BETA, GENS, L, RADIX4, NT>;
    using Tb = typename Sm::Tb;
    constexpr int NREC = Sm::NREC;
    extern __shared__ __align__(16) uint4 vd_dyn_smem[];
    auto stg = reinterpret_cast<uint32_t (*)[Tb::STAGE_WORDS]>(vd_dyn_smem);
    auto tbs = reinterpret_cast<TbState (*)[NT]>(reinterpret_cast<unsigned char *>(vd_dyn_smem) + Sm::STG_BYTES);
    const int wlane = (int)(threadIdx.x & 31u);
    const int group = wlane / L;
    const int lane = wlane % L;
    const unsigned gmask = (L == 32) ? 0xFFFFFFFFu : (((1u << L) - 1u) << (wlane & ~(L - 1)));
    const int grp_base = wlane & ~(L - 1);
    const int64_t gwarp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
    const size_t buf_words = (size_t)p.wpad_cap * 32u * (size_t)SW;
    uint32_t *surv = p.surv + (size_t)gwarp * 2u * buf_words;
    uint32_t *my_stg = stg[threadIdx.x >> 5];
    int cur = 0;   // record of the pair being traced back
    tbs[0][threadIdx.x].t0 = -1;
    tbs[0][threadIdx.x].tau_store = 0;
    tbs[0][threadIdx.x].slot = 0;
    tbs[0][threadIdx.x].R[0] = tbs[0][threadIdx.x].R[1] = 0;
    int buf = 0;
    // A chained launch (programmatic dependent launch) may start while the
    // kernel before it on the stream still runs.  Each warp waits for that
    // kernel to complete before its first output word (the traceback of its
    // first task) and only then lets the next kernel start, so outputs of
    // consecutive launches land in stream order and a launch never overlaps
    // the one two back, whose scratch and counters it shares.  Without a
    // chained launch the wait returns at once and the release does nothing.
    bool dep_waited = false;
    while (true) {
        int t = 0;
        if (wlane == 0) t = atomicAdd(p.counter, 1);
        t = __shfl_sync(0xFFFFFFFFu, t, 0);
        if (t >= p.n_tasks) break;
        const int64_t pi = (int64_t)t * PPW + group;
        FrameTask ft[2];
        if (pi < p.n_pairs) {
            const PairRef r = p.pairs[pi];
            ft[0] = packet_frame<K>(p, r.p0, r.s0);
            ft[1] = packet_frame<K>(p, r.p1, r.s1);
        } else {
            ft[0] = packet_frame<K>(p, 0xFFFFFFFFu, 0);
            ft[1] = ft[0];
        }
        TbState &pend = tbs[cur][threadIdx.x];
        typename Tb::Live live;
        if (!dep_waited && Tb::active(pend)) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            dep_waited = true;
            // the next launch may start as soon as every block has got here:
            // its blocks then take the SMs this launch's blocks leave, the
            // moment they leave them
            asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        }
        if constexpr (NREC == 2) {
            TbState &next = tbs[cur ^ 1][threadIdx.x];
            forward_pair<K, BETA, GENS, L, RADIX4>(
                ft, surv + (size_t)buf * buf_words, p.wpad_cap, wlane, lane, gmask, grp_base, p.status, next,
                [&](auto Sc, int c) {
                    Tb::template sub<decltype(Sc)::value, Cfg::U>(pend, my_stg, live, wlane, lane, gmask,
                                                                  grp_base, c);
                });
            Tb::drain(pend, my_stg, wlane, lane, gmask, grp_base);
            cur ^= 1;
        } else {
            TbState tb;
            forward_pair<K, BETA, GENS, L, RADIX4>(
                ft, surv + (size_t)buf * buf_words, p.wpad_cap, wlane, lane, gmask, grp_base, p.status, tb,
                [&](auto Sc, int c) {
                    Tb::template sub<decltype(Sc)::value, Cfg::U>(pend, my_stg, live, wlane, lane, gmask,
                                                                  grp_base, c);
                });
            Tb::drain(pend, my_stg, wlane, lane, gmask, grp_base);
            pend = tb;
        }
        TbState &now = tbs[cur][threadIdx.x];
        if (Tb::active(now)) Tb::begin(now, my_stg, wlane);
        buf ^= 1;
        __syncwarp();
    }
    if (!dep_waited) asm volatile("griddepcontrol.wait;" ::: "memory");
    if (wlane == 0) {
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        // the last warp to run out of tasks zeroes the counters for the next
        // launch that uses them (no warp of this launch takes a task after it)
        const int total = (int)(gridDim.x * (NT / 32));
        if (atomicAdd(p.counter + 1, 1) == total - 1) {
            atomicExch(p.counter, 0);
            atomicExch(p.counter + 1, 0);
        }
    }
    Tb::drain(tbs[cur][threadIdx.x], my_stg, wlane, lane, gmask, grp_base);
}

// One long stream (vd_decode): pair q is frames 2q and 2q+1 of the stream.
// counter and n_tasks come in through StreamParams; p.surv holds the
// persistent warps' double buffers (p.wpad_max stages each).
template <int K, int BETA, uint64_t GENS, int L, bool RADIX4, int NT>
__global__ void __launch_bounds__(NT, (K <= 7 ? 3 : 2)) stream_persistent_kernel(const StreamParams p) {
    constexpr int NS = 1 << (K - 1);
    persistent_decode<K, BETA, GENS, L, RADIX4, NT>(
        p.counter, p.n_tasks, p.surv, p.wpad_max, p.status, [=](int64_t q, FrameTask (&ft)[2]) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t s = 2 * q + h;
                ft[h] = frame_task(p.llr, p.out, p.pm_out ? p.pm_out + s * NS : nullptr, s, p.n_win, p.n_info,
                                   p.T, p.f, p.v, p.flags);
            }
        });
}

}  // namespace vd
