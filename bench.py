#!/usr/bin/env python3
"""Throughput benchmark of the GB300 Viterbi decoder.

Default workload: the segmented stream decode of the (2,1,7) 171/133 code
with int8 LLRs — six streams of 2^24 information bits (BPSK/AWGN at Eb/N0 =
1..6 dB), frames of f = 256 stages with v = 42 stages of overlap on each side.
One step decodes all six streams (6 x 2^24 bits); the inputs (6 x 32 MiB)
stay resident and each step cycles through 192 MiB of LLRs, more than the L2.

Prints one JSON line (rank 0).  ``--impl reference`` times the plain CPU
oracle on the same workload instead (a bounded sample per step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "decoded Gbit/s, K=7 r1/2 int8 LLR, batched vs plain; p99 packet latency"
N_INFO = 1 << 24
F, V = 256, 42
EBN0S = (1.0, 2.0, 3.0, 4.0, 5.0, 6.0)
K, BETA = 7, 2
PLAIN_STREAMS = 32


def workload_config(radix, lanes, path="batch"):
    paths = {"batch": "one persistent batched launch per step, chained (vd_batch_plan_launch_chained: a "
                      "step's kernel starts while the previous step's kernel finishes its last tasks and "
                      "tracebacks; each waits for the one before it before writing output)",
             "stream": "one vd_decode launch per stream",
             "oracle": "CPU oracle (int64 radix-2), bounded sample of one stream per step"}
    return {"workload": "segmented stream decode, K=7 r1/2 (171,133), 6 streams x 2^24 info bits, "
                        "Eb/N0 1..6 dB, f=256, v=42, int8 LLR",
            "n_info_per_stream": N_INFO, "streams_per_step": len(EBN0S), "f": F, "v": V,
            "radix": radix, "lanes": lanes, "path": paths[path],
            "l2": "inputs larger than L2 (192 MiB cycled per step)"}


def stream_plan(vd, code, n_streams, radix, lanes, stream, first=0):
    """Streams first .. first+n_streams-1 of the arena as the packets of one
    batch plan (f=256, v=42); offsets are into the whole arena."""
    tune = vd.VdTune()
    tune.radix = radix
    tune.lanes = lanes
    idx = np.arange(first, first + n_streams, dtype=np.int64)
    pk = {"code_id": np.zeros(n_streams, np.int32), "llr_type": np.zeros(n_streams, np.int32),
          "llr_offset": idx * BETA * N_INFO,
          "n_info": np.full(n_streams, N_INFO, np.int64), "flags": np.zeros(n_streams, np.uint32),
          "f": np.full(n_streams, F, np.int32), "v": np.full(n_streams, V, np.int32),
          "out_word_offset": idx * (N_INFO // 32)}
    return vd.BatchPlan([code], pk, tune=tune, stream=stream)


def ops_per_bit(f=F, v=V, k=K):
    """Algorithmic ACS operations per decoded bit: 2 adds + 1 compare-select per
    state per trellis stage, over f + 2v stages per f decoded bits."""
    return 3 * (1 << (k - 1)) * (f + 2 * v) / f


def kernel_source_hash():
    """Hash of the decode kernels' code (comments and blank lines dropped): a
    traffic figure measured on other code does not describe this kernel."""
    import hashlib
    h = hashlib.sha256()
    for f in ("paper_2011_13579_gb300/csrc/vd_stream.cuh", "paper_2011_13579_gb300/csrc/vd_device.cuh",
              "paper_2011_13579_gb300/csrc/vd_batch.cuh"):
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            for line in fh:
                code = line.split("//", 1)[0].strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sms)}


# --------------------------------------------------------------- CPU oracle

def cpu_oracle_run(seconds_budget=15.0, threads=None):
    """The plain oracle on a bounded sample of the workload: one 2^24-bit stream
    (Eb/N0 = 3 dB), or a prefix of it sized to the time budget."""
    import oracle
    from paper_2011_13579_gb300 import synth
    threads = threads or len(os.sched_getaffinity(0))
    code = oracle.Code(K, synth.K7_GENS)
    st = synth.segmented_stream(3.0)
    q = st.s8().reshape(-1, BETA).astype(np.int32)
    # calibrate on 2^16 bits, then size the sample to the budget
    n0 = 1 << 16
    t = time.perf_counter()
    oracle.decode(code, q[:n0], n0, F, V, threads=threads)
    rate = n0 / max(time.perf_counter() - t, 1e-6)
    n = int(min(N_INFO, max(n0, rate * seconds_budget)))
    n -= n % F
    t = time.perf_counter()
    oracle.decode(code, q[:n], n, F, V, threads=threads)
    dt = time.perf_counter() - t
    return {"value": n / dt / 1e9, "unit": "Gbit/s", "cores": threads, "kind": "oracle",
            "sample": f"{n} info bits of the Eb/N0=3 dB stream, f=256 v=42, int64 radix-2 oracle, "
                      f"{threads} threads, {dt:.1f} s"}


# ------------------------------------------------------------------- GPU

def whole_job_value(ms_local, bits_per_rank_step, steps, world, device=None):
    """Whole-job throughput (Gbit/s) of `world` replicas: every rank's bits over
    the slowest rank's time, taken with a MAX all-reduce.  Returns (ms, value)."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, bits_per_rank_step * steps * world / (ms / 1e3) / 1e9


def run_gpu(args, rank, world):
    import torch
    import torch.distributed as dist
    import paper_2011_13579_gb300 as vd
    from paper_2011_13579_gb300 import synth

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    code = vd.Code(K, synth.K7_GENS)
    streams = []
    for e in EBN0S:
        st = synth.segmented_stream(e)
        streams.append(st.s8().view(np.uint8))
    nw = N_INFO // 32
    arena = torch.from_numpy(np.concatenate(streams)).to(dev)
    out_arena = torch.empty(nw * len(streams), dtype=torch.int32, device=dev)
    llr_dev = [arena[i * BETA * N_INFO:(i + 1) * BETA * N_INFO] for i in range(len(streams))]
    outs = [out_arena[i * nw:(i + 1) * nw] for i in range(len(streams))]
    s = torch.cuda.Stream(dev)
    tune = None
    if args.lanes:
        tune = vd.VdTune()
        tune.lanes = args.lanes
    flags = 0
    plan = stream_plan(vd, code, len(streams), args.radix, args.lanes, s) if args.path == "batch" else None
    shape = {"radix": args.radix, "lanes": args.lanes}
    if plan is not None:
        info = plan.info()   # lanes chosen by the plan's measured autotuner when --lanes is 0
        shape = {"radix": int(info.radix), "lanes": int(info.lanes)}

    def one_launch(i, chained=True):
        """Launch i of a step: one stream, or the whole batch (chained: the
        step's kernel may start while the previous step's kernel finishes its
        last tasks and tracebacks, vd_batch_plan_launch_chained)."""
        if plan is not None:
            plan.launch(arena, out_arena, stream=s, chained=chained)
        else:
            vd.vd_decode(code.handle, llr_dev[i], vd.VD_LLR_S8, N_INFO, F, V, args.radix, flags,
                         outs[i], None, tune, s)

    launches_per_step = 1 if plan is not None else len(streams)

    def step():
        for i in range(launches_per_step):
            one_launch(i)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()

    sampler = ClockSampler(dev.index) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    # per-launch events on the launching stream, for the kernel's own
    # duration; chained batch launches overlap their neighbours, and an event
    # between two of them would end the overlap, so those are timed over the
    # whole region (its time / launches) and, after it, once more one by one
    # as ordinary launches ("isolated_launch_ms")
    chained = plan is not None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps * launches_per_step)]
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(s)
    k = 0
    for _ in range(args.steps):
        for i in range(launches_per_step):
            if not chained:
                ev[k][0].record(s)
            one_launch(i)
            if not chained:
                ev[k][1].record(s)
            k += 1
    t1.record(s)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ms = t0.elapsed_time(t1)
    launch_ms = [ms / k] * k if chained else [a.elapsed_time(b) for a, b in ev]
    clocks = sampler.stop() if sampler else None
    isolated_ms = None
    if chained:
        n_iso = min(k, 20)
        for e0, e1 in ev[:n_iso]:
            e0.record(s)
            one_launch(0, chained=False)
            e1.record(s)
        torch.cuda.synchronize(dev)
        isolated_ms = statistics.mean(a.elapsed_time(b) for a, b in ev[:n_iso])

    bits_per_step = N_INFO * len(streams)
    ms, value = whole_job_value(ms, bits_per_step, args.steps, world, dev)

    # end to end through the C ABI with host buffers: vd_decode_host uploads
    # each stream from pinned host memory, decodes it (the persistent batch
    # kernel, two decode streams) and downloads its words, all inside the timed
    # region; stream i+1's upload overlaps stream i's decode.
    host_in = [torch.from_numpy(x).pin_memory() for x in streams]
    host_out = [torch.empty(nw, dtype=torch.int32).pin_memory() for _ in streams]
    e2e_steps = max(1, min(args.steps, 5))
    radix_e2e = shape["radix"]
    vd.vd_decode_host(code.handle, host_in, N_INFO, F, V, radix_e2e, flags, host_out, stream=s)   # set-up
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(e2e_steps):
        vd.vd_decode_host(code.handle, host_in, N_INFO, F, V, radix_e2e, flags, host_out, stream=s)
    e1.record(s)
    torch.cuda.synchronize(dev)
    vd.vd_sync(s)
    e2e_ms = e0.elapsed_time(e1)
    e2e_value = bits_per_step * e2e_steps / (e2e_ms / 1e3) / 1e9
    h2d = sum(int(x.size) for x in streams)
    d2h = nw * 4 * len(streams)
    e2e_same = all(torch.equal(host_out[i], outs[i].cpu()) for i in range(len(streams)))

    # sanity: the decode of the 6 dB stream is nearly error-free
    dec = outs[-1].cpu().numpy().view(np.uint32)
    bits = ((dec[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8).reshape(-1)
    ref_bits = synth.segmented_stream(6.0).bits
    ber6 = float(np.mean(bits != ref_bits))

    # decoded words of every stream, radix 2 (the timed plan's last run) and
    # radix 4 (one launch of a radix-4 plan), for the segmentation-BER leg
    words_r2 = words_r4 = None
    if plan is not None and rank == 0 and world == 1 and not args.no_ber:
        words_r2 = [o.cpu().numpy().view(np.uint32).copy() for o in outs]
        p4 = stream_plan(vd, code, len(streams), 4, 0, s)
        p4.launch(arena, out_arena, stream=s)
        torch.cuda.synchronize(dev)
        p4.status(stream=s)
        words_r4 = [o.cpu().numpy().view(np.uint32).copy() for o in outs]
        p4.close()

    if plan is not None:
        plan.close()
    packets = None
    if rank == 0 and args.packets > 0:
        packets = run_packets(args, dev, s)
    return {"shape": shape, "packets": packets, "ms": ms, "value": value, "launch_ms": launch_ms,
            "isolated_launch_ms": isolated_ms, "chained": chained, "clocks": clocks,
            "words_r2": words_r2, "words_r4": words_r4,
            "launches_per_step": launches_per_step, "bits_per_launch": bits_per_step // launches_per_step,
            "e2e": {"value": e2e_value, "unit": "Gbit/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "same_bits_as_device_run": bool(e2e_same),
                    "form": "one vd_decode_host call per step (C ABI, pinned host buffers): per stream an "
                            "upload, one persistent batch launch and a download, uploads overlapping decodes"},
            "ber_6db": ber6, "n_sm": torch.cuda.get_device_properties(dev).multi_processor_count}


def run_packets(args, dev, s):
    """Batched persistent decode vs one launch per packet on the uneven-packet
    workload: 65,536 terminated K=7 packets, log-uniform 96..12,000 info bits,
    r1/2, r2/3, r3/4 in equal shares, Eb/N0 ~ U(2, 7) dB, int8 kept LLRs.
    The batched form is one autotuned plan replayed from a CUDA graph; the
    plain form is one vd_decode call per packet at the f/v/radix the plan
    chose, so both must give the same bits."""
    import ctypes
    import torch
    import paper_2011_13579_gb300 as vd
    from paper_2011_13579_gb300 import synth

    batch = synth.uneven_packets(args.packets)
    pats = (None, synth.PUNCT_R23, synth.PUNCT_R34)
    codes = [vd.Code(K, synth.K7_GENS, puncture=None if p is None else p.tolist()) for p in pats]
    n = batch.n_packets
    pk = {"code_id": batch.rate_id.astype(np.int32), "llr_type": np.zeros(n, np.int32),
          "llr_offset": batch.llr_offset, "n_info": batch.n_info,
          "flags": np.full(n, vd.VD_TERMINATED, np.uint32), "f": np.zeros(n, np.int32),
          "v": np.zeros(n, np.int32), "out_word_offset": batch.out_word_offset}
    plan = vd.BatchPlan(codes, pk, stream=s)
    info = plan.info()
    f, v = plan.packet_tune()
    llr = torch.from_numpy(batch.llr_s8.view(np.uint8)).to(dev)
    nw = int(batch.out_word_offset[-1] + (batch.n_info[-1] + 31) // 32)
    out_b = torch.empty(nw, dtype=torch.int32, device=dev)
    out_p = torch.full((nw,), -1, dtype=torch.int32, device=dev)
    bits = int(batch.n_info.sum())

    for _ in range(max(3, args.warmup)):
        plan.launch(llr, out_b, stream=s, graph=True)
    torch.cuda.synchronize(dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    reps = max(3, min(args.steps, 50))
    a.record(s)
    for _ in range(reps):
        plan.launch(llr, out_b, stream=s, graph=True)
    b.record(s)
    torch.cuda.synchronize(dev)
    ms_b = a.elapsed_time(b) / reps
    plan.status(stream=s)

    # plain: one vd_decode per packet (raw pointers, the library's default kernel
    # shape), round-robin over PLAIN_STREAMS streams so independent packets overlap
    L = vd.lib()
    llr_base, out_base = llr.data_ptr(), out_p.data_ptr()
    handles = [c.handle for c in codes]
    side = [torch.cuda.Stream(dev) for _ in range(PLAIN_STREAMS)]
    shs = [ctypes.c_void_p(x.cuda_stream) for x in side]
    radix = int(info.radix)
    order = np.argsort(-batch.n_info, kind="stable")   # warm-up: largest first sizes the scratch once

    def plain_pass(idx):
        for k, i in enumerate(idx):
            st = L.vd_decode(ctypes.c_void_p(handles[batch.rate_id[i]]),
                             ctypes.c_void_p(llr_base + int(batch.llr_offset[i])), vd.VD_LLR_S8,
                             int(batch.n_info[i]), int(f[i]), int(v[i]), radix, vd.VD_TERMINATED,
                             ctypes.c_void_p(out_base + 4 * int(batch.out_word_offset[i])), None, None,
                             shs[k % PLAIN_STREAMS])
            if st != 0:
                raise RuntimeError(f"vd_decode failed on packet {i}: {L.vd_last_error().decode()}")

    plain_pass(np.repeat(order[:4], PLAIN_STREAMS))   # every stream's scratch sized by the largest packets
    torch.cuda.synchronize(dev)
    a.record(s)
    for x in side:
        x.wait_event(a)
    plain_pass(range(n))
    for x in side:
        e = torch.cuda.Event()
        e.record(x)
        s.wait_event(e)
    b.record(s)
    torch.cuda.synchronize(dev)
    ms_p = a.elapsed_time(b)
    for x in side:
        vd.vd_sync(x)
    identical = bool(torch.equal(out_b, out_p))

    # the same per-packet calls issued by the library's C loop (vd_decode_each)
    pk_each = dict(pk)
    pk_each["f"] = np.asarray(f, np.int32)
    pk_each["v"] = np.asarray(v, np.int32)
    out_c = torch.full((nw,), -1, dtype=torch.int32, device=dev)
    vd.vd_decode_each(codes, pk_each, llr, out_c, radix, side)   # warm-up (scratch already sized)
    torch.cuda.synchronize(dev)
    a.record(s)
    for x in side:
        x.wait_event(a)
    vd.vd_decode_each(codes, pk_each, llr, out_c, radix, side)
    for x in side:
        e = torch.cuda.Event()
        e.record(x)
        s.wait_event(e)
    b.record(s)
    torch.cuda.synchronize(dev)
    ms_c = a.elapsed_time(b)
    for x in side:
        vd.vd_sync(x)
    identical_c = bool(torch.equal(out_b, out_c))
    plan.close()
    return {"workload": f"{n} terminated K=7 packets, log-uniform 96..12000 info bits, r1/2 r2/3 r3/4 "
                        "equal shares, Eb/N0 U(2,7) dB, int8 kept LLRs",
            "info_bits": bits, "batched_gbps": bits / (ms_b / 1e3) / 1e9, "batched_ms": ms_b,
            "plain_gbps": bits / (ms_p / 1e3) / 1e9, "plain_ms": ms_p, "speedup": ms_p / ms_b,
            "identical_output": identical,
            "plain_c_loop_gbps": bits / (ms_c / 1e3) / 1e9, "plain_c_loop_ms": ms_c,
            "speedup_vs_c_loop": ms_c / ms_b, "identical_output_c_loop": identical_c,
            "batched_form": "one persistent launch per step (autotuned plan, CUDA-graph replay)",
            "plain_form": f"one vd_decode call per packet, same f/v/radix, round-robin over {PLAIN_STREAMS} "
                          "CUDA streams (as many hardware queues), issued from Python via ctypes; "
                          "plain_c_loop: the same calls issued by the library's C loop (vd_decode_each)",
            "tune": {"radix": radix, "lanes": int(info.lanes), "resident_warps": int(info.resident_warps),
                     "f_median": int(np.median(f)), "v_median": int(np.median(v))}}


def run_serving(args, device_resident=False):
    """Continuous-batching server under open-loop Poisson load.  A pool of
    serving packets (payloads U{40..1500} bytes; 80% K=7 171/133, half of
    those punctured to r3/4; 20% K=9 557/663/711; Eb/N0 U(1, 6) dB; int8;
    terminated) is first replayed all at once to measure the server's peak
    packet rate; then for each offered load x the packets arrive as a Poisson
    process of rate x * peak (the aggregate of 256 streams), cycling through
    the pool.  Latency is from a packet's scheduled arrival time to the
    server seeing its batch complete (host steady clock).
    device_resident: the pool's values are uploaded once and submitted in
    place (vd_server_submit_device), as from an upstream GPU stage."""
    import torch
    import paper_2011_13579_gb300 as vd
    from paper_2011_13579_gb300 import synth

    pool = synth.serving_packets(args.serving_pool, index=0)
    fl = synth.flatten_packets(pool)
    n = len(pool)
    codes = [vd.Code(Kc, gens, puncture=None if pat is None else pat.tolist())
             for (Kc, gens, pat) in synth.SERVING_CODES]
    server = vd.Server(codes)
    src = torch.from_numpy(fl["llr"].view(np.uint8)).cuda() if device_resident else fl["llr"]
    types = np.zeros(n, np.int32)
    flags = np.full(n, vd.VD_TERMINATED, np.uint32)
    # warm-up, then the closed-loop peak (every packet offered at t = 0)
    server.replay(fl["code_id"][:256], types[:256], src, fl["llr_offset"][:256], fl["n_values"][:256],
                  fl["n_info"][:256], flags[:256], np.zeros(256, np.int64), timeout_ms=120000)
    _, ref_words, span = server.replay(fl["code_id"], types, src, fl["llr_offset"], fl["n_values"],
                                       fl["n_info"], flags, np.zeros(n, np.int64), timeout_ms=300000,
                                       word_offset=fl["word_offset"])
    pool_bits = int(fl["n_info"].sum())
    peak_pps = n / (span / 1e9)
    points = []
    rng = np.random.Generator(np.random.PCG64(2011135790 + 500))
    consistent = True
    for x in args.serving_loads:
        rate = x * peak_pps
        m = int(min(max(n, rate * args.serving_seconds), args.serving_max_packets))
        idx = np.arange(m) % n
        arr = synth.poisson_arrivals(rng, m, rate)
        lat, words, span = server.replay(fl["code_id"][idx], types[idx], src, fl["llr_offset"][idx],
                                         fl["n_values"][idx], fl["n_info"][idx], flags[idx], arr,
                                         timeout_ms=600000, word_offset=fl["word_offset"][idx])
        consistent &= bool(np.array_equal(words[:ref_words.size], ref_words))
        bits = int(fl["n_info"][idx].sum())
        points.append({"offered": x, "packets": m, "offered_pps": rate,
                       "gbps": bits / (span / 1e9) / 1e9,
                       "p50_ms": float(np.percentile(lat, 50)) / 1e6,
                       "p99_ms": float(np.percentile(lat, 99)) / 1e6})
    st = server.stats()
    server.close()
    return {"submission": "device-resident values, submitted in place" if device_resident
            else "host values, copied at submit",
            "workload": f"pool of {n} packets, payload U(40..1500) B, 80% K=7 r1/2 (half punctured to r3/4), "
                        "20% K=9 r1/3, Eb/N0 U(1,6) dB, int8, terminated; Poisson arrivals (256 streams "
                        "aggregated) at x * peak",
            "peak_pps": peak_pps, "peak_gbps": pool_bits / (n / peak_pps) / 1e9,
            "points": points, "same_bits_at_every_load": consistent, "batches": int(st.batches),
            "latency": "scheduled arrival -> batch completion seen by the server (host steady clock)"}


def run_bm_gate(dev, s):
    """Branch metrics (Eq. BM) of the (2,1,7) code on CUDA cores vs tensor cores
    (mma.sync m16n8k32 s8 plus a transpose into the decoder's layout), on an
    L2-resident LLR block: 3 x 128 threads per SM x 152 SMs of frame pairs x
    256 stages.  Both kernels fold the same metrics into the same checksum."""
    import torch
    import paper_2011_13579_gb300 as vd
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    n_pairs, n_stages = n_sm * 3 * 128, 256
    rng = np.random.Generator(np.random.PCG64(2011135790 + 700))
    words = torch.from_numpy(rng.integers(0, 2 ** 32, size=n_pairs * n_stages, dtype=np.uint64)
                             .astype(np.uint32).view(np.int32)).to(dev)
    res = {}
    sums = []
    for variant, name in ((0, "cuda_core"), (1, "tensor_core_mma_sync")):
        cs = torch.zeros(n_pairs, dtype=torch.int32, device=dev)
        for _ in range(3):
            vd.vd_bm_gate(variant, words, n_pairs, n_stages, cs, stream=s)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(20):
            vd.vd_bm_gate(variant, words, n_pairs, n_stages, cs, stream=s)
        b.record(s)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / 20
        res[name] = {"ms": ms, "ps_per_pair_stage": ms * 1e9 / (n_pairs * n_stages)}
        sums.append(cs.cpu().numpy())
    res["same_metrics"] = bool(np.array_equal(sums[0], sums[1]))
    res["tensor_over_cuda_time"] = res["tensor_core_mma_sync"]["ms"] / res["cuda_core"]["ms"]
    res["workload"] = f"{n_pairs} frame pairs x {n_stages} stages, int8 LLRs, L2-resident"
    return res


INT_PEAK_VARIANTS = (
    # (variant, name, instructions per body, algorithmic ops per body or None)
    (0, "add.u16x2", 8, None), (1, "max.u16x2", 8, None), (2, "add+max.u16x2 (fused)", 8, None),
    (3, "mad.lo.u32", 8, None), (4, "lop3.b32", 8, None), (5, "prmt.b32", 8, None),
    (6, "shf.l.wrap.b32", 8, None), (7, "add.u16x2 + mad.lo.u32 (1:1)", 8, None),
    (8, "add+max.u16x2 + mad.lo.u32 (1:1)", 8, None), (9, "max.u16x2 + lop3.b32 (1:1)", 8, None),
    (10, "radix-2 butterfly: 2 add.u16x2 + 2 add+max.u16x2", 16, 48),
)


# The SM pipe each single-class variant issues to, read once from ncu's
# sm__inst_executed_pipe_{alu,fmaheavy} counters on GB300 (profiles/int_peak_gb300.md):
# 16x2 add and 32-bit multiply-add on the FMA pipe; fused add-max, 16x2 max,
# three-input logic, byte permute and funnel shift on the ALU pipe.
INT_PEAK_PIPE = {0: "fma", 1: "alu", 2: "alu", 3: "fma", 4: "alu", 5: "alu", 6: "alu"}


def run_int_peak(dev, s, iters=2048):
    """Integer-issue rates on this GPU (vd_int_peak): per variant, thread-level
    operations per SM per SM-clock, from each block's clock64() span (one block
    of 1024 threads per SM, 8 chains per thread).  The roofline's peak lane
    rate is the ALU pipe's best single-class rate plus the FMA pipe's (the two
    pipes issue concurrently; the decoder's instructions all run on them); the
    butterfly variant is the ACS alone (12 algorithmic ops per 4
    instructions), and the 1:1 mixes show how close two classes get to the sum."""
    import torch
    import paper_2011_13579_gb300 as vd
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    cyc = torch.zeros(n_sm, dtype=torch.int64, device=dev)
    sink = torch.zeros(n_sm * 1024, dtype=torch.int32, device=dev)
    res = []
    for var, name, ipb, apb in INT_PEAK_VARIANTS:
        vd.vd_int_peak(var, 64, n_sm, cyc, sink, stream=s)      # warm-up
        vd.vd_int_peak(var, iters, n_sm, cyc, sink, stream=s)
        torch.cuda.synchronize(dev)
        c = cyc.cpu().numpy().astype(np.float64)
        ops = 1024.0 * iters * 16 * ipb                           # thread instructions per SM
        r = {"variant": var, "ops": name, "per_sm_per_clk": float(ops / np.median(c)),
             "cycles_median": float(np.median(c)), "cycles_max": float(np.max(c))}
        if apb:
            r["alg_ops_per_sm_per_clk"] = float(1024.0 * iters * 16 * apb / np.median(c))
        res.append(r)
    alu = max(r["per_sm_per_clk"] for r in res if INT_PEAK_PIPE.get(r["variant"]) == "alu")
    fma = max(r["per_sm_per_clk"] for r in res if INT_PEAK_PIPE.get(r["variant"]) == "fma")
    mix = max(r["per_sm_per_clk"] for r in res if r["variant"] in (7, 8, 9))
    return {"n_sm": n_sm, "iters": iters, "variants": res, "lanes_per_sm_per_clk": alu + fma,
            "alu_lanes_per_sm_per_clk": alu, "fma_lanes_per_sm_per_clk": fma,
            "best_two_class_mix_per_sm_per_clk": mix,
            "lanes_from": f"ALU pipe {alu:.1f} + FMA pipe {fma:.1f}",
            "butterfly_alg_ops_per_sm_per_clk": next(r["alg_ops_per_sm_per_clk"] for r in res
                                                     if r["variant"] == 10)}


def run_ber(args, outs_r2, outs_r4):
    """BER cost of segmentation on the bench's six 2^24-bit streams (Sec. III:
    frames trade BER for parallelism): per Eb/N0, the GPU's segmented decode
    (radix 2 and radix 4, which must agree bit for bit) against the true bits,
    the segmented oracle (bit-exactness) and the full-length oracle decode
    (one frame over the whole stream, one host thread per stream).  BER at or
    below 100/n is reported as "< floor"."""
    import concurrent.futures as cf
    import oracle
    from paper_2011_13579_gb300 import synth
    oracle.build()
    code = oracle.Code(K, synth.K7_GENS)
    threads = len(os.sched_getaffinity(0))
    floor = 100.0 / N_INFO
    streams = [synth.segmented_stream(e) for e in EBN0S]
    qs = [st.s8().reshape(-1, BETA).astype(np.int32) for st in streams]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=min(len(streams), threads)) as ex:
        fulls = list(ex.map(lambda q: oracle.unpack_bits(oracle.decode_full(code, q, N_INFO), N_INFO), qs))
    t_full = time.perf_counter() - t0

    def fmt(x):
        return x if x > floor else f"< {floor:.2e}"

    pts = []
    for e, st, q, full, g2, g4 in zip(EBN0S, streams, qs, fulls, outs_r2, outs_r4):
        seg = oracle.unpack_bits(oracle.decode(code, q, N_INFO, F, V, threads=threads), N_INFO)
        b2 = oracle.unpack_bits(g2, N_INFO)
        b4 = oracle.unpack_bits(g4, N_INFO)
        ber_full = float(np.mean(full != st.bits))
        ber_seg = float(np.mean(b2 != st.bits))
        pts.append({"ebn0_db": e, "ber_full_length_oracle": fmt(ber_full), "ber_segmented_gpu": fmt(ber_seg),
                    "ber_cost": ber_seg - ber_full,
                    "bits_differing_segmented_vs_full": int(np.count_nonzero(b2 != full)),
                    "gpu_radix2_equals_segmented_oracle": bool(np.array_equal(b2, seg)),
                    "gpu_radix4_equals_radix2": bool(np.array_equal(b4, b2))})
    return {"workload": "6 streams x 2^24 info bits, K=7 r1/2, f=256, v=42, int8 LLR, unterminated",
            "ber_floor": floor, "full_length_oracle_s": t_full, "points": pts}


def run_precision(args):
    """Precision study on the (3,1,9) 557/663/711 code: 2^24 information bits
    per Eb/N0 in 0..4 dB, f=512, v=64, decoded on the GPU three ways — int8 and
    4-bit LLRs with integer metrics (checked bit for bit against the int64
    oracle on the same values) and fp16 LLRs with fp32 metrics (disagreement
    with the FP64 oracle on the same fp16 values, every disagreeing frame
    checked against the tie margin) — and BER of each form against the true
    bits, with the FP64 oracle on the unquantised LLRs (2y/sigma^2) as the
    BER reference.  GPU throughput per form is the time of one vd_decode."""
    import torch
    import oracle
    import paper_2011_13579_gb300 as vd
    from paper_2011_13579_gb300 import synth
    oracle.build()
    n, f, v = args.precision_bits, 512, 64
    threads = len(os.sched_getaffinity(0))
    code = vd.Code(9, synth.K9_GENS)
    oc = oracle.Code(9, synth.K9_GENS)
    s = torch.cuda.Stream()
    points = []

    def gpu(buf, ltype, lanes):
        out = vd.decode(code, buf, n, f, v, llr_type=ltype, lanes=lanes, stream=s)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        vd.decode(code, buf, n, f, v, llr_type=ltype, lanes=lanes, stream=s, out=out)
        b.record(s)
        torch.cuda.synchronize()
        vd.vd_sync(s)
        return oracle.unpack_bits(out.cpu().numpy().view(np.uint32), n), n / (a.elapsed_time(b) / 1e3) / 1e9

    for e in args.precision_ebn0:
        st = synth.precision_stream(e, n_info=n)
        T = st.T
        pt = {"ebn0_db": e}
        ref = oracle.unpack_bits(oracle.decode_f64(oc, st.f64().reshape(T, 3), n, f, v, threads=threads)[0], n)
        ber_ref = float(np.mean(ref != st.bits))
        pt["ber_fp64_unquantised"] = ber_ref
        q8 = st.s8()
        g8, t8 = gpu(torch.from_numpy(q8.view(np.uint8)).cuda(), vd.VD_LLR_S8, 0)
        o8 = oracle.unpack_bits(oracle.decode(oc, q8.reshape(T, 3).astype(np.int32), n, f, v, threads=threads), n)
        pt["int8"] = {"gbps": t8, "bit_exact_vs_oracle": bool(np.array_equal(g8, o8)),
                      "ber": float(np.mean(g8 != st.bits)), "ber_delta": float(np.mean(g8 != st.bits)) - ber_ref}
        q4 = st.s4()
        g4, t4 = gpu(torch.from_numpy(synth.pack_s4(q4)).cuda(), vd.VD_LLR_S4, 0)
        o4 = oracle.unpack_bits(oracle.decode(oc, q4.reshape(T, 3).astype(np.int32), n, f, v, threads=threads), n)
        pt["int4"] = {"gbps": t4, "bit_exact_vs_oracle": bool(np.array_equal(g4, o4)),
                      "ber": float(np.mean(g4 != st.bits)), "ber_delta": float(np.mean(g4 != st.bits)) - ber_ref}
        h = st.f16()
        gh, th = gpu(torch.from_numpy(h.view(np.uint16)).cuda(), vd.VD_LLR_F16, 8)
        ow, gap, mx = oracle.decode_f64(oc, h.astype(np.float64).reshape(T, 3), n, f, v, threads=threads)
        oh = oracle.unpack_bits(ow, n)
        dis_frames, unexplained = 0, 0
        bad = np.nonzero(gh != oh)[0]
        frames = np.unique(bad // f)
        for fr in frames:
            a = max(0, fr * f - v)
            b = min(T, (fr + 1) * f + v)
            tau = 4.0 * (b - a) * 2.0 ** -24 * max(mx[fr], 1.0)
            dis_frames += 1
            unexplained += int(not gap[fr] <= tau)
        pt["fp16_fp32"] = {"gbps": th, "disagree_bits": int(bad.size), "disagree_rate": float(bad.size / n),
                           "disagree_frames": dis_frames, "frames_outside_tie_margin": unexplained,
                           "ber": float(np.mean(gh != st.bits)), "ber_delta": float(np.mean(gh != st.bits)) - ber_ref}
        points.append(pt)
        print(json.dumps(pt), file=sys.stderr, flush=True)
    # roofline of the forms (work = 2 adds + 1 compare-select per state and
    # stage): the integer forms against 128 lanes x 2 halves per SM and clock,
    # the fp32 form (one frame per 32-bit lane) against 128 lanes
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = float(load_peaks().get("sm_max_mhz", 2070.0))
    opb = ops_per_bit(f, v, 9)
    peak_int = n_sm * 128 * 2 * mhz * 1e6
    peak_f32 = n_sm * 128 * mhz * 1e6
    for pt in points:
        for form, peak in (("int8", peak_int), ("int4", peak_int), ("fp16_fp32", peak_f32)):
            pt[form]["roofline_frac"] = pt[form]["gbps"] * 1e9 * opb / peak
    return {"workload": f"K=9 r1/3 (557,663,711), {n} info bits per Eb/N0, f=512, v=64, unterminated",
            "ber_floor": 100.0 / n, "oracle_threads": threads, "ops_per_bit": opb,
            "roofline_peaks_tops": {"int": peak_int / 1e12, "fp32": peak_f32 / 1e12}, "points": points}


def run_tc(args):
    """The tensor-core radix-4 variant (vd_decode_tc, the paper's D = Theta_hat L
    + Lambda with dragonfly groups, Sec. VIII) on the bench workload: one
    launch per 2^24-bit stream, six per step, against the CUDA-core batch
    decode of the same streams (identical bits).  Roofline as the bench line
    (255 ACS ops per decoded bit against the integer-issue peak), plus the
    tensor operations it issues: 2 mma m16n8k16 per stage pair and frame."""
    import torch
    import paper_2011_13579_gb300 as vd
    from paper_2011_13579_gb300 import synth
    dev = torch.device("cuda", 0)
    code = vd.Code(K, synth.K7_GENS)
    streams = [synth.segmented_stream(e).s8().view(np.uint8) for e in EBN0S]
    nw = N_INFO // 32
    arena = torch.from_numpy(np.concatenate(streams)).to(dev)
    llr = [arena[i * BETA * N_INFO:(i + 1) * BETA * N_INFO] for i in range(len(streams))]
    out = torch.empty(nw * len(streams), dtype=torch.int32, device=dev)
    outs = [out[i * nw:(i + 1) * nw] for i in range(len(streams))]
    s = torch.cuda.Stream(dev)

    def step():
        for i in range(len(streams)):
            vd.vd_decode_tc(code.handle, llr[i], N_INFO, F, V, 0, outs[i], stream=s)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(3, min(args.steps, 20))
    a.record(s)
    for _ in range(reps):
        step()
    b.record(s)
    torch.cuda.synchronize(dev)
    vd.vd_sync(s)
    ms = a.elapsed_time(b) / reps
    ref = torch.empty_like(out)
    plan = stream_plan(vd, code, len(streams), 2, 1, s)
    plan.launch(arena, ref, stream=s)
    torch.cuda.synchronize(dev)
    plan.close()
    bits = N_INFO * len(streams)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = n_sm * 128 * 2 * float(load_peaks().get("sm_max_mhz", 2070.0)) * 1e6
    frames = len(streams) * (N_INFO // F)
    return {"workload": "6 streams x 2^24 info bits, K=7 r1/2, f=256, v=42, int8 LLR; one vd_decode_tc per stream",
            "gbps": bits / (ms / 1e3) / 1e9, "ms_per_step": ms, "identical_to_cuda_core": bool(torch.equal(out, ref)),
            "roofline_frac_integer_peak": bits / (ms / 1e3) * ops_per_bit() / peak,
            "mma_m16n8k16_per_step": frames * ((F + 2 * V) // 2) * 2,
            "form": "one warp per frame; 2 mma.sync.m16n8k16 f16->f32 per stage pair; 4-way max by shuffles"}


def run_radix(args):
    """The general radix-2^rho variant (vd_decode_radix, Sec. VI / Eq.
    general:S) for rho = 1, 2, 3 on the bench workload (one launch per 2^24-bit
    stream), each checked bit for bit against the CUDA-core batch decode."""
    import torch
    import paper_2011_13579_gb300 as vd
    from paper_2011_13579_gb300 import synth
    dev = torch.device("cuda", 0)
    code = vd.Code(K, synth.K7_GENS)
    streams = [synth.segmented_stream(e).s8().view(np.uint8) for e in EBN0S]
    nw = N_INFO // 32
    arena = torch.from_numpy(np.concatenate(streams)).to(dev)
    llr = [arena[i * BETA * N_INFO:(i + 1) * BETA * N_INFO] for i in range(len(streams))]
    s = torch.cuda.Stream(dev)
    ref = torch.empty(nw * len(streams), dtype=torch.int32, device=dev)
    plan = stream_plan(vd, code, len(streams), 2, 1, s)
    plan.launch(arena, ref, stream=s)
    torch.cuda.synchronize(dev)
    plan.close()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = n_sm * 128 * 2 * float(load_peaks().get("sm_max_mhz", 2070.0)) * 1e6
    res = {"workload": "6 streams x 2^24 info bits, K=7 r1/2, f=256, v=42, int8 LLR; one vd_decode_radix per stream",
           "form": "one warp per frame, int32 metrics in shared memory, survivors in global scratch", "rho": {}}
    bits = N_INFO * len(streams)
    for rho in (1, 2, 3):
        out = torch.empty_like(ref)
        outs = [out[i * nw:(i + 1) * nw] for i in range(len(streams))]

        def step():
            for i in range(len(streams)):
                vd.vd_decode_radix(code.handle, llr[i], N_INFO, F, V, rho, 0, outs[i], stream=s)

        step()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        a.record(s)
        for _ in range(reps):
            step()
        b.record(s)
        torch.cuda.synchronize(dev)
        vd.vd_sync(s)
        ms = a.elapsed_time(b) / reps
        res["rho"][str(rho)] = {"gbps": bits / (ms / 1e3) / 1e9, "ms_per_step": ms,
                                "identical_to_cuda_core": bool(torch.equal(out, ref)),
                                "roofline_frac_integer_peak": bits / (ms / 1e3) * ops_per_bit() / peak}
    return res


def packets_only(args):
    """The uneven-packet plan (65,536 packets by default) with a fixed kernel
    shape (radix 2, one lane: no autotuning launches), W + K CUDA-graph
    launches and nothing else, for profilers."""
    import torch
    import paper_2011_13579_gb300 as vd
    from paper_2011_13579_gb300 import synth
    batch = synth.uneven_packets(args.packets)
    pats = (None, synth.PUNCT_R23, synth.PUNCT_R34)
    codes = [vd.Code(K, synth.K7_GENS, puncture=None if p is None else p.tolist()) for p in pats]
    n = batch.n_packets
    pk = {"code_id": batch.rate_id.astype(np.int32), "llr_type": np.zeros(n, np.int32),
          "llr_offset": batch.llr_offset, "n_info": batch.n_info,
          "flags": np.full(n, vd.VD_TERMINATED, np.uint32), "f": np.zeros(n, np.int32),
          "v": np.zeros(n, np.int32), "out_word_offset": batch.out_word_offset}
    tune = vd.VdTune()
    tune.radix = 2
    tune.lanes = args.lanes or 1
    s = torch.cuda.Stream()
    plan = vd.BatchPlan(codes, pk, tune=tune, stream=s)
    llr = torch.from_numpy(batch.llr_s8.view(np.uint8)).cuda()
    nw = int(batch.out_word_offset[-1] + (batch.n_info[-1] + 31) // 32)
    out = torch.empty(nw, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup + args.steps):
        plan.launch(llr, out, stream=s, graph=True)
    torch.cuda.synchronize()
    plan.close()
    print(json.dumps({"mode": "packets", "launches": args.warmup + args.steps}))


def kernel_only(args):
    """W + K launches and nothing else, for profilers: the batch plan of the six
    2^24-bit streams (--path batch) or one stream's vd_decode (--path stream)."""
    import torch
    import paper_2011_13579_gb300 as vd
    from paper_2011_13579_gb300 import synth
    code = vd.Code(K, synth.K7_GENS)
    if args.path == "batch":
        streams = [synth.segmented_stream(e).s8().view(np.uint8) for e in EBN0S]
        arena = torch.from_numpy(np.concatenate(streams)).cuda()
        out = torch.empty(len(streams) * N_INFO // 32, dtype=torch.int32, device="cuda")
        # an explicit shape: no autotuning launches before the profiled ones
        plan = stream_plan(vd, code, len(streams), args.radix, args.lanes or 1, None)
        for _ in range(args.warmup + args.steps):
            plan.launch(arena, out, stream=None)
        torch.cuda.synchronize()
        plan.close()
    else:
        # one 2^24-bit stream: the K=7 bench code at f=256, v=42, or (--code k9)
        # the precision study's K=9 r1/3 code at f=512, v=64, 2 dB
        if args.code == "k9":
            code = vd.Code(9, synth.K9_GENS)
            st, f, v = synth.precision_stream(2.0), 512, 64
        else:
            st, f, v = synth.segmented_stream(3.0), F, V
        llr = torch.from_numpy(st.s8().view(np.uint8)).cuda()
        out = torch.empty(N_INFO // 32, dtype=torch.int32, device="cuda")
        tune = None
        if args.lanes:
            tune = vd.VdTune()
            tune.lanes = args.lanes
        for _ in range(args.warmup + args.steps):
            vd.vd_decode(code.handle, llr, vd.VD_LLR_S8, N_INFO, f, v, args.radix, 0, out, None, tune, None)
        torch.cuda.synchronize()
    print(json.dumps({"mode": "kernel", "launches": args.warmup + args.steps}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--radix", type=int, default=2, choices=[2, 4])
    ap.add_argument("--lanes", type=int, default=0)
    ap.add_argument("--path", default="batch", choices=["batch", "stream"])
    ap.add_argument("--code", default="k7", choices=["k7", "k9"],
                    help="--mode kernel --path stream: decode one K=7 bench stream or one K=9 precision-study stream")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bm-gate", action="store_true", help="skip the branch-metric CUDA/tensor-core gate")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serving-loads", type=lambda t: [float(x) for x in t.split(",")] if t else [],
                    default=[round(0.1 * i, 1) for i in range(1, 11)],
                    help="offered loads (fractions of peak); empty: skip serving")
    ap.add_argument("--serving-pool", type=int, default=8192)
    ap.add_argument("--serving-seconds", type=float, default=2.0)
    ap.add_argument("--serving-max-packets", type=int, default=400000)
    ap.add_argument("--workload", default="stream",
                    choices=["stream", "precision", "packets", "intpeak", "tc", "radix"],
                    help="precision: the K=9 precision study (int8 / 4-bit / fp16) instead of the bench line; "
                         "packets: only W+K graph launches of the uneven-packet plan (for profilers); "
                         "intpeak: only the integer-issue microbenchmark")
    ap.add_argument("--no-ber", action="store_true", help="skip the segmentation-BER leg (CPU oracle)")
    ap.add_argument("--precision-bits", type=int, default=1 << 24)
    ap.add_argument("--precision-ebn0", type=lambda t: [float(x) for x in t.split(",")],
                    default=[0.0, 1.0, 2.0, 3.0, 4.0])
    ap.add_argument("--packets", type=int, default=65536,
                    help="packets of the batched-vs-plain comparison (0: skip it)")
    ap.add_argument("--mode", default="full", choices=["full", "kernel"],
                    help="kernel: only W+K launches of one stream decode (for profilers)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    # one hardware queue per stream of the one-launch-per-packet comparison
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", str(PLAIN_STREAMS))

    if args.impl == "reference":
        # the reference arm is the plain CPU oracle; rank 0 alone runs it
        if rank != 0:
            return
        import oracle
        oracle.build()
        vals = []
        for _ in range(args.warmup):
            cpu_oracle_run(seconds_budget=min(2.0, args.cpu_seconds))
        t = time.perf_counter()
        for _ in range(args.steps):
            vals.append(cpu_oracle_run(seconds_budget=min(5.0, args.cpu_seconds)))
        wall = time.perf_counter() - t
        v = statistics.median(x["value"] for x in vals)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gbit/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * wall / max(1, args.steps), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": workload_config(2, 1, path="oracle"),
                "cpu_baseline": {**vals[-1], "value": v},
                "e2e": {"value": v, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2011_13579_gb300 as vd
    vd.build()
    if args.workload == "precision":
        if rank == 0:
            print(json.dumps({"precision_study": run_precision(args)}), flush=True)
        return
    if args.workload == "packets":
        packets_only(args)
        return
    if args.workload == "radix":
        print(json.dumps({"radix_variant": run_radix(args)}), flush=True)
        return
    if args.workload == "tc":
        print(json.dumps({"tensor_core_variant": run_tc(args)}), flush=True)
        return
    if args.workload == "intpeak":
        import torch
        print(json.dumps({"int_peak": run_int_peak(torch.device("cuda", 0), torch.cuda.current_stream())}),
              flush=True)
        return
    if args.mode == "kernel":
        kernel_only(args)
        return

    r = run_gpu(args, rank, world)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import torch
    peaks = load_peaks()
    n_sm = r["n_sm"]
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    # Integer roofline: the integer lanes per SM per clock measured by the
    # vd_int_peak microbenchmark on this GPU (best instruction class or 1:1
    # mix), each 16x2 instruction carrying two frames (two 16-bit halves), at
    # the maximum SM clock.  The fused add-then-max of the butterfly does two
    # algorithmic operations per half in one lane slot, so frac = 1 is not a
    # ceiling: the ACS alone (the butterfly variant) reaches more.
    ip = run_int_peak(torch.device("cuda", 0), torch.cuda.current_stream())
    lanes = ip["lanes_per_sm_per_clk"]
    peak_ops = n_sm * lanes * 2 * sm_max_mhz * 1e6
    launch_ms = r["launch_ms"]
    avg_launch_s = statistics.mean(launch_ms) / 1e3
    ops_per_launch = ops_per_bit() * r["bits_per_launch"]
    achieved = ops_per_launch / avg_launch_s
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        try:
            tr = json.load(open(tr_path))
            if (tr.get("radix") == args.radix and tr.get("lanes", 0) == args.lanes
                    and tr.get("path", "stream") == args.path
                    and tr.get("source_hash") == kernel_source_hash()):
                traffic = tr.get("bytes_per_launch")
        except (OSError, ValueError):
            traffic = None
    line = {
        "metric": METRIC,
        "value": r["value"],
        "unit": "Gbit/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r["ms"] / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int8 LLR / exact 16x2 metrics",
        "data": "synthetic",
        "config": {**workload_config(r["shape"]["radix"], r["shape"]["lanes"], args.path),
                   "parallelism": f"replicas{world}"},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "Tops/s", "frac": achieved / peak_ops, "traffic": traffic,
                     "kernel": "vd::batch_kernel" if args.path == "batch" else "vd::stream_kernel",
                     "avg_launch_ms": avg_launch_s * 1e3,
                     "launch_timing": ("timed region / launches: consecutive chained launches overlap, "
                                       "so a per-launch event pair would serialise them" if r["chained"]
                                       else "mean of per-launch CUDA event pairs"),
                     "isolated_launch_ms": r["isolated_launch_ms"],
                     "frac_isolated": (ops_per_launch / (r["isolated_launch_ms"] / 1e3) / peak_ops
                                       if r["isolated_launch_ms"] else None),
                     "ops_per_bit": ops_per_bit(),
                     "peak_basis": (f"{n_sm} SMs x {lanes:.1f} integer lanes per SM per clock (measured by "
                                    f"vd_int_peak: {ip['lanes_from']}) x 2 halves (16x2) x {sm_max_mhz:.0f} MHz "
                                    "max SM clock; a fused add-then-max counts 2 algorithmic ops per half in one "
                                    "lane slot, so frac = 1 is not the ceiling: the ACS alone reaches "
                                    f"{ip['butterfly_alg_ops_per_sm_per_clk'] / (2 * lanes):.2f} of this peak"),
                     "issue_ceiling_acs_only": ip["butterfly_alg_ops_per_sm_per_clk"] / (2 * lanes)},
        "int_peak": ip,
        "e2e": r["e2e"],
        "gpu_launches": args.steps * r["launches_per_step"],
        "clocks": r["clocks"],
        "ber_6db": r["ber_6db"],
    }
    if r.get("packets"):
        line["batched_vs_plain"] = r["packets"]
    if world == 1 and r.get("words_r2") is not None:
        line["segmentation_ber"] = run_ber(args, r["words_r2"], r["words_r4"])
    if world == 1 and args.serving_loads:
        line["serving"] = run_serving(args)
        line["serving_device"] = run_serving(args, device_resident=True)
    if world == 1 and not args.no_bm_gate:
        import torch
        line["bm_gate"] = run_bm_gate(torch.device("cuda", 0), torch.cuda.current_stream())
    if world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_oracle_run(args.cpu_seconds)
            one = cpu_oracle_run(min(5.0, args.cpu_seconds), threads=1)
            line["cpu_baseline"]["single_thread"] = {"value": one["value"], "cores": 1, "sample": one["sample"]}
        except Exception as exc:  # noqa: BLE001
            line["cpu_baseline"] = {"value": None, "error": str(exc)[:200]}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
