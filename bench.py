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


def workload_config(radix, lanes, path="batch"):
    return {"workload": "segmented stream decode, K=7 r1/2 (171,133), 6 streams x 2^24 info bits, "
                        "Eb/N0 1..6 dB, f=256, v=42, int8 LLR",
            "n_info_per_stream": N_INFO, "streams_per_step": len(EBN0S), "f": F, "v": V,
            "radix": radix, "lanes": lanes,
            "path": ("one persistent batched launch per step (vd_batch_plan_launch)" if path == "batch"
                     else "one vd_decode launch per stream"),
            "l2": "inputs larger than L2 (192 MiB cycled per step)"}


def stream_plan(vd, code, n_streams, radix, lanes, stream):
    """The six streams as six packets of one batch plan (f=256, v=42)."""
    tune = vd.VdTune()
    tune.radix = radix
    tune.lanes = lanes
    pk = {"code_id": np.zeros(n_streams, np.int32), "llr_type": np.zeros(n_streams, np.int32),
          "llr_offset": np.arange(n_streams, dtype=np.int64) * BETA * N_INFO,
          "n_info": np.full(n_streams, N_INFO, np.int64), "flags": np.zeros(n_streams, np.uint32),
          "f": np.full(n_streams, F, np.int32), "v": np.full(n_streams, V, np.int32),
          "out_word_offset": np.arange(n_streams, dtype=np.int64) * (N_INFO // 32)}
    return vd.BatchPlan([code], pk, tune=tune, stream=stream)


def ops_per_bit(f=F, v=V, k=K):
    """Algorithmic ACS operations per decoded bit: 2 adds + 1 compare-select per
    state per trellis stage, over f + 2v stages per f decoded bits."""
    return 3 * (1 << (k - 1)) * (f + 2 * v) / f


def kernel_source_hash():
    """Hash of the stream kernel's sources: a traffic figure measured on other
    sources does not describe this kernel."""
    import hashlib
    h = hashlib.sha256()
    for f in ("paper_2011_13579_gb300/csrc/vd_stream.cuh", "paper_2011_13579_gb300/csrc/vd_device.cuh"):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
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

    def one_launch(i):
        """Launch i of a step: one stream, or the whole batch."""
        if plan is not None:
            plan.launch(arena, out_arena, stream=s)
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
    # per-launch events on the launching stream, for the kernel's own duration
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
            ev[k][0].record(s)
            one_launch(i)
            ev[k][1].record(s)
            k += 1
    t1.record(s)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ms = t0.elapsed_time(t1)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    clocks = sampler.stop() if sampler else None

    if world > 1:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())

    bits_per_step = N_INFO * len(streams)
    value = bits_per_step * args.steps * world / (ms / 1e3) / 1e9

    # end to end through the public API with host buffers: pinned H2D of the
    # step's LLRs, decode, D2H of the decoded words, all inside the timed region
    host_in = [torch.from_numpy(x).pin_memory() for x in streams]
    host_out = [torch.empty(nw, dtype=torch.int32).pin_memory() for _ in streams]
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    with torch.cuda.stream(s):
        for _ in range(e2e_steps):
            for i in range(len(streams)):
                llr_dev[i].copy_(host_in[i], non_blocking=True)
            for i in range(launches_per_step):
                one_launch(i)
            for i in range(len(streams)):
                host_out[i].copy_(outs[i], non_blocking=True)
    e1.record(s)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1)
    e2e_value = bits_per_step * e2e_steps / (e2e_ms / 1e3) / 1e9
    h2d = sum(int(x.size) for x in streams)
    d2h = nw * 4 * len(streams)

    # sanity: the decode of the 6 dB stream is nearly error-free
    dec = outs[-1].cpu().numpy().view(np.uint32)
    bits = ((dec[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.uint8).reshape(-1)
    ref_bits = synth.segmented_stream(6.0).bits
    ber6 = float(np.mean(bits != ref_bits))

    if plan is not None:
        plan.close()
    return {"ms": ms, "value": value, "launch_ms": launch_ms, "clocks": clocks,
            "launches_per_step": launches_per_step, "bits_per_launch": bits_per_step // launches_per_step,
            "e2e": {"value": e2e_value, "unit": "Gbit/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "ber_6db": ber6, "n_sm": torch.cuda.get_device_properties(dev).multi_processor_count}


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
        plan = stream_plan(vd, code, len(streams), args.radix, args.lanes, None)
        for _ in range(args.warmup + args.steps):
            plan.launch(arena, out, stream=None)
        torch.cuda.synchronize()
        plan.close()
    else:
        llr = torch.from_numpy(synth.segmented_stream(3.0).s8().view(np.uint8)).cuda()
        out = torch.empty(N_INFO // 32, dtype=torch.int32, device="cuda")
        tune = None
        if args.lanes:
            tune = vd.VdTune()
            tune.lanes = args.lanes
        for _ in range(args.warmup + args.steps):
            vd.vd_decode(code.handle, llr, vd.VD_LLR_S8, N_INFO, F, V, args.radix, 0, out, None, tune, None)
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
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--mode", default="full", choices=["full", "kernel"],
                    help="kernel: only W+K launches of one stream decode (for profilers)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

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
                "config": workload_config(2, 0),
                "cpu_baseline": {**vals[-1], "value": v},
                "e2e": {"value": v, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2011_13579_gb300 as vd
    vd.build()
    if args.mode == "kernel":
        kernel_only(args)
        return

    r = run_gpu(args, rank, world)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    peaks = load_peaks()
    n_sm = r["n_sm"]
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    # ALU roofline: 128 integer lanes per SM per clock, each 16x2 instruction
    # carrying two frames (two 16-bit halves), at the maximum SM clock
    peak_ops = n_sm * 128 * 2 * sm_max_mhz * 1e6
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
        "dtype": "u16x2",
        "data": "synthetic",
        "config": {**workload_config(args.radix, args.lanes, args.path), "parallelism": f"replicas{world}"},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "Tops/s", "frac": achieved / peak_ops, "traffic": traffic,
                     "kernel": "vd::batch_kernel" if args.path == "batch" else "vd::stream_kernel",
                     "avg_launch_ms": avg_launch_s * 1e3,
                     "ops_per_bit": ops_per_bit(),
                     "peak_basis": f"{n_sm} SMs x 128 lanes x 2 halves x {sm_max_mhz:.0f} MHz"},
        "e2e": r["e2e"],
        "gpu_launches": args.steps * r["launches_per_step"],
        "clocks": r["clocks"],
        "ber_6db": r["ber_6db"],
    }
    if world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_oracle_run(args.cpu_seconds)
        except Exception as exc:  # noqa: BLE001
            line["cpu_baseline"] = {"value": None, "error": str(exc)[:200]}
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
