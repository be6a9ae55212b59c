#!/usr/bin/env python
"""Benchmark of the integer convex-hull path (reduce + chain + hull) on GB300.

Default workload (the configuration the headline metric is quoted on):
p = 65536, n = 2^26 int32 points per instance, three seeded distributions
(uniform square, inscribed disc, Gaussian sigma = p/8) run separately.  One
step = one ch_convex_hull call per distribution (3 * 2^26 points).  Inputs
(537 MB each) are resident in HBM and larger than L2, so no flush is needed.

Prints ONE JSON line (rank 0).  `value` is device-timed whole-job throughput in
Gpoints/s; `e2e` is the same metric through ch_convex_hull_host (host buffers,
copies inside the timed region); `roofline` is for the dominant kernel (the
reduction), timed per launch with CUDA events recorded on its stream;
`cpu_baseline` is the CPU oracle on the host cores.

--impl reference times the CPU oracle itself on the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpoints/s reduce+chain+hull, % of HBM roofline; batched/learned vs plain"

WORKLOADS = {
    # name: (p, n, distributions)
    "plain_at_scale": (65536, 1 << 26, ("uniform", "disc", "gaussian")),
    "plain_small": (1024, 100_000, ("uniform",)),
    "projected_shells": (4096, 10_000_000, ("shells",)),
    # profiling case of the filtered reduction: 268 MB of points, above L2
    "profile_reduce": (65536, 1 << 25, ("uniform",)),
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_sha(src_path, name):
    """Digest of one kernel's source text: from the line that names it in a
    definition to the end of its body (the first line that is a lone "}")."""
    lines = open(src_path).read().split("\n")
    start = next(i for i, l in enumerate(lines) if l.strip().startswith(name + "("))
    while start > 0 and lines[start - 1].strip() and not lines[start - 1].startswith("//"):
        start -= 1
    end = next(i for i in range(start, len(lines)) if lines[i] == "}")
    return hashlib.sha256("\n".join(lines[start:end + 1]).encode()).hexdigest()[:16]


def _traffic(kernel, n, p):
    """DRAM bytes per launch of the reduction kernel from the committed ncu
    counters, scaled from the captured n to this n (the kernel streams each
    point once); None when the kernel's source changed since the capture or
    the capture was at another p."""
    try:
        with open(os.path.join(ROOT, "profiles", "reduce_traffic.json")) as f:
            rec = json.load(f)
        src = os.path.join(ROOT, "paper_1505_00914_gb300", "csrc", "reduce.cu")
        if rec.get("kernel") != kernel or rec.get("p") != p:
            return None
        if rec.get("kernel_sha") != _kernel_sha(src, kernel):
            return None
        return (rec["dram_bytes_read"] + rec["dram_bytes_write"]) * n / rec["n"]
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gen_inputs(workload, rank):
    from paper_1505_00914_gb300 import synth
    p, n, dists = WORKLOADS[workload]
    return p, n, [(d, synth.points(d, n, p, seed=1 + 1000 * rank)) for d in dists]


def cpu_oracle_rate(p, inputs, budget_s):
    """The CPU oracle as it stands (single thread): Algorithm 1 + hull of the
    reduced set, over the workload's instances until ~budget_s elapsed."""
    import oracle
    done, t0 = 0, time.perf_counter()
    passes = 0
    while True:
        for _, P in inputs:
            oracle.hull_chain(oracle.reduce(P, p))
            done += P.shape[0]
        passes += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return done / dt / 1e9, dt, passes


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p, n, inputs = gen_inputs(args.workload, 0)
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        for _, P in inputs[:1]:
            oracle.hull_chain(oracle.reduce(P, p))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _, P in inputs:
            oracle.hull_chain(oracle.reduce(P, p))
    dt = time.perf_counter() - t0
    pts = args.steps * n * len(inputs)
    v = pts / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "Gpoints/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": {"workload": args.workload, "p": p, "n_per_instance": n,
                                        "distributions": [d for d, _ in inputs]},
        "cpu_baseline": {"value": v, "unit": "Gpoints/s", "cores": 1, "kind": "oracle",
                         "sample": f"full workload, {args.steps} steps x {len(inputs)} instances"},
        "e2e": {"value": v, "unit": "Gpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1505_00914_gb300 import _build, ch
    ch.lib()

    p, n, inputs = gen_inputs(args.workload, rank)
    dev_in = [torch.from_numpy(P).cuda() for _, P in inputs]
    nws = ch.ch_convex_hull_workspace_size(n, p)
    ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
    hulls = [torch.empty((2 * p, 2), dtype=torch.int32, device="cuda") for _ in inputs]
    hcs = [torch.empty(1, dtype=torch.int32, device="cuda") for _ in inputs]
    stream = torch.cuda.current_stream()

    def step():
        for d, h, c in zip(dev_in, hulls, hcs):
            ch.ch_convex_hull(d, p, hull=h, hull_count=c, workspace=ws, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    rc = ch.ch_sync_status()
    if rc != ch.CH_OK:
        raise RuntimeError(f"warm-up failed: {ch.strerror(rc)}")

    # reduction kernel timing inside the timed region
    nl = args.steps * len(inputs)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nl)]
    for a, b in evs:
        a.record(stream)
        b.record(stream)
    torch.cuda.synchronize()
    ch.ch_trace_set(evs)

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ch.ch_trace_set([])
    rc = ch.ch_sync_status()
    if rc != ch.CH_OK:
        raise RuntimeError(f"timed run failed: {ch.strerror(rc)}")
    ms = t0.elapsed_time(t1)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    red_ms = [a.elapsed_time(b) for a, b in evs]
    red_avg = sum(red_ms) / len(red_ms)

    pts_step = n * len(inputs)
    value = world * pts_step * args.steps / (ms / 1e3) / 1e9
    peak, peak_kind = _peaks()

    # e2e through the host-buffer entry point (pinned host memory)
    e2e_steps = max(1, min(args.steps, 5))
    host_in = [torch.from_numpy(P).pin_memory() for _, P in inputs]
    nws_h = ch.ch_convex_hull_host_workspace_size(n, p)
    del ws
    ws_h = torch.empty(nws_h, dtype=torch.uint8, device="cuda")
    hh = torch.empty((2 * p, 2), dtype=torch.int32).pin_memory()
    hsz = []
    for hp in host_in:  # warm-up
        hsz.append(ch.ch_convex_hull_host(hp, p, ws_h, stream=stream, host_hull=hh).shape[0])
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    d2h = 0
    for _ in range(e2e_steps):
        for hp in host_in:
            d2h += ch.ch_convex_hull_host(hp, p, ws_h, stream=stream, host_hull=hh).shape[0] * 8 + 4
    e2e_s = time.perf_counter() - w0
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_val = world * pts_step * e2e_steps / e2e_s / 1e9

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    kernel_bytes = 8 * n + 8 * p  # points read + L produced, per launch
    achieved = kernel_bytes / (red_avg / 1e3) / 1e9
    kname = ["k_reduce_private", "k_reduce_filtered", "k_reduce_global"][ch.ch_plan_info(n, p)[0]]
    cpu_v, cpu_dt, cpu_passes = cpu_oracle_rate(p, inputs, args.cpu_budget)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "Gpoints/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": args.workload, "p": p, "n_per_instance": n,
                   "distributions": [d for d, _ in inputs], "instances_per_step": len(inputs),
                   "l2": "inputs 8n bytes per instance, larger than L2; no flush"},
        "hbm_frac_step": (pts_step * 8 / (ms / args.steps / 1e3) / 1e9) / peak,
        "roofline": {"bound": "hbm", "kernel": kname,
                     "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "algorithmic_bytes_per_launch": kernel_bytes, "avg_launch_ms": red_avg,
                     "traffic": _traffic(kname, n, p)},
        "e2e": {"value": e2e_val, "unit": "Gpoints/s", "h2d_bytes_per_step": pts_step * 8,
                "d2h_bytes_per_step": d2h // e2e_steps, "steps": e2e_steps},
        "cpu_baseline": {"value": cpu_v, "unit": "Gpoints/s", "cores": 1, "kind": "oracle",
                         "sample": f"{cpu_passes} pass(es) over the step's {len(inputs)} instances "
                                   f"({cpu_dt:.1f} s, single thread)"},
        "gpu_launches": args.steps * len(inputs) * ch.ch_plan_info(n, p)[1],
        "clocks": clocks,
        "hull_vertices": hsz,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="plain_at_scale")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
