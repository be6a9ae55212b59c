#!/usr/bin/env python
"""Benchmark of the integer convex-hull path (reduce + chain + hull) on GB300.

Default workload (the configuration the headline metric is quoted on):
p = 65536, n = 2^26 int32 points per instance, three seeded distributions
(uniform square, inscribed disc, Gaussian sigma = p/8) run separately.  One
step = one ch_convex_hull call per distribution (3 * 2^26 points), each
instance on its own CUDA stream and workspace (independent problems);
consecutive steps are pipelined: each instance's stream runs its calls in
order and the streams are joined only at the ends of a timed region.
Inputs (537 MB each) are resident in HBM and larger than L2, so no flush is
needed.

Prints ONE JSON line (rank 0).  `value` is device-timed whole-job throughput in
Gpoints/s; `e2e` is the same metric through ch_convex_hull_host (host buffers,
copies inside the timed region); `roofline` is for the dominant kernel (the
reduction), timed per launch with CUDA events recorded on its stream;
`cpu_baseline` is the CPU oracle on one host core (Algorithm 1 + the hull of
the reduced set), with two more host figures beside it: the hull of all points
by sort + Andrew (the paper's t_n) and Algorithm 1 alone on every host core
(one L per thread, merged by min/max).  `value` comes from a
timed region without instrumentation; the roofline's launch times come from
a second timed region of the same steps, instances one after another on one
stream, with events around each reduction launch (its step time is reported
as roofline.ms_per_step_while_timed).

--impl reference times the CPU oracle itself on the same workload (rank 0 only).

Other workloads (--workload):
  plain_at_scale_u16  the default workload with the points stored as packed
            16-bit pairs (ch_convex_hull_u16: 4 bytes per point instead of 8).
  box       Steps 1-2 for int32 points anywhere: three instances of 2^26
            points (uniform in a 65536 x 65536 box at (-1.5e9, 7e8), disc in a
            120000 x 40000 box at (1e9, -2e9), Gaussian in a 30000 x 90000
            box at (-123456789, 987654321)); a step is ch_bbox on each, one
            read of the three boxes, then ch_convex_hull_box on each (columns
            along the shorter side), each instance on its own stream.
  sparse    the sparse regime p > n (Section 4): p = 2^24, n = 2^20 per
            instance, uniform / disc / Gaussian, through the tree of bit words
            (ch_convex_hull_sparse) against the plain path (an array L of p
            entries) on the same inputs; plus, as in Fig. 11, both paths at
            column densities s/p of 5 % to 85 % (uniform x).
  rxy       Algorithm 1 along x, then the second scan along y (Section 2,
            Figs. 4 and 7) and the hull of the rxy points
            (ch_convex_hull_rxy), against the plain path, on the
            projected-shells stand-in; reports the rx and rxy counts.
  melkman   the paper's Melkman experiment (Section 3, Fig. 10) on the
            projected-shells stand-in (p = 4096, 10^7 points): Algorithm 1,
            the Lemma 1 polyline and Melkman's hull (ch_convex_hull_melkman)
            against the plain path on the same input, hulls checked equal.
  learned   p = 65536, n = 2^27 per instance, one instance each of uniform,
            disc, Gaussian and thin annulus (r in [0.45p, 0.5p]); the path
            with the trained culling network (ch_hull_learned) against the
            plain path and against culling from the sector centres (no
            network) on the same inputs, with the cull rates and a check that
            all three hulls agree.
  batched   10,000 sets, n log-uniform in [1e2, 1e6], p from {256, 1024,
            4096, 16384}, uniform/disc/Gaussian by seeded choice, in one
            ragged buffer: ch_hull_batched (autotuned chunk size and CTA shape, replayed
            from a captured CUDA graph) against one ch_convex_hull per set.
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
L2_FLUSH_BELOW = 192 << 20  # inputs below this many bytes per instance get an L2 flush per step

WORKLOADS = {
    # name: (p, n, distributions)
    "plain_at_scale": (65536, 1 << 26, ("uniform", "disc", "gaussian")),
    # the same sets as packed 16-bit points (x - 1) | (y - 1) << 16, 4 bytes each
    "plain_at_scale_u16": (65536, 1 << 26, ("uniform", "disc", "gaussian")),
    "plain_small": (1024, 100_000, ("uniform",)),
    "projected_shells": (4096, 10_000_000, ("shells",)),
    # profiling cases of the filtered reduction: 268 MB (134 MB) of points, above L2
    "profile_reduce": (65536, 1 << 25, ("uniform",)),
    "profile_reduce_u16": (65536, 1 << 25, ("uniform",)),
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the dominant kernel of each form ch_plan_info reports (3: the whole path in one launch)
KERNEL_OF_FORM = ("k_reduce_private", "k_reduce_filtered", "k_reduce_global", "k_small")


# device functions every reduction kernel streams its points through: a change
# to them changes the kernels' traffic as much as a change to their own text
STREAM_HELPERS = ("stream_pairs_wide", "stream_pairs")


def _def_text(lines, name):
    """Source text of one definition: from the line that names it (a kernel's
    name starts its line, a device function's follows `void`) back over its
    template lines, to the end of its body (the first lone "}")."""
    start = next(i for i, l in enumerate(lines)
                 if l.strip().startswith(name + "(") or (" void " + name + "(") in l)
    while start > 0 and lines[start - 1].strip() and not lines[start - 1].startswith("//"):
        start -= 1
    end = next(i for i in range(start, len(lines)) if lines[i] == "}")
    return "\n".join(lines[start:end + 1])


def _kernel_sha(src_path, name):
    """Digest of one kernel's source text and of the streaming helpers it
    calls."""
    lines = open(src_path).read().split("\n")
    text = "\n".join(_def_text(lines, k) for k in (name,) + STREAM_HELPERS)
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def _traffic(kernel, n, p, u16=False):
    """DRAM bytes per launch of the reduction kernel from the committed ncu
    counters (int32 or packed 16-bit points), scaled from the captured n to
    this n (the kernel streams each point once); None when the kernel's source
    changed since the capture or the capture was at another p."""
    try:
        name = "reduce_traffic_u16.json" if u16 else "reduce_traffic.json"
        with open(os.path.join(ROOT, "profiles", name)) as f:
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
                 "-lms", "20"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        try:
            with open(self.path) as f:
                lines = f.readlines()
            os.unlink(self.path)
        except Exception:
            return None
        return self.summarize(lines)

    @staticmethod
    def summarize(lines):
        """The `clocks` object from nvidia-smi CSV rows (fields as in Q):
        median SM clock, maximum SM clock, the throttle reasons seen active."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
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
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gen_inputs(workload, rank):
    from paper_1505_00914_gb300 import synth
    p, n, dists = WORKLOADS[workload]
    return p, n, [(d, synth.points(d, n, p, seed=1 + 1000 * rank)) for d in dists]


def pack_u16(P):
    """Host int32 (n, 2) points -> int32 (n,) words (x - 1) | (y - 1) << 16."""
    P = np.asarray(P, dtype=np.int64)
    return np.ascontiguousarray((((P[:, 1] - 1) << 16) | (P[:, 0] - 1)).astype(np.uint32).view(np.int32))


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


def cpu_andrew_all_points(p, inputs, m=1 << 22):
    """The paper's comparison on the host: the hull of all points (sort +
    Andrew, t_n) against Algorithm 1 + the hull of the reduced set
    (t_r + t_s), single thread, on the first m points of each instance."""
    import oracle
    t_n = t_rs = 0.0
    for _, P in inputs:
        Q = np.ascontiguousarray(P[:m])
        t0 = time.perf_counter()
        a = oracle.hull_points(Q)
        t1 = time.perf_counter()
        b = oracle.hull_chain(oracle.reduce(Q, p))
        t2 = time.perf_counter()
        if not np.array_equal(a, b):
            raise RuntimeError("oracle hulls differ")
        t_n += t1 - t0
        t_rs += t2 - t1
    pts = sum(min(m, P.shape[0]) for _, P in inputs)
    return {"sample": f"the first {min(m, inputs[0][1].shape[0])} points of each instance, "
                      f"single thread",
            "sort_andrew_gpoints_s": pts / t_n / 1e9, "reduce_then_hull_gpoints_s": pts / t_rs / 1e9,
            "speedup_t_n_over_t_r_plus_t_s": t_n / t_rs}


def cpu_reduce_all_cores(p, inputs, passes=3):
    """Algorithm 1 on every host core: each thread reduces a contiguous shard
    of an instance into its own L with the oracle, and the partial arrays are
    merged column by column (min of ly, max of hy; exact because min and max
    commute).  The oracle's C call releases the interpreter lock, so the
    threads run in parallel.  Best of `passes` passes over all instances."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    threads = max(1, int(threads or 1))

    def shards(P):
        cut = np.linspace(0, P.shape[0], threads + 1).astype(np.int64)
        return [P[cut[k]:cut[k + 1]] for k in range(threads)]

    parts = [shards(P) for _, P in inputs]
    best, merged = None, []
    with ThreadPoolExecutor(max_workers=threads) as pool:
        for _ in range(passes):
            merged = []
            t0 = time.perf_counter()
            for sh in parts:
                Ls = list(pool.map(lambda q: oracle.reduce(q, p), sh))
                L = Ls[0].copy()
                for Lk in Ls[1:]:
                    np.minimum(L[:, 0], Lk[:, 0], out=L[:, 0])
                    np.maximum(L[:, 1], Lk[:, 1], out=L[:, 1])
                merged.append(L)
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
    for L, (_, P) in zip(merged, inputs):
        if not np.array_equal(L, oracle.reduce(P, p)):
            raise RuntimeError("merged partial arrays differ from one pass of Algorithm 1")
    pts = sum(P.shape[0] for _, P in inputs)
    return {"reduce_gpoints_s": pts / best / 1e9, "threads": threads,
            "sample": f"all {len(inputs)} instances, Algorithm 1 only, one L per thread "
                      f"merged by min/max, best of {passes} passes"}


def workload_config(workload):
    """The `config` object of a workload, the same for both arms."""
    if workload == "learned":
        p, n, dists = LEARNED
        return {"workload": "learned", "p": p, "n_per_instance": n, "distributions": list(dists),
                "instances_per_step": len(dists),
                "concurrency": ("each instance on its own CUDA stream and workspace, in every arm; "
                                "consecutive steps pipelined (streams joined at the ends of each "
                                "timed region)"),
                "l2": "inputs 8n bytes per instance, larger than L2; no flush"}
    if workload == "box":
        return {"workload": "box", "n_per_instance": BOX_N,
                "boxes": [{"distribution": d, "width": sx, "height": sy, "x0": x0, "y0": y0}
                          for d, sx, sy, x0, y0 in BOX],
                "instances_per_step": len(BOX),
                "concurrency": "each instance on its own CUDA stream and workspace",
                "l2": "inputs 8n bytes per instance, larger than L2; no flush"}
    if workload == "sparse":
        p, n, dists = SPARSE
        return {"workload": "sparse", "p": p, "n_per_instance": n, "distributions": list(dists),
                "instances_per_step": len(dists),
                "concurrency": "each instance on its own CUDA stream and workspace",
                "l2": "points 8 MB per instance, below L2: a 256 MB write precedes every step "
                      "and its time is subtracted"}
    if workload in ("melkman", "rxy"):
        p, n, dists = WORKLOADS[MELKMAN]
        return {"workload": workload, "p": p, "n_per_instance": n, "distributions": list(dists),
                "instances_per_step": 1,
                "l2": "80 MB of points, below L2 (129 MB): a 256 MB write precedes every step "
                      "and its time is subtracted"}
    if workload in ("batched", "profile_batched"):
        return {"workload": workload,
                "sets": BATCH_SETS if workload == "batched" else PROFILE_BATCH_SETS,
                "ps": [256, 1024, 4096, 16384],
                "n_range": [100, 1_000_000], "distributions": ["uniform", "disc", "gaussian"],
                "l2": ("about 8.5 GB" if workload == "batched" else "about 0.9 GB")
                      + " of points per step, larger than L2; no flush"}
    p, n, dists = WORKLOADS[workload]
    bpp = 4 if workload.endswith("_u16") else 8
    return {"workload": workload, "p": p, "n_per_instance": n, "distributions": list(dists),
            "point_format": ("packed uint16 pairs (x - 1, y - 1), 4 bytes per point"
                             if bpp == 4 else "int32 pairs, 8 bytes per point"),
            "instances_per_step": len(dists),
            "concurrency": ("each instance on its own CUDA stream and workspace"
                            + ("; consecutive steps pipelined (an instance's calls in order on "
                               "its stream, the streams joined at the ends of each timed region)"
                               if n * bpp >= L2_FLUSH_BELOW else
                               "; the streams joined after every step (each step follows a flush)")),
            "l2": (f"inputs {bpp}n bytes per instance, larger than L2; no flush"
                   if n * bpp >= L2_FLUSH_BELOW else
                   "inputs smaller than L2: a 256 MB write precedes every step and its time "
                   "is subtracted")}


def _reference_units(workload):
    """The workload as a list of (p, name, points) problems for the oracle."""
    from paper_1505_00914_gb300 import synth
    if workload == "learned":
        p, n, dists = LEARNED
        return [(p, d, synth.points(d, n, p, seed=101 + i)) for i, d in enumerate(dists)]
    if workload == "batched":
        pts, off, ps, _ = synth.batched(BATCH_SETS, seed=4)
        return [(int(ps[s]), f"set{s}", pts[off[s]:off[s + 1]]) for s in range(len(ps))]
    if workload == "box":
        return [(None, d, P) for d, P in box_inputs(0)]
    if workload == "sparse":
        p, n, dists = SPARSE
        return [(p, d, synth.points(d, n, p, seed=51 + i)) for i, d in enumerate(dists)]
    p, n, inputs = gen_inputs(MELKMAN if workload in ("melkman", "rxy") else workload, 0)
    return [(p, d, P) for d, P in inputs]


def oracle_solver(workload):
    """The oracle's form of one problem of the workload: Algorithm 1 + the
    hull of the reduced set; Steps 1-2 first for `box`; Melkman's hull of the
    Lemma 1 polyline for `melkman`."""
    import oracle
    if workload == "box":
        return lambda p, P: oracle.hull_box(P)
    if workload == "melkman":
        return lambda p, P: oracle.melkman(oracle.polyline(oracle.reduce(P, p)))
    if workload == "rxy":
        return lambda p, P: oracle.hull_points(oracle.rxy_points(oracle.reduce_rows(
            oracle.reduce(P, p))))
    if workload == "sparse":  # the chains from the points (no array of p), then the hull
        def solve(p, P):
            oracle.chain_points(P)
            return oracle.hull_points(P)
        return solve
    return lambda p, P: oracle.hull_chain(oracle.reduce(P, p))


def run_reference(args):
    """The CPU oracle as it stands (Algorithm 1 + the hull of the reduced set,
    single thread) on the same workload.  A step is a bounded sample of it:
    the whole step for the plain workloads, one instance per step (in turn)
    for `learned` and `box`, the next sets up to 1e8 points for `batched`."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    units = _reference_units(args.workload)
    per_step = {"learned": 1, "box": 1}.get(args.workload)
    solve = oracle_solver(args.workload)
    cursor = [0]

    def step():
        done = 0
        if args.workload == "batched":
            while done < 100_000_000:
                p, _, P = units[cursor[0] % len(units)]
                cursor[0] += 1
                solve(p, P)
                done += P.shape[0]
            return done
        todo = units if per_step is None else [units[cursor[0] % len(units)]]
        cursor[0] += 1
        for p, _, P in todo:
            solve(p, P)
            done += P.shape[0]
        return done

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    pts = sum(step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    v = pts / dt / 1e9
    sample = {"learned": "one n = 2^27 instance per step, in turn",
              "box": "one n = 2^26 instance per step, in turn",
              "batched": "consecutive sets up to 1e8 points per step"}.get(
                  args.workload, f"the whole step ({len(units)} instances)")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "Gpoints/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": workload_config(args.workload),
        "cpu_baseline": {"value": v, "unit": "Gpoints/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
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
    u16 = args.workload.endswith("_u16")
    bpp = 4 if u16 else 8  # bytes per point
    host_fmt = [pack_u16(P) if u16 else P for _, P in inputs]
    dev_in = [torch.from_numpy(Q).cuda() for Q in host_fmt]
    hull_fn = ch.ch_convex_hull_u16 if u16 else ch.ch_convex_hull
    nws = ch.ch_convex_hull_workspace_size(n, p)
    # the instances of a step are independent problems: each has its own
    # stream and workspace, so that one instance's latency-bound chain and
    # hull kernels overlap the others' streaming
    wss = [torch.empty(nws, dtype=torch.uint8, device="cuda") for _ in inputs]
    hulls = [torch.empty((2 * p, 2), dtype=torch.int32, device="cuda") for _ in inputs]
    hcs = [torch.empty(1, dtype=torch.int32, device="cuda") for _ in inputs]
    stream = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in inputs]
    # inputs that fit in L2 are evicted before every step (a 256 MB write on
    # the main stream, timed alone and subtracted)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if n * bpp < L2_FLUSH_BELOW else None

    # without a flush between steps, consecutive steps are pipelined: an
    # instance's stream runs that instance's calls in order (one workspace
    # each), and the streams are joined only at the ends of a timed region,
    # so the last instance's chain and final-hull kernels of one step overlap
    # the next step's first instance
    pipelined = flush is None

    def step(concurrent=True):
        if flush is not None:
            flush.zero_()
        if not concurrent:  # one after another on the main stream
            for d, h, c, w in zip(dev_in, hulls, hcs, wss):
                hull_fn(d, p, hull=h, hull_count=c, workspace=w, stream=stream)
            return
        if pipelined:
            for d, h, c, w, st in zip(dev_in, hulls, hcs, wss, streams):
                hull_fn(d, p, hull=h, hull_count=c, workspace=w, stream=st)
            return
        fork = torch.cuda.Event()
        fork.record(stream)
        for d, h, c, w, st in zip(dev_in, hulls, hcs, wss, streams):
            st.wait_event(fork)
            hull_fn(d, p, hull=h, hull_count=c, workspace=w, stream=st)
        for st in streams:
            join = torch.cuda.Event()
            join.record(st)
            stream.wait_event(join)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    rc = _status(ch, None, *streams)
    if rc != ch.CH_OK:
        raise RuntimeError(f"warm-up failed: {ch.strerror(rc)}")

    # value: the timed steps as a user runs them (instances concurrent); then
    # the same steps again with the instances one after another on one stream
    # and CUDA events recorded around every launch of the reduction kernel
    # (the roofline: each launch alone on the GPU); that second region's step
    # time is reported beside the first
    nl = args.steps * len(inputs)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nl)]
    for a, b in evs:
        a.record(stream)
        b.record(stream)
    torch.cuda.synchronize()

    fl = _timed(torch, dist, world, lambda: flush.zero_(), args.steps, stream) if flush is not None else 0.0
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    ms, regions = _timed_regions(torch, dist, world, step, args.steps, stream, args.regions, fl,
                                 side=streams if pipelined else ())
    for _ in range(2):
        step(False)
    ch.ch_trace_set(evs)
    ms_traced = _timed(torch, dist, world, lambda: step(False), args.steps, stream) - fl
    ch.ch_trace_set([])
    clocks = sampler.stop()
    rc = _status(ch, None, *streams)
    if rc != ch.CH_OK:
        raise RuntimeError(f"timed run failed: {ch.strerror(rc)}")
    red_ms = [a.elapsed_time(b) for a, b in evs]
    red_avg = sum(red_ms) / len(red_ms)

    pts_step = n * len(inputs)
    value = world * pts_step * args.steps / (ms / 1e3) / 1e9
    peak, peak_kind = _peaks()

    # e2e through the host-buffer entry point (pinned host memory); the
    # packed format has no host entry point, so its copies are made here
    e2e_steps = max(1, min(args.steps, 5))
    host_in = [torch.from_numpy(Q).pin_memory() for Q in host_fmt]
    hh = torch.empty((2 * p, 2), dtype=torch.int32).pin_memory()
    if u16:
        def e2e_one(i, hp):
            dev_in[i].copy_(hp, non_blocking=True)
            hull_fn(dev_in[i], p, hull=hulls[i], hull_count=hcs[i], workspace=wss[i], stream=stream)
            k = int(hcs[i].item())
            hh[:k].copy_(hulls[i][:k])
            return k
    else:
        nws_h = ch.ch_convex_hull_host_workspace_size(n, p)
        del wss
        ws_h = torch.empty(nws_h, dtype=torch.uint8, device="cuda")

        def e2e_one(i, hp):
            return ch.ch_convex_hull_host(hp, p, ws_h, stream=stream, host_hull=hh).shape[0]
    hsz = []
    for i, hp in enumerate(host_in):  # warm-up
        hsz.append(e2e_one(i, hp))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    d2h = 0
    for _ in range(e2e_steps):
        for i, hp in enumerate(host_in):
            d2h += e2e_one(i, hp) * 8 + 4
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

    kernel_bytes = bpp * n + 8 * p  # points read + L produced, per launch
    achieved = kernel_bytes / (red_avg / 1e3) / 1e9
    kname = KERNEL_OF_FORM[ch.ch_plan_info(n, p)[0]]
    cpu_v, cpu_dt, cpu_passes = cpu_oracle_rate(p, inputs, args.cpu_budget)
    cpu_tn = cpu_andrew_all_points(p, inputs)
    cpu_mt = cpu_reduce_all_cores(p, inputs)
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
        "config": workload_config(args.workload),
        "hbm_frac_step": (pts_step * bpp / (ms / args.steps / 1e3) / 1e9) / peak,
        "roofline": {"bound": "hbm", "kernel": kname,
                     "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "algorithmic_bytes_per_launch": kernel_bytes, "avg_launch_ms": red_avg,
                     "ms_per_step_while_timed": ms_traced / args.steps,
                     "traffic": _traffic(kname, n, p, u16)},
        "e2e": {"value": e2e_val, "unit": "Gpoints/s", "h2d_bytes_per_step": pts_step * bpp,
                "d2h_bytes_per_step": d2h // e2e_steps, "steps": e2e_steps},
        "cpu_baseline": {"value": cpu_v, "unit": "Gpoints/s", "cores": 1, "kind": "oracle",
                         "sample": f"{cpu_passes} pass(es) over the step's {len(inputs)} instances "
                                   f"({cpu_dt:.1f} s, single thread)",
                         "hull_of_all_points": cpu_tn, "reduce_all_cores": cpu_mt},
        "gpu_launches": args.steps * len(inputs) * ch.ch_plan_info(n, p)[1],
        "clocks": clocks,
        "l2_flush_ms_subtracted": fl / args.steps,
        "timed_regions": {"count": len(regions), "steps_each": args.steps,
                          "ms_per_step_each": [t / args.steps for t in regions],
                          "reported": "median region"},
        "hull_vertices": hsz,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


LEARNED = (65536, 1 << 27, ("uniform", "disc", "gaussian", "annulus"))
# Steps 1-2: (distribution, box width, box height, x0, y0) per instance
BOX_N = 1 << 26
BOX = (("uniform", 65536, 65536, -1_500_000_000, 700_000_000),
       ("disc", 120_000, 40_000, 1_000_000_000, -2_000_000_000),
       ("gaussian", 30_000, 90_000, -123_456_789, 987_654_321))
MELKMAN = "projected_shells"
# sparse regime p > n: side, points per instance, distributions
SPARSE = (1 << 24, 1 << 20, ("uniform", "disc", "gaussian"))
SPARSE_DENSITIES = (0.05, 0.25, 0.45, 0.65, 0.85)


def box_inputs(rank):
    from paper_1505_00914_gb300 import synth
    return [(d, synth.boxed(d, BOX_N, sx, sy, x0, y0, seed=31 + 1000 * rank + i))
            for i, (d, sx, sy, x0, y0) in enumerate(BOX)]
WEIGHTS = os.path.join(ROOT, "paper_1505_00914_gb300", "weights", "cull_mlp_k16.npz")
BATCH_SETS = 10_000
PROFILE_BATCH_SETS = 1_000  # the profiling case of the batched kernel (~0.9 GB of points)


def _setup_dist():
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
    return torch, dist, world, rank


def _max_over_ranks(torch, dist, world, v):
    if world == 1:
        return v
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _status(ch, *streams):
    """The first error recorded on any of the given streams (None: torch's
    current stream); every stream's status word is read and cleared."""
    rc = ch.CH_OK
    for st in streams:
        r = ch.ch_sync_status(st)
        if rc == ch.CH_OK:
            rc = r
    return rc


def _timed_regions(torch, dist, world, fn, steps, stream, regions, offset=0.0, side=()):
    """`regions` timed regions of exactly `steps` calls of fn each, back to
    back (each bracketed by a barrier and a synchronize on both sides, max
    over ranks); returns (median region ms minus offset, [every region's ms
    minus offset]).  More than one region keeps the GPU under load long
    enough for the clock sampler to see it several times."""
    ts = [_timed(torch, dist, world, fn, steps, stream, side) - offset
          for _ in range(max(1, regions))]
    return statistics.median(ts), ts


def _timed(torch, dist, world, fn, steps, stream, side=()):
    """Device time in ms of `steps` calls of fn, barrier + synchronize on
    both sides, max over ranks.  side: streams fn also launches on without
    joining them itself (pipelined steps): they start after the region's
    start event and the end event waits for all of them."""
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for st in side:
        st.wait_event(a)
    for _ in range(steps):
        fn()
    for st in side:
        j = torch.cuda.Event()
        j.record(st)
        stream.wait_event(j)
    b.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    return _max_over_ranks(torch, dist, world, a.elapsed_time(b))


def run_learned(args):
    torch, dist, world, rank = _setup_dist()
    from paper_1505_00914_gb300 import ch, synth, train
    ch.lib()
    p, n, dists = LEARNED
    inputs = [(d, synth.points(d, n, p, seed=101 + 1000 * rank + i)) for i, d in enumerate(dists)]
    dev_in = [torch.from_numpy(P).cuda() for _, P in inputs]
    have_w = os.path.exists(WEIGHTS)
    params = train.load_params(WEIGHTS) if have_w else None
    nws = max(ch.ch_hull_learned_workspace_size(n, p), ch.ch_convex_hull_workspace_size(n, p))
    # as in the plain workload, the independent instances of a step run on
    # their own streams and workspaces, in every arm alike
    wss = [torch.empty(nws, dtype=torch.uint8, device="cuda") for _ in inputs]
    ws = wss[0]
    stream = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in inputs]
    arms = ("learned", "centres", "plain")
    hulls = {a: [torch.empty((2 * p, 2), dtype=torch.int32, device="cuda") for _ in inputs] for a in arms}
    hcs = {a: [torch.empty(1, dtype=torch.int32, device="cuda") for _ in inputs] for a in arms}
    Linit = {a: [torch.empty((p, 2), dtype=torch.int32, device="cuda") for _ in inputs]
             for a in ("learned", "centres")}

    # as in the plain workload, consecutive steps are pipelined on the
    # instances' streams (joined at the ends of a timed region), in every arm
    def step(arm, concurrent=True, pipelined=False):
        sts = streams if concurrent else [stream] * len(inputs)
        fork_join = concurrent and not pipelined
        if fork_join:
            fork = torch.cuda.Event()
            fork.record(stream)
        for i, d in enumerate(dev_in):
            h, c, st = hulls[arm][i], hcs[arm][i], sts[i]
            if fork_join:
                st.wait_event(fork)
            if arm == "plain":
                ch.ch_convex_hull(d, p, hull=h, hull_count=c, workspace=wss[i], stream=st)
            else:
                ch.ch_hull_learned(d, p, params=params if arm == "learned" else None,
                                   Linit=Linit[arm][i], hull=h, hull_count=c, workspace=wss[i],
                                   stream=st)
        if fork_join:
            for st in streams:
                join = torch.cuda.Event()
                join.record(st)
                stream.wait_event(join)

    for arm in arms:
        for _ in range(args.warmup):
            step(arm)
    torch.cuda.synchronize()
    rc = _status(ch, None, *streams)
    if rc != ch.CH_OK:
        raise RuntimeError(f"warm-up failed: {ch.strerror(rc)}")
    # every arm must give the same hull
    exact = True
    hv = []
    for i in range(len(inputs)):
        ref = hulls["plain"][i][: int(hcs["plain"][i].item())].cpu()
        hv.append(ref.shape[0])
        for arm in ("learned", "centres"):
            got = hulls[arm][i][: int(hcs[arm][i].item())].cpu()
            exact &= bool(torch.equal(got, ref))
    # cull rate: share of the points strictly inside the culling polygon
    # (Linit.lo <= y <= Linit.hi in their column), counted by the library
    # (the call's ch_cull_stats output; one untimed call per instance and arm)
    cull = {}
    for i, (dname, _) in enumerate(inputs):
        cull[dname] = {}
        for arm in ("learned", "centres"):
            stt = ch.cull_stats_tensor()
            ch.ch_hull_learned(dev_in[i], p, params=params if arm == "learned" else None,
                               hull=hulls[arm][i], hull_count=hcs[arm][i], stats=stt,
                               workspace=wss[i], stream=stream)
            cs = ch.cull_stats(stt)
            cull[dname][arm] = cs["culled"] / n
            cull[dname][arm + "_polygon_vertices"] = cs["poly_vertices"]

    # the network's gain on held-out stretched and rotated shapes of the
    # training family (seeds the training set never used)
    stretched = {"network": [], "centres": [], "network_polygon_used": 0, "sets": 0}
    if params is not None:
        rng = np.random.default_rng(4242)
        for t in range(16):
            dname = ("uniform", "disc", "gaussian", "shells")[t % 4]
            ps_ = int(rng.choice([1024, 4096, 16384, 65536]))
            Q = synth.affine(synth.points(dname, 300_000, ps_, seed=20_000_000 + t), ps_,
                             seed=20_000_000 + t)
            dq = torch.from_numpy(Q).cuda()
            for arm, prm in (("network", params), ("centres", None)):
                o = ch.ch_cull_propose(dq, ps_, params=prm)
                li = o["Linit"].long()
                col = li[dq[:, 0].long() - 1]
                yq = dq[:, 1].long()
                stretched[arm].append(float(((yq >= col[:, 0]) & (yq <= col[:, 1])).float().mean()))
                if arm == "network":
                    stretched["network_polygon_used"] += int(o["chosen"].item() == 1)
            stretched["sets"] += 1
        for arm in ("network", "centres"):
            stretched[arm] = float(np.mean(stretched[arm]))

    nl = args.steps * len(inputs)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nl)]
    for a, b in evs:
        a.record(stream)
        b.record(stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    ms = {}
    for arm in ("learned", "plain", "centres"):
        ms[arm] = _timed(torch, dist, world, lambda arm=arm: step(arm, pipelined=True), args.steps,
                         stream, side=streams)
    for _ in range(2):
        step("learned", False)
    ch.ch_trace_set(evs)  # the learned arm again, one instance after another, reductions timed
    ms_traced = _timed(torch, dist, world, lambda: step("learned", False), args.steps, stream)
    ch.ch_trace_set([])
    clocks = sampler.stop()
    rc = _status(ch, None, *streams)
    if rc != ch.CH_OK:
        raise RuntimeError(f"timed run failed: {ch.strerror(rc)}")
    red_avg = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
    pts_step = n * len(inputs)
    rate = {arm: world * pts_step * args.steps / (t / 1e3) / 1e9 for arm, t in ms.items()}

    # e2e: pinned host points -> device, the learned path, hull back to the host
    e2e_steps = max(1, min(args.steps, 3))
    host_in = [torch.from_numpy(P).pin_memory() for _, P in inputs]
    hh = torch.empty((2 * p, 2), dtype=torch.int32).pin_memory()
    hc_h = torch.empty(1, dtype=torch.int32).pin_memory()
    d2h = 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        for i, hp in enumerate(host_in):
            dev_in[i].copy_(hp, non_blocking=True)
            ch.ch_hull_learned(dev_in[i], p, params=params, hull=hulls["learned"][i],
                               hull_count=hcs["learned"][i], workspace=ws, stream=stream)
            hc_h.copy_(hcs["learned"][i], non_blocking=True)
            torch.cuda.synchronize()
            k = int(hc_h[0])
            hh[:k].copy_(hulls["learned"][i][:k], non_blocking=True)
            torch.cuda.synchronize()
            d2h += 4 + 8 * k
    e2e_s = _max_over_ranks(torch, dist, world, time.perf_counter() - w0)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    kernel_bytes = 8 * n + 8 * p
    achieved = kernel_bytes / (red_avg / 1e3) / 1e9
    cpu_v, cpu_dt, cpu_passes = cpu_oracle_rate(p, inputs[:1], args.cpu_budget)
    kl = ch.ch_hull_learned_kernel_count(n, p, params is not None)
    line = {
        "metric": METRIC, "value": rate["learned"], "unit": "Gpoints/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms["learned"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": workload_config("learned"),
        "learned": {"network": "trained weights" if have_w else "none found: sector centres",
                    "plain_gpoints_s": rate["plain"], "centres_gpoints_s": rate["centres"],
                    "speedup_vs_plain": rate["learned"] / rate["plain"],
                    "speedup_vs_centres": rate["learned"] / rate["centres"],
                    "ms_per_step": {a: t / args.steps for a, t in ms.items()},
                    "cull_rate": cull, "hulls_identical": exact, "hull_vertices": hv,
                    "cull_rate_stretched_heldout": stretched},
        "roofline": {"bound": "hbm", "kernel": KERNEL_OF_FORM[ch.ch_plan_info(n, p)[0]],
                     "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "algorithmic_bytes_per_launch": kernel_bytes, "avg_launch_ms": red_avg,
                     "ms_per_step_while_timed": ms_traced / args.steps,
                     "traffic": _traffic(KERNEL_OF_FORM[ch.ch_plan_info(n, p)[0]], n, p)},
        "e2e": {"value": world * pts_step * e2e_steps / e2e_s / 1e9, "unit": "Gpoints/s",
                "h2d_bytes_per_step": pts_step * 8, "d2h_bytes_per_step": d2h // e2e_steps,
                "steps": e2e_steps},
        "cpu_baseline": {"value": cpu_v, "unit": "Gpoints/s", "cores": 1, "kind": "oracle",
                         "sample": f"{cpu_passes} pass(es) over the {inputs[0][0]} instance "
                                   f"({cpu_dt:.1f} s, single thread, Algorithm 1 + hull)"},
        "gpu_launches": args.steps * len(inputs) * kl,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batched(args):
    torch, dist, world, rank = _setup_dist()
    from paper_1505_00914_gb300 import autotune, ch, synth
    ch.lib()
    sets = BATCH_SETS if args.workload == "batched" else PROFILE_BATCH_SETS
    pts, off, ps, _ = synth.batched(sets, seed=4 + 1000 * rank)
    ps = ps.astype(np.int32)
    B = len(ps)
    n_tot = int(off[-1])
    d_pts = torch.from_numpy(pts).cuda()
    d_off = torch.from_numpy(off).cuda()
    d_ps = torch.from_numpy(ps).cuda()
    hoff = ch.hull_capacity_offsets(off, ps)
    d_hoff = torch.from_numpy(hoff).cuda()
    hull = torch.zeros((int(hoff[-1]), 2), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(B, dtype=torch.int32, device="cuda")
    if args.no_aux:  # profiling runs: the usual choice, no tuning launches
        (best, fold), tune_ms = (1024, ch.CH_BATCH_FOLD_DEFAULT), {}
    else:
        (best, fold), tune_ms = autotune.tune_batched(d_pts, off, ps, d_off, d_ps, hull, d_hoff, cnt)
    ws = torch.empty(ch.ch_batched_workspace_size(off, ps, best), dtype=torch.uint8, device="cuda")
    ch.ch_batched_prepare(off, ps, ws, best, fold_threads=fold)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ch.ch_hull_batched(d_pts, d_off, d_ps, hull, d_hoff, cnt, ws)  # first call: set-up
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        ch.ch_hull_batched(d_pts, d_off, d_ps, hull, d_hoff, cnt, ws)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    rc = _status(ch, stream, None)
    if rc != ch.CH_OK:
        raise RuntimeError(f"warm-up failed: {ch.strerror(rc)}")
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    cur = torch.cuda.current_stream()
    ms, regions = _timed_regions(torch, dist, world, graph.replay, args.steps, cur, args.regions)
    clocks = sampler.stop()
    # per-set plain launches on the same data (one pass, same stream)
    pmax = int(ps.max())
    ws1 = torch.empty(ch.ch_convex_hull_workspace_size(int(np.diff(off).max()), pmax),
                      dtype=torch.uint8, device="cuda")
    h1 = torch.empty((B, 2 * pmax, 2), dtype=torch.int32, device="cuda")
    c1 = torch.empty((B, 1), dtype=torch.int32, device="cuda")
    views = [d_pts[off[s]:off[s + 1]] for s in range(B)]

    def per_set():
        for s in range(B):
            ch.ch_convex_hull(views[s], int(ps[s]), hull=h1[s], hull_count=c1[s], workspace=ws1,
                              stream=cur)

    per_set()  # warm-up
    ms_plain = _timed(torch, dist, world, per_set, 1, cur)
    # the same per-set calls captured in one CUDA graph (no host launch cost)
    gstream = torch.cuda.Stream()
    gstream.wait_stream(cur)
    per_graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(per_graph, stream=gstream):
        for s in range(B):
            ch.ch_convex_hull(views[s], int(ps[s]), hull=h1[s], hull_count=c1[s], workspace=ws1,
                              stream=gstream)
    per_graph.replay()  # warm-up
    ms_plain_graph = _timed(torch, dist, world, per_graph.replay, 1, cur)
    rc = _status(ch, stream, cur, gstream)
    if rc != ch.CH_OK:
        raise RuntimeError(f"timed run failed: {ch.strerror(rc)}")
    # identical hulls, set by set
    cnt_h, c1_h = cnt.cpu().numpy(), c1.cpu().numpy()[:, 0]
    hull_h, h1_h = hull.cpu().numpy(), h1.cpu().numpy()
    exact = bool(np.array_equal(cnt_h, c1_h)) and all(
        np.array_equal(hull_h[hoff[s]:hoff[s] + cnt_h[s]], h1_h[s, :cnt_h[s]]) for s in range(B))
    # e2e: points from pinned host memory, the graph, hull counts and hulls back
    host_pts = torch.from_numpy(pts).pin_memory()
    host_hull = torch.empty_like(hull, device="cpu").pin_memory()
    host_cnt = torch.empty_like(cnt, device="cpu").pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        d_pts.copy_(host_pts, non_blocking=True)
        graph.replay()
        host_cnt.copy_(cnt, non_blocking=True)
        host_hull.copy_(hull, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = _max_over_ranks(torch, dist, world, time.perf_counter() - w0)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    rate = world * n_tot * args.steps / (ms / 1e3) / 1e9
    kernel_bytes = 8 * n_tot
    achieved = kernel_bytes / (ms / args.steps / 1e3) / 1e9
    # CPU oracle on a bounded sample of the sets
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    done = 0
    s = 0
    while time.perf_counter() - t0 < args.cpu_budget and s < B:
        oracle.hull_chain(oracle.reduce(pts[off[s]:off[s + 1]], int(ps[s])))
        done += int(off[s + 1] - off[s])
        s += 1
    cpu_dt = time.perf_counter() - t0
    line = {
        "metric": METRIC, "value": rate, "unit": "Gpoints/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": workload_config(args.workload),
        "batched": {"points": n_tot, "chunk_mult": best, "fold_threads": fold,
                    "launch": "one captured CUDA graph replay per step",
                    "per_set_plain_gpoints_s": world * n_tot / (ms_plain / 1e3) / 1e9,
                    "per_set_plain_ms": ms_plain, "speedup_vs_per_set": ms_plain / (ms / args.steps),
                    "per_set_plain_graph_ms": ms_plain_graph,
                    "per_set_plain_graph_gpoints_s": world * n_tot / (ms_plain_graph / 1e3) / 1e9,
                    "speedup_vs_per_set_graph": ms_plain_graph / (ms / args.steps),
                    "hulls_identical": exact, "autotune_ms": tune_ms},
        "roofline": {"bound": "hbm", "kernel": "k_batched", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "algorithmic_bytes_per_launch": kernel_bytes,
                     "avg_launch_ms": ms / args.steps, "traffic": None},
        "e2e": {"value": world * n_tot * e2e_steps / e2e_s / 1e9, "unit": "Gpoints/s",
                "h2d_bytes_per_step": 8 * n_tot,
                "d2h_bytes_per_step": int(host_hull.numel() * 4 + host_cnt.numel() * 4),
                "steps": e2e_steps},
        "cpu_baseline": {"value": done / cpu_dt / 1e9, "unit": "Gpoints/s", "cores": 1,
                         "kind": "oracle", "sample": f"first {s} of {B} sets ({done} points, "
                                                     f"{cpu_dt:.1f} s, single thread)"},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "timed_regions": {"count": len(regions), "steps_each": args.steps,
                          "ms_per_step_each": [t / args.steps for t in regions],
                          "reported": "median region"},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_box(args):
    """Steps 1-2 (bounding box, translation fused into Algorithm 1, columns
    along the shorter side) on int32 points anywhere."""
    torch, dist, world, rank = _setup_dist()
    from paper_1505_00914_gb300 import ch
    ch.lib()
    inputs = box_inputs(rank)
    n = BOX_N
    dev_in = [torch.from_numpy(P).cuda() for _, P in inputs]
    stream = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in inputs]
    boxes_d = [torch.empty(4, dtype=torch.int32, device="cuda") for _ in inputs]
    boxes_h = torch.empty((len(inputs), 4), dtype=torch.int32).pin_memory()
    bws = [torch.empty(max(ch._size(ch.lib().ch_bbox_workspace_size), 1), dtype=torch.uint8,
                       device="cuda") for _ in inputs]
    # the boxes are known from the data; size the workspaces once
    truth = [np.array([P[:, 0].min(), P[:, 0].max(), P[:, 1].min(), P[:, 1].max()], np.int32)
             for _, P in inputs]
    side = [int(min(b[1] - b[0], b[3] - b[2])) + 1 for b in truth]
    wss = [torch.empty(ch.ch_convex_hull_box_workspace_size(n, b), dtype=torch.uint8, device="cuda")
           for b in truth]
    hulls = [torch.empty((2 * s + 2, 2), dtype=torch.int32, device="cuda") for s in side]
    hcs = [torch.empty(1, dtype=torch.int32, device="cuda") for _ in inputs]

    def step(concurrent=True):
        sts = streams if concurrent else [stream] * len(inputs)
        fork = torch.cuda.Event()
        fork.record(stream)
        for i, st in enumerate(sts):
            st.wait_event(fork)
            ch.ch_bbox(dev_in[i], box=boxes_d[i], workspace=bws[i], stream=st)
            with torch.cuda.stream(st):
                boxes_h[i].copy_(boxes_d[i], non_blocking=True)
        for st in set(sts):
            st.synchronize()  # the one host read of the boxes
        for i, st in enumerate(sts):
            ch.ch_convex_hull_box(dev_in[i], boxes_h[i].numpy(), hull=hulls[i], hull_count=hcs[i],
                                  workspace=wss[i], stream=st)
        for st in set(sts):
            if st is not stream:
                join = torch.cuda.Event()
                join.record(st)
                stream.wait_event(join)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    rc = _status(ch, None, *streams)
    if rc != ch.CH_OK:
        raise RuntimeError(f"warm-up failed: {ch.strerror(rc)}")
    for i in range(len(inputs)):
        if not np.array_equal(boxes_h[i].numpy(), truth[i]):
            raise RuntimeError("bounding box mismatch")
    nl = args.steps * len(inputs)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nl)]
    for a, b in evs:
        a.record(stream)
        b.record(stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    ms = _timed(torch, dist, world, step, args.steps, stream)
    for _ in range(2):
        step(False)
    ch.ch_trace_set(evs)
    ms_traced = _timed(torch, dist, world, lambda: step(False), args.steps, stream)
    ch.ch_trace_set([])
    clocks = sampler.stop()
    rc = _status(ch, None, *streams)
    if rc != ch.CH_OK:
        raise RuntimeError(f"timed run failed: {ch.strerror(rc)}")
    # launches follow the instances in order: the reduction of instance i
    # is evs[k] with k % 3 == i
    red = [a.elapsed_time(b) for a, b in evs]
    pts_step = n * len(inputs)
    value = world * pts_step * args.steps / (ms / 1e3) / 1e9
    hv = [int(c.item()) for c in hcs]

    # e2e: pinned host points -> device, the same step, hulls back to the host
    e2e_steps = max(1, min(args.steps, 3))
    host_in = [torch.from_numpy(P).pin_memory() for _, P in inputs]
    hh = [torch.empty(tuple(h.shape), dtype=torch.int32).pin_memory() for h in hulls]
    d2h = 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        for i, hp in enumerate(host_in):
            dev_in[i].copy_(hp, non_blocking=True)
        step()
        torch.cuda.synchronize()
        for i in range(len(inputs)):
            k = int(hcs[i].item())
            hh[i][:k].copy_(hulls[i][:k])
            d2h += 4 + 8 * k
    e2e_s = _max_over_ranks(torch, dist, world, time.perf_counter() - w0)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    # dominant kernel: the main reduction of the largest frame (instance 0,
    # 65536 columns); per launch it reads the points and writes L
    red0 = [red[k] for k in range(0, len(red), len(inputs))]
    red0_avg = sum(red0) / len(red0)
    kernel_bytes = 8 * n + 8 * side[0]
    achieved = kernel_bytes / (red0_avg / 1e3) / 1e9
    cpu_v, cpu_dt, cpu_passes = _cpu_rate(oracle_solver("box"), [(None, P) for _, P in inputs[:1]],
                                          args.cpu_budget)
    line = {
        "metric": METRIC, "value": value, "unit": "Gpoints/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": workload_config("box"),
        "hbm_frac_step": (pts_step * 16 / (ms / args.steps / 1e3) / 1e9) / peak,
        "box": {"columns": side, "transposed": [bool(b[3] - b[2] < b[1] - b[0]) for b in truth],
                "reduction_ms_per_instance": [sum(red[i::len(inputs)]) / args.steps
                                              for i in range(len(inputs))],
                "hull_vertices": hv,
                "note": "two passes over the points per instance (bounding box, then the "
                        "reduction) and one 16-byte host read of the boxes per step"},
        "roofline": {"bound": "hbm", "kernel": KERNEL_OF_FORM[ch.ch_plan_info(n, side[0])[0]],
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "algorithmic_bytes_per_launch": kernel_bytes,
                     "avg_launch_ms": red0_avg, "ms_per_step_while_timed": ms_traced / args.steps,
                     "traffic": None},
        "e2e": {"value": world * pts_step * e2e_steps / e2e_s / 1e9, "unit": "Gpoints/s",
                "h2d_bytes_per_step": pts_step * 8, "d2h_bytes_per_step": d2h // e2e_steps,
                "steps": e2e_steps},
        "cpu_baseline": {"value": cpu_v, "unit": "Gpoints/s", "cores": 1, "kind": "oracle",
                         "sample": f"{cpu_passes} pass(es) over the uniform instance "
                                   f"({cpu_dt:.1f} s, single thread, Steps 1-2 + Algorithm 1 "
                                   f"+ hull)"},
        "gpu_launches": args.steps * len(inputs) * (2 + ch.ch_plan_info(n, side[0])[1] + 1),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _cpu_rate(solve, problems, budget_s):
    """Points per second of the oracle over (p, points) problems, repeated
    until about budget_s elapsed."""
    done, passes, t0 = 0, 0, time.perf_counter()
    while True:
        for p, P in problems:
            solve(p, P)
            done += P.shape[0]
        passes += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return done / dt / 1e9, dt, passes


def run_alt(args):
    """One alternative form of the path against the plain path, on the
    projected-shells stand-in for the paper's scans (p = 4096, 10^7 points):
    `melkman` - Algorithm 1, the Lemma 1 polyline and Melkman's hull
    (Section 3, Fig. 10); `rxy` - Algorithm 1 along x, the second scan along y
    and the hull of the rxy points (Section 2, Figs. 4 and 7)."""
    torch, dist, world, rank = _setup_dist()
    from paper_1505_00914_gb300 import ch
    ch.lib()
    alt = args.workload
    p, n, inputs = gen_inputs(MELKMAN, rank)
    P = inputs[0][1]
    d = torch.from_numpy(P).cuda()
    stream = torch.cuda.current_stream()
    if alt == "melkman":
        ws_a = torch.empty(ch.ch_convex_hull_melkman_workspace_size(n, p), dtype=torch.uint8,
                           device="cuda")
    else:
        ws_a = torch.empty(ch.ch_convex_hull_rxy_workspace_size(n, p), dtype=torch.uint8,
                           device="cuda")
    ws_p = torch.empty(ch.ch_convex_hull_workspace_size(n, p), dtype=torch.uint8, device="cuda")
    poly = torch.empty((2 * p, 2), dtype=torch.int32, device="cuda")
    pc = torch.empty(1, dtype=torch.int32, device="cuda")
    La = torch.empty((p, 2), dtype=torch.int32, device="cuda")
    Ra = torch.empty((p, 2), dtype=torch.int32, device="cuda")
    ha, hca = torch.empty((2 * p, 2), dtype=torch.int32, device="cuda"), torch.empty(1, dtype=torch.int32, device="cuda")
    hp, hcp = torch.empty((2 * p, 2), dtype=torch.int32, device="cuda"), torch.empty(1, dtype=torch.int32, device="cuda")
    # the input (80 MB) fits in L2: each step starts after a 256 MB write
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def run_alt_once():
        if alt == "melkman":
            ch.ch_convex_hull_melkman(d, p, poly=poly, poly_count=pc, hull=ha, hull_count=hca,
                                      workspace=ws_a, stream=stream)
        else:
            ch.ch_convex_hull_rxy(d, p, L=La, R=Ra, hull=ha, hull_count=hca, workspace=ws_a,
                                  stream=stream)

    def step(arm):
        flush.zero_()
        if arm == alt:
            run_alt_once()
        else:
            ch.ch_convex_hull(d, p, hull=hp, hull_count=hcp, workspace=ws_p, stream=stream)

    for arm in (alt, "plain"):
        for _ in range(args.warmup):
            step(arm)
    torch.cuda.synchronize()
    rc = _status(ch, None)
    if rc != ch.CH_OK:
        raise RuntimeError(f"warm-up failed: {ch.strerror(rc)}")
    same = bool(torch.equal(ha[: int(hca.item())].cpu(), hp[: int(hcp.item())].cpu()))
    detail = {"polyline_vertices_after_prefilter": int(pc.item())} if alt == "melkman" else {}
    if alt == "melkman" and not args.no_aux:
        # the paper's exact pipeline as well: the full Lemma 1 polyline
        # (ch_polyline) and Melkman on it (ch_hull_melkman)
        L1 = ch.ch_reduce(d, p)
        full, fc = ch.ch_polyline(L1, p)
        ws_m = ch.ch_hull_melkman_workspace_size(p)
        wsm = torch.empty(max(ws_m, 1), dtype=torch.uint8, device="cuda")
        for _ in range(3):
            ch.ch_hull_melkman(full, fc, p, workspace=wsm, stream=stream)
        t = _timed(torch, dist, world, lambda: ch.ch_hull_melkman(full, fc, p, workspace=wsm,
                                                                  stream=stream), 5, stream)
        detail = {"polyline_vertices": int(fc.item()),
                  "polyline_vertices_after_prefilter": int(pc.item()),
                  "melkman_ms_on_full_polyline": t / 5}
    else:
        Lh, Rh = La.cpu().numpy(), Ra.cpu().numpy()
        vl = ~((Lh[:, 0] == p + 1) & (Lh[:, 1] == -1))
        vr = ~((Rh[:, 0] == p + 1) & (Rh[:, 1] == -1))
        detail = {"rx": int(vl.sum() + (vl & (Lh[:, 0] != Lh[:, 1])).sum()),
                  "rxy": int(vr.sum() + (vr & (Rh[:, 0] != Rh[:, 1])).sum())}
    fl = _timed(torch, dist, world, lambda: flush.zero_(), args.steps, stream)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for a, b in evs:
        a.record(stream)
        b.record(stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    ms = {arm: _timed(torch, dist, world, lambda arm=arm: step(arm), args.steps, stream) - fl
          for arm in (alt, "plain")}
    ch.ch_trace_set(evs)
    ms_traced = _timed(torch, dist, world, lambda: step(alt), args.steps, stream) - fl
    ch.ch_trace_set([])
    clocks = sampler.stop()
    rc = _status(ch, None)
    if rc != ch.CH_OK:
        raise RuntimeError(f"timed run failed: {ch.strerror(rc)}")
    red_avg = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
    rate = {arm: world * n * args.steps / (t / 1e3) / 1e9 for arm, t in ms.items()}

    e2e_steps = max(1, min(args.steps, 5))
    host_in = torch.from_numpy(P).pin_memory()
    hh = torch.empty((2 * p, 2), dtype=torch.int32).pin_memory()
    d2h = 0
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        d.copy_(host_in, non_blocking=True)
        run_alt_once()
        k = int(hca.item())
        hh[:k].copy_(ha[:k])
        d2h += 4 + 8 * k
    e2e_s = _max_over_ranks(torch, dist, world, time.perf_counter() - w0)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    kname = KERNEL_OF_FORM[ch.ch_plan_info(n, p)[0]]
    kernel_bytes = 8 * n + 8 * p
    achieved = kernel_bytes / (red_avg / 1e3) / 1e9
    cpu_v, cpu_dt, cpu_passes = _cpu_rate(oracle_solver(alt), [(p, P)], args.cpu_budget)
    # reduce kernels + (polyline, Melkman) or (fill, row scan, chain, final, unframe)
    nk = ch.ch_plan_info(n, p)[1] - 2 + (2 if alt == "melkman" else 5)
    what = {"melkman": "Algorithm 1 + polyline + Melkman",
            "rxy": "Algorithm 1 + second scan + hull"}[alt]
    line = {
        "metric": METRIC, "value": rate[alt], "unit": "Gpoints/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms[alt] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": workload_config(alt),
        alt: dict({"plain_gpoints_s": rate["plain"],
                   "ms_per_step": {a: t / args.steps for a, t in ms.items()},
                   "reduction_ms": red_avg,
                   "after_reduction_ms": ms_traced / args.steps - red_avg,
                   "hull_vertices": int(hca.item()), "hulls_identical": same,
                   "l2_flush_ms_subtracted": fl / args.steps}, **detail),
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "algorithmic_bytes_per_launch": kernel_bytes, "avg_launch_ms": red_avg,
                     "ms_per_step_while_timed": ms_traced / args.steps, "traffic": None},
        "e2e": {"value": world * n * e2e_steps / e2e_s / 1e9, "unit": "Gpoints/s",
                "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": d2h // e2e_steps,
                "steps": e2e_steps},
        "cpu_baseline": {"value": cpu_v, "unit": "Gpoints/s", "cores": 1, "kind": "oracle",
                         "sample": f"{cpu_passes} pass(es) over the instance ({cpu_dt:.1f} s, "
                                   f"single thread, {what})"},
        "gpu_launches": args.steps * nk,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_sparse(args):
    """The tree of bit words against the array L of p entries, p > n."""
    torch, dist, world, rank = _setup_dist()
    from paper_1505_00914_gb300 import ch, synth
    ch.lib()
    p, n, dists = SPARSE
    inputs = [(d, synth.points(d, n, p, seed=51 + 1000 * rank + i)) for i, d in enumerate(dists)]
    dev_in = [torch.from_numpy(P).cuda() for _, P in inputs]
    stream = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in inputs]
    ws_s = [ch.ch_sparse_workspace(n, p) for _ in inputs]
    ws_p = [torch.empty(ch.ch_convex_hull_workspace_size(n, p), dtype=torch.uint8, device="cuda")
            for _ in inputs]
    cap = min(p, n)
    out = {a: [(torch.empty((2 * cap, 2), dtype=torch.int32, device="cuda"),
                torch.empty(1, dtype=torch.int32, device="cuda")) for _ in inputs]
           for a in ("sparse", "plain")}
    cnts = [torch.empty(2, dtype=torch.int32, device="cuda") for _ in inputs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def run(arm, i, st):
        h, hc = out[arm][i]
        if arm == "sparse":
            ch.ch_convex_hull_sparse(dev_in[i], p, ws_s[i], counts=cnts[i], hull=h, hull_count=hc,
                                     stream=st)
        else:
            ch.ch_convex_hull(dev_in[i], p, hull=h, hull_count=hc, workspace=ws_p[i], stream=st)

    def step(arm, concurrent=True):
        flush.zero_()
        if not concurrent:
            for i in range(len(inputs)):
                run(arm, i, stream)
            return
        fork = torch.cuda.Event()
        fork.record(stream)
        for i, st in enumerate(streams):
            st.wait_event(fork)
            run(arm, i, st)
        for st in streams:
            join = torch.cuda.Event()
            join.record(st)
            stream.wait_event(join)

    for arm in ("sparse", "plain"):
        for _ in range(args.warmup):
            step(arm)
    torch.cuda.synchronize()
    rc = _status(ch, None, *streams)
    if rc != ch.CH_OK:
        raise RuntimeError(f"warm-up failed: {ch.strerror(rc)}")
    same = all(torch.equal(out["sparse"][i][0][: int(out["sparse"][i][1].item())].cpu(),
                           out["plain"][i][0][: int(out["plain"][i][1].item())].cpu())
               for i in range(len(inputs)))
    cols = [int(c[0].item()) for c in cnts]
    fl = _timed(torch, dist, world, lambda: flush.zero_(), args.steps, stream)
    nl = args.steps * len(inputs)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nl)]
    for a, b in evs:
        a.record(stream)
        b.record(stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    ms = {arm: _timed(torch, dist, world, lambda arm=arm: step(arm), args.steps, stream) - fl
          for arm in ("sparse", "plain")}
    ch.ch_trace_set(evs)
    ms_traced = _timed(torch, dist, world, lambda: step("sparse", False), args.steps, stream) - fl
    ch.ch_trace_set([])
    # Fig. 11: both paths at column densities s/p (uniform x), one instance each
    sweep = []
    for dens in (() if args.no_aux else SPARSE_DENSITIES):
        nd = int(round(-p * np.log1p(-dens)))
        Q = torch.from_numpy(synth.points("uniform", nd, p, seed=61)).cuda()
        wsd = ch.ch_sparse_workspace(nd, p)
        wpd = torch.empty(ch.ch_convex_hull_workspace_size(nd, p), dtype=torch.uint8, device="cuda")
        hd = torch.empty((2 * min(p, nd), 2), dtype=torch.int32, device="cuda")
        hcd = torch.empty(1, dtype=torch.int32, device="cuda")
        cd = torch.empty(2, dtype=torch.int32, device="cuda")
        fns = {"sparse": lambda: ch.ch_convex_hull_sparse(Q, p, wsd, counts=cd, hull=hd,
                                                          hull_count=hcd, stream=stream),
               "array": lambda: ch.ch_convex_hull(Q, p, hull=hd, hull_count=hcd, workspace=wpd,
                                                  stream=stream)}
        row = {"density_target": dens, "n": nd}
        for k, fn in fns.items():
            for _ in range(3):
                fn()
            reps = 5
            t = _timed(torch, dist, world, lambda fn=fn: (flush.zero_(), fn()), reps, stream)
            row[k + "_ms"] = (t - fl / args.steps * reps) / reps
        row["density"] = int(cd[0].item()) / p
        sweep.append(row)
        del wsd, wpd, Q
    clocks = sampler.stop()
    rc = _status(ch, None, *streams)
    if rc != ch.CH_OK:
        raise RuntimeError(f"timed run failed: {ch.strerror(rc)}")
    red_avg = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
    pts_step = n * len(inputs)
    rate = {arm: world * pts_step * args.steps / (t / 1e3) / 1e9 for arm, t in ms.items()}

    e2e_steps = max(1, min(args.steps, 5))
    host_in = [torch.from_numpy(P).pin_memory() for _, P in inputs]
    hh = torch.empty((2 * cap, 2), dtype=torch.int32).pin_memory()
    d2h = 0
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        for i, hp in enumerate(host_in):
            dev_in[i].copy_(hp, non_blocking=True)
            run("sparse", i, stream)
            k = int(out["sparse"][i][1].item())
            hh[:k].copy_(out["sparse"][i][0][:k])
            d2h += 4 + 8 * k
    e2e_s = _max_over_ranks(torch, dist, world, time.perf_counter() - w0)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    # the reduction kernel reads the points and reads and writes each touched
    # entry of L (16 bytes per valid column)
    s_avg = sum(cols) / len(cols)
    kernel_bytes = 8 * n + 16 * s_avg
    achieved = kernel_bytes / (red_avg / 1e3) / 1e9
    cpu_v, cpu_dt, cpu_passes = _cpu_rate(oracle_solver("sparse"), [(p, P) for _, P in inputs],
                                          args.cpu_budget)
    line = {
        "metric": METRIC, "value": rate["sparse"], "unit": "Gpoints/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms["sparse"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "config": workload_config("sparse"),
        "sparse": {"plain_gpoints_s": rate["plain"], "speedup_vs_plain": rate["sparse"] / rate["plain"],
                   "ms_per_step": {a: t / args.steps for a, t in ms.items()},
                   "valid_columns": cols, "hulls_identical": same,
                   "l2_flush_ms_subtracted": fl / args.steps, "density_sweep": sweep},
        "roofline": {"bound": "hbm", "kernel": "k_sparse_reduce", "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "algorithmic_bytes_per_launch": kernel_bytes, "avg_launch_ms": red_avg,
                     "ms_per_step_while_timed": ms_traced / args.steps, "traffic": None,
                     "note": "scattered atomics on L and the tree, not a streaming pass"},
        "e2e": {"value": world * pts_step * e2e_steps / e2e_s / 1e9, "unit": "Gpoints/s",
                "h2d_bytes_per_step": pts_step * 8, "d2h_bytes_per_step": d2h // e2e_steps,
                "steps": e2e_steps},
        "cpu_baseline": {"value": cpu_v, "unit": "Gpoints/s", "cores": 1, "kind": "oracle",
                         "sample": f"{cpu_passes} pass(es) over the step's instances "
                                   f"({cpu_dt:.1f} s, single thread: chains from the points "
                                   f"+ hull)"},
        "gpu_launches": args.steps * len(inputs) * ch.ch_sparse_kernel_count(n, p),
        "clocks": clocks,
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
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["learned", "batched", "box",
                                                                "melkman", "rxy", "sparse",
                                                                "profile_batched"],
                    default="plain_at_scale")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--regions", type=int, default=5,
                    help="timed regions of --steps steps each, back to back; the median is reported")
    ap.add_argument("--no-aux", action="store_true",
                    help="skip the side measurements (density sweep, Melkman on the full "
                         "polyline): for profiling runs")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload in ("batched", "profile_batched"):
        run_batched(args)
    elif args.workload == "box":
        run_box(args)
    elif args.workload in ("melkman", "rxy"):
        run_alt(args)
    elif args.workload == "sparse":
        run_sparse(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
