#!/usr/bin/env python
"""Benchmark of the GB300 near-field P2P operator: pair-interactions per second.

Workload (default): the occupancy sweep on the unit sphere -- N = 2^20 points
uniform on the sphere surface, leaf grids of 180^3 / 124^3 / 86^3 / 61^3 boxes
(mean 8 / 16 / 32 / 64 points per non-empty box), leaf edge a quarter
wavelength, Helmholtz kernel, complex64 strengths ~ N(0, 1), one right-hand
side, FP32 arithmetic.  One step applies the operator once at each of the four
occupancies (strength staging + pair kernel + scatter); the plans (binning,
neighbour lists, packed layout) are built once per geometry before timing.

value = pairs of the step / step time, pairs = ordered (target, source) pairs
with r > 0 in every 27-box neighbourhood.  L2 is flushed (256 MiB write)
between timed steps, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--layout auto|indexed|redundant]

After the timed steps (outside them) the default run adds two sub-records to
its line: `redundant` -- the same sweep through the redundant layout of Sec.
3.3 (per-occupancy repack and pair-kernel times, the pair kernel against the
MUFU roofline, and the apply against its binding term, HBM or MUFU) -- and
`multirhs` -- the 2:1:1 ellipsoid (2^21 points, 64 right-hand sides): the
tensor-core path against the per-RHS and shared-G FP32 paths, rel-L2 per RHS
against the FP64 oracle on sampled targets, and the tensor-core kernel's
roofline fraction.  --no-extras skips them.

--impl reference times the FP64 CPU oracle, as it stands, on a bounded sample
of targets of the same workload (no GPU use).  Under torchrun each rank runs
an independent replica (the operator has no exchange step on one GPU per
box set); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "P2P pair-interactions/s (G/s) + roofline fraction at stated L2 err vs FP64"
UNIT = "Gpair/s"
OCCUPANCIES = (8, 16, 32, 64)
MUFU_PER_PAIR = {"helmholtz": 3, "laplace": 1}  # rsqrt, sin, cos per Helmholtz pair
MUFU_LANES_PER_SM_CLK = 16
L2_FLUSH_BYTES = 256 << 20
REFERENCE_BUDGET_S = 120.0  # oracle work of one --impl reference run (warm-up + timed steps)


def _peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
            "source": "fallback"}


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# --------------------------------------------------------------- clocks ----

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 100 ms."""

    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id.lower() if bus_id else None
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        rows = self.rows
        if self.bus_id:
            mine = [r for r in rows if len(r) > 1 and self.bus_id.endswith(r[1].lower()[-12:])]
            rows = mine or rows
        sm = [float(r[2]) for r in rows if len(r) >= 10 and r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if len(r) >= 10 and r[3].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows if len(r) >= 10 for i in range(4) if r[6 + i] == "Active"})
        power = [float(r[4]) for r in rows if len(r) >= 10 and r[4].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(sm), "power_w_max": max(power) if power else None}


# --------------------------------------------------------------- workload --

def sweep_workloads():
    from paper_2403_01596_gb300 import workloads as W
    return [W.sphere_density(d) for d in OCCUPANCIES]


def _sample_targets(n, count, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=min(count, n), replace=False))


def _sample_pairs(struct_host, points, targets) -> int:
    """Exact pair count of the sampled targets from the box structure (r > 0 pairs)."""
    box_ptr, nbr_ptr, nbr_idx, point_box, perm = struct_host
    sizes = np.diff(box_ptr)
    total = 0
    for i in targets:
        b = point_box[i]
        s = int(sizes[nbr_idx[nbr_ptr[b]:nbr_ptr[b + 1]]].sum())
        own = perm[box_ptr[b]:box_ptr[b + 1]]
        dup = int(np.all(points[own] == points[i], axis=1).sum())
        total += s - dup
    return total


def _oracle_call_time(oracle, wl, lam, m, seed):
    targets = _sample_targets(wl.n, m, seed)
    t = time.perf_counter()
    oracle.p2p_targets(wl.points, lam, targets, wl.lo, wl.h, wl.ng, wl.k)
    return time.perf_counter() - t


def _oracle_worker(occupancies, jobs, done, barrier):
    """One host core of the all-cores oracle timing: rebuilds the seeded sweep workloads itself (no point data
    crosses a pipe), then per request runs the unchanged oracle on its share of the sampled targets, started
    together with the other workers by a barrier."""
    import oracle
    from paper_2403_01596_gb300 import workloads as W
    oracle.build()
    wls = [W.sphere_density(d) for d in occupancies]
    lams = [W.strengths(wl.n, 1, wl.seed) for wl in wls]
    oracle.p2p_targets(wls[0].points, lams[0], np.arange(4), wls[0].lo, wls[0].h, wls[0].ng, wls[0].k)
    done.put("ready")
    while True:
        job = jobs.get()
        if job is None:
            return
        i, targets = job
        barrier.wait(timeout=900)
        wl = wls[i]
        oracle.p2p_targets(wl.points, lams[i], targets, wl.lo, wl.h, wl.ng, wl.k)
        done.put(len(targets))


class OraclePool:
    """The FP64 oracle, as it stands (single-threaded C), run as one spawned process per host core on disjoint
    target shares of the occupancy sweep; run() returns the wall time from the common start to the last finish."""

    def __init__(self, workers: int | None = None):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")  # the parent may hold a CUDA context: no fork
        self.workers = max(1, workers or os.cpu_count() or 1)
        self.done = ctx.Queue()
        self.barrier = ctx.Barrier(self.workers + 1)
        self.jobs = [ctx.Queue() for _ in range(self.workers)]
        self.procs = [ctx.Process(target=_oracle_worker, args=(OCCUPANCIES, q, self.done, self.barrier),
                                  daemon=True) for q in self.jobs]
        for pr in self.procs:
            pr.start()
        self._collect()

    def _collect(self):
        """One message from every worker; raises as soon as a worker has died."""
        import queue
        got = 0
        while got < self.workers:
            try:
                self.done.get(timeout=1.0)
                got += 1
            except queue.Empty:
                dead = [pr.exitcode for pr in self.procs if not pr.is_alive()]
                if dead:
                    self.close()
                    raise RuntimeError(f"oracle worker exited with {dead[0]}")

    def run(self, i: int, targets) -> float:
        for q, share in zip(self.jobs, np.array_split(np.asarray(targets), self.workers)):
            q.put((i, share))
        self.barrier.wait(timeout=900)
        t = time.perf_counter()
        self._collect()
        return time.perf_counter() - t

    def close(self):
        for q in self.jobs:
            q.put(None)
        for pr in self.procs:
            pr.join(timeout=60)
            if pr.is_alive():
                pr.terminate()


def _sample_pairs_fast(struct_host, points, targets) -> int:
    """_sample_pairs without the per-target loop when the point set has no repeated coordinates (every target's
    only r = 0 pair is with itself)."""
    box_ptr, nbr_ptr, nbr_idx, point_box, perm = struct_host
    if np.unique(points, axis=0).shape[0] != points.shape[0]:
        return _sample_pairs(struct_host, points, targets)
    sizes = np.diff(box_ptr).astype(np.int64)
    per_box = np.add.reduceat(sizes[nbr_idx], nbr_ptr[:-1]) if len(nbr_idx) else np.zeros(len(sizes), np.int64)
    return int((per_box[point_box[targets]] - 1).sum())


def cpu_oracle_all_cores(wls, structs, calib, seconds_per_density: float, seed: int):
    """The oracle on every host core (OraclePool), each core given about seconds_per_density of work per
    occupancy (calib = the single-thread (fixed, per-target) cost of one oracle call)."""
    pool = OraclePool()
    try:
        pairs, seconds = 0, 0.0
        for i, (wl, st) in enumerate(zip(wls, structs)):
            fixed, per_target = calib[i]
            m = int(min(wl.n // pool.workers, max(512, (seconds_per_density - fixed) / per_target)))
            targets = _sample_targets(wl.n, m * pool.workers, seed + 7 + i)
            seconds += pool.run(i, targets)
            pairs += _sample_pairs_fast(st, wl.points, targets)
    finally:
        pool.close()
    return {"pairs": pairs, "seconds": seconds, "workers": pool.workers}


def cpu_oracle_sample(wls, structs, seconds_per_density: float, seed: int):
    """Times the FP64 oracle (as it stands, single thread) on sampled targets."""
    import oracle
    from paper_2403_01596_gb300 import workloads as W
    oracle.build()
    res = []
    for wl, st in zip(wls, structs):
        lam = W.strengths(wl.n, 1, wl.seed)
        # calibrate: t(m) = fixed (the oracle's own binning) + m * per_target
        t_small, t_big = _oracle_call_time(oracle, wl, lam, 256, seed), _oracle_call_time(oracle, wl, lam, 4096, seed)
        per_target = max((t_big - t_small) / (4096 - 256), 1e-7)
        fixed = max(t_small - 256 * per_target, 0.0)
        m = int(min(wl.n, max(512, (seconds_per_density - fixed) / per_target)))
        targets = _sample_targets(wl.n, m, seed + 1)
        t = time.perf_counter()
        ref = oracle.p2p_targets(wl.points, lam, targets, wl.lo, wl.h, wl.ng, wl.k)
        dt = time.perf_counter() - t
        pairs = _sample_pairs(st, wl.points, targets)
        # sum of the terms' magnitudes per target: |exp(ikr)| = 1, so the Laplace sum of |lambda| (not timed)
        abs_sum = oracle.p2p_targets(wl.points, np.abs(lam).astype(np.float64), targets, wl.lo, wl.h, wl.ng, 0.0,
                                     kernel=oracle.LAPLACE).real
        res.append({"occupancy": wl.meta["target_occupancy"], "targets": targets, "ref": ref, "seconds": dt,
                    "pairs": pairs, "calib": (fixed, per_target), "abs_sum": abs_sum})
    return res


def host_structure(plan):
    s = plan.structure
    n = s.n
    return (s.box_ptr.cpu().numpy(), s.nbr_ptr.cpu().numpy(), s.nbr_idx.cpu().numpy()[:s.nnz],
            s.point_box.cpu().numpy()[:n], s.perm.cpu().numpy()[:n])


def _oracle_structure(wl):
    import oracle
    b = oracle.bin_points(wl.points, wl.lo, wl.h, wl.ng)
    nptr, nidx = oracle.neighbors(b["box_keys"], wl.ng)
    return (b["box_ptr"], nptr, nidx, b["point_box"], b["perm"])


# ------------------------------------------------------------ reference --

def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    from paper_2403_01596_gb300 import workloads as W
    import oracle
    oracle.build()
    wls = sweep_workloads()
    structs = [_oracle_structure(wl) for wl in wls]
    lams = [W.strengths(wl.n, 1, wl.seed) for wl in wls]
    # size the samples so the whole run (warm-up + timed steps) takes about REFERENCE_BUDGET_S of oracle work;
    # one oracle call costs t(m) = fixed + m * per_target for m sampled targets
    steps_total = args.warmup + args.steps
    step_budget = REFERENCE_BUDGET_S / max(steps_total, 1)
    fixed, per_target = [], []
    for i, wl in enumerate(wls):
        t_small = _oracle_call_time(oracle, wl, lams[i], 256, 7)
        t_big = _oracle_call_time(oracle, wl, lams[i], 4096, 7)
        per_target.append(max((t_big - t_small) / (4096 - 256), 1e-7))
        fixed.append(max(t_small - 256 * per_target[-1], 0.0))
    # every occupancy in every step while that fits the step's budget, else one occupancy per step in turn
    rotate = step_budget < sum(fixed) + 4 * 256 * max(per_target)
    share = step_budget if rotate else step_budget / len(wls)
    # every host core runs the oracle on its own share of each step's targets (OraclePool), each core about the
    # single-thread budget's worth
    pool = OraclePool()
    workers = pool.workers
    samples = [int(min(wl.n // workers, max(256, (share - fixed[i]) / per_target[i]))) * workers
               for i, wl in enumerate(wls)]
    times, pairs = [], []
    try:
        for step in range(steps_total):
            dt, p = 0.0, 0
            for i, wl in enumerate(wls):
                if rotate and i != step % len(wls):
                    continue
                targets = _sample_targets(wl.n, samples[i], 1000 + step)
                dt += pool.run(i, targets)
                p += _sample_pairs_fast(structs[i], wl.points, targets) if step >= args.warmup else 0
            if step >= args.warmup:
                times.append(dt)
                pairs.append(p)
    finally:
        pool.close()
    value = sum(pairs) / sum(times) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args, "oracle"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": f"{samples} sampled targets at occupancy 8/16/32/64, "
                                   + ("one occupancy per step in turn" if rotate else "all four per step")
                                   + f"; FP64 oracle as one process per core ({workers}) on disjoint shares, wall "
                                     "time; each call includes the oracle's own binning of all 2^20 points"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _config(args, layout):
    return {"workload": "sphere_occupancy_sweep", "n_points": 1 << 20, "occupancies": list(OCCUPANCIES),
            "grids": [180, 124, 86, 61], "kernel": "helmholtz", "k": "2*pi/(4h)", "nrhs": 1, "layout": layout,
            "tuning": {"chunk": getattr(args, "chunk", 0), "warps_per_cta": getattr(args, "warps", 0),
                       "target_group": getattr(args, "target_group", 0), "warp_boxes": getattr(args, "warp_boxes", 0),
                       "note": "0 = chosen by each plan; the launch tuning used is in roofline.per_occupancy"},
            "l2": "flushed between timed steps (256 MiB write, outside the timed events)"}


# ------------------------------------------------------------------- ours --

def _traffic_for(kernel_src_hash: str, layout: str):
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except ValueError:
        return None
    e = d.get(layout)
    if not e or e.get("source_sha256") != kernel_src_hash:
        return None
    return e.get("dram_bytes_per_launch")


def _kernel_name(warp_boxes: int) -> str:
    """The one-RHS pair kernel a plan runs, from its tuning's warp_boxes."""
    if warp_boxes == -2:
        return "k_pair_group (box groups)"
    if warp_boxes > 0:
        return f"k_pair_direct ({warp_boxes} boxes per warp)"
    return "k_pair (staged pipeline)"


def _kernel_hash() -> str:
    """Hash of the pair kernels' sources with comments and blank lines removed (a comment edit keeps the DRAM
    traffic record valid; any code change drops it)."""
    import re
    h = hashlib.sha256()
    for f in ("p2p_apply.cu", "p2p_pair.cuh", "p2p_direct.cuh", "p2p_group.cu", "p2p_internal.cuh", "p2p_plan.cu"):
        src = open(os.path.join(ROOT, "paper_2403_01596_gb300", "csrc", f), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("\n".join(line.rstrip() for line in src.splitlines() if line.strip()).encode())
    return h.hexdigest()


def run_ours(args):
    import torch
    from paper_2403_01596_gb300 import _capi as C
    from paper_2403_01596_gb300 import api, workloads as W

    from paper_2403_01596_gb300 import replicas
    rank, local, world = replicas.world()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    peaks = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count

    wls = sweep_workloads()
    pts = torch.from_numpy(wls[0].points).to(dev)
    plans, lams, outs, pairs = [], [], [], []
    layouts = []
    t_plan = []
    for wl in wls:
        layout = args.layout
        if layout == "auto":
            from paper_2403_01596_gb300 import autotune
            tune = autotune.best_config(wl, pts)
            layout, tuning = tune["layout"], tune["tuning"]
        else:
            tuning = {k: v for k, v in (("chunk", args.chunk), ("warps_per_cta", args.warps),
                                        ("target_group", args.target_group), ("warp_boxes", args.warp_boxes))
                      if v} or None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = api.Plan(pts, wl.lo, wl.h, wl.ng, wl.k, layout=layout, tuning=tuning)
        torch.cuda.synchronize()
        t_plan.append(time.perf_counter() - t0)
        plans.append(plan)
        layouts.append(layout)
        lam = torch.from_numpy(W.strengths(wl.n, 1, wl.seed)).to(dev)
        lams.append(lam)
        outs.append(torch.empty_like(lam))
        pairs.append(plan.pair_count())
    step_pairs = sum(pairs)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    path = C.P2P_PATH_FP32_SHARED

    def one_apply(i, evs=None):
        p = plans[i]
        if evs and i == 0:
            evs[0].record(stream)  # later occupancies start at the previous one's end event
        C.p2p_apply_stage(p._plan, lams[i], 1, 1, path, stream)
        if evs:
            evs[1].record(stream)
        C.p2p_apply_staged(p._plan, outs[i], 1, 1, 0, path, stream)
        if evs:
            evs[2].record(stream)

    for _ in range(args.warmup):
        for i in range(len(plans)):
            one_apply(i)
    torch.cuda.synchronize()
    nd = len(plans)
    evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(nd)] for _ in range(args.steps)]
    bus = None
    try:
        bus = "%04x:%02x:%02x" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except AttributeError:
        bus = None
    clocks = ClockSampler(bus)
    clocks.start()
    time.sleep(0.3)
    replicas.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.zero_()
        for i in range(nd):
            one_apply(i, evs[s][i])
        for i in range(1, nd):
            evs[s][i][0] = evs[s][i - 1][2]
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    replicas.barrier()
    clk = clocks.stop()
    step_ms = [evs[s][0][0].elapsed_time(evs[s][nd - 1][2]) for s in range(args.steps)]
    pair_ms = [[evs[s][i][1].elapsed_time(evs[s][i][2]) for s in range(args.steps)] for i in range(nd)]
    stage_ms = [[evs[s][i][0].elapsed_time(evs[s][i][1]) for s in range(args.steps)] for i in range(nd)]
    total_ms = replicas.max_over_ranks(sum(step_ms), device=dev)
    ms_per_step = total_ms / args.steps
    value = replicas.job_throughput(step_pairs, world, ms_per_step * 1e-3) / 1e9

    # ---------------- end to end through the public API with host buffers
    # (api.HostPipe = p2p_apply_host: page-locked host strengths in, host results out; the upload of the next
    # occupancy and the download of the previous one overlap each occupancy's kernels)
    host_lam = [lam.cpu().pin_memory() for lam in lams]
    host_out = [torch.empty_like(h).pin_memory() for h in host_lam]
    pipe = api.HostPipe(max(p.n for p in plans), 1)
    e2e_ms = []
    for s in range(args.warmup + args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pipe.apply(plans, host_lam, host_out)
        e1.record(stream)
        torch.cuda.synchronize()
        if s >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_check = max(float(np.abs(host_out[i].numpy() - outs[i].cpu().numpy().reshape(-1)).max()
                          / max(float(np.abs(outs[i].cpu().numpy()).max()), 1e-30)) for i in range(nd))
    pipe.close()
    e2e_bytes = sum(h.numel() * 8 for h in host_lam)
    e2e_value = world * step_pairs / (statistics.mean(e2e_ms) * 1e-3) / 1e9

    # ---------------- roofline of the dominant kernel (the pair kernel)
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak_pairs = sms * MUFU_LANES_PER_SM_CLK * f_max / MUFU_PER_PAIR["helmholtz"] / 1e9
    pair_total_ms = sum(statistics.mean(pm) for pm in pair_ms)
    achieved = step_pairs / (pair_total_ms * 1e-3) / 1e9
    detail = []
    for i, wl in enumerate(wls):
        pm, sm = statistics.mean(pair_ms[i]), statistics.mean(stage_ms[i])
        detail.append({"occupancy": wl.meta["target_occupancy"], "layout": layouts[i], "boxes": plans[i].num_boxes,
                       "pairs": pairs[i], "pair_kernel_ms": pm, "stage_ms": sm,
                       "gpair_s": pairs[i] / (pm + sm) / 1e6, "pair_kernel_frac_of_mufu": pairs[i] / pm / 1e6 / peak_pairs,
                       "plan_s": t_plan[i], "work_items": plans[i].info["work_items"],
                       "tuning": plans[i].info["tuning"]})
    khash = _kernel_hash()
    traffic = _traffic_for(khash, layouts[0]) if len(set(layouts)) == 1 else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_pairs, "unit": "Gpair/s",
                "frac": achieved / peak_pairs, "traffic": traffic,
                "kernel": "the FP32 pair kernels the plans choose: " + ", ".join(
                    f"D = {d['occupancy']}: " + _kernel_name(d["tuning"].get("warp_boxes", -1)) for d in detail),
                "peak_basis": f"MUFU: {sms} SMs x 16 lanes/clk x {f_max / 1e6:.0f} MHz / 3 MUFU per Helmholtz pair "
                              f"(sm_max_mhz {peaks['source']})",
                "peak_at_measured_clock": (sms * 16 * clk["sm_mhz"] * 1e6 / 3 / 1e9) if clk.get("sm_mhz") else None,
                "per_occupancy": detail}

    # ---------------- the two layout / precision comparisons, as sub-records (rank 0, N = 1)
    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras["redundant"] = measure_redundant(wls, pts, [p.structure for p in plans], pairs, args.extra_steps,
                                                flush, peaks, sms)
        extras["multirhs"] = measure_multirhs(1.0, args.extra_steps, args.samples)

    # ---------------- CPU oracle baseline and sampled accuracy (rank 0, N = 1)
    cpu = None
    err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        structs = [host_structure(p) for p in plans]
        res = cpu_oracle_sample(wls, structs, args.cpu_seconds / len(wls), 17)
        cpu_pairs = sum(r["pairs"] for r in res)
        cpu_s = sum(r["seconds"] for r in res)
        single = cpu_pairs / cpu_s / 1e9
        allc = cpu_oracle_all_cores(wls, structs, [r["calib"] for r in res], args.cpu_seconds / len(wls), 17)
        cpu = {"value": allc["pairs"] / allc["seconds"] / 1e9, "unit": UNIT, "cores": allc["workers"],
               "kind": "oracle",
               "sample": f"FP64 oracle as one process per core ({allc['workers']}) on disjoint sampled targets, "
                         f"{allc['pairs']} pairs in {allc['seconds']:.1f} s wall; each call includes the oracle's own "
                         "binning of all 2^20 points",
               "single_thread": {"value": single, "cores": 1,
                                 "sample": "FP64 oracle on " + ", ".join(
                                     f"{len(r['targets'])} targets at occupancy {r['occupancy']}" for r in res)
                                           + f" ({cpu_pairs} pairs, {cpu_s:.1f} s)"}}
        errs, relmax, normwise = [], [], []
        for r, out in zip(res, outs):
            got = out.cpu().numpy()[r["targets"]]
            errs.append(float(np.linalg.norm(got - r["ref"]) / np.linalg.norm(r["ref"])))
            d = np.abs(got - r["ref"])
            relmax.append(float((d / np.abs(r["ref"])).max()))
            normwise.append(float((d / r["abs_sum"]).max()))
        err = {"rel_l2_max": max(errs), "per_occupancy": errs,
               "max_per_target_rel": relmax,
               "max_per_target_err_over_abs_sum": normwise,
               "sample": "targets of the cpu_baseline sample; abs_sum = sum_j |G(r_ij) lambda_j| (oracle)",
               "tolerance": 1e-5}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(args, layouts[0] if len(set(layouts)) == 1 else "per-occupancy:" + ",".join(layouts)),
            "pairs_per_step": step_pairs * world, "rel_l2_vs_fp64": err,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": e2e_bytes, "d2h_bytes_per_step": e2e_bytes,
                    "api": "p2p_apply_host (api.HostPipe), page-locked host buffers",
                    "max_rel_diff_vs_device_apply": e2e_check},
            "gpu_launches": 2 * nd * args.steps,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clk, **extras,
            "wall_s_timed_region": wall, "device": props.name, "sms": sms,
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------- extension workloads --
# Non-default modes (python bench.py --workload cube|multirhs|grad|batched): the
# dense cube, the 64-RHS tensor-core comparison on the 2:1:1 ellipsoid, the
# differentiable step on the sphere, and the batched uneven geometries.  Each
# prints one JSON line of the same shape as the default occupancy sweep.

def _events_time(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms), ms


def _oracle_sampled(wl, lam_np, targets, adjoint=False):
    import oracle
    oracle.build()
    t = time.perf_counter()
    ref = oracle.p2p_targets(wl.points, lam_np, targets, wl.lo, wl.h, wl.ng, wl.k, adjoint=adjoint)
    return ref, time.perf_counter() - t


def _rel_l2_cols(x, ref):
    x = np.asarray(x).reshape(ref.shape[0], -1)
    ref = np.asarray(ref).reshape(ref.shape[0], -1)
    return np.linalg.norm(x - ref, axis=0) / np.linalg.norm(ref, axis=0)


def measure_multirhs(scale, steps, samples, free_first=()):
    """The 64-RHS comparison on the 2:1:1 ellipsoid (2^21 points, 188^3 grid, leaf edge 0.2 wavelength):
    the tensor-core paths (BF16 hi/lo split with 3 MMAs, hi/mid/lo with 6; tcgen05, FP32 accumulation)
    against the FP32 path with G shared over RHS blocks and the plain per-RHS FP32 path, each timed with CUDA
    events; rel-L2 vs the FP64 oracle per right-hand side and the largest |err| / sum_j |G lambda_j| on
    `samples` sampled targets.  Returns the record (timings, errors, roofline)."""
    import torch
    from paper_2403_01596_gb300 import _capi as C
    from paper_2403_01596_gb300 import api, workloads as W
    peaks = _peaks()
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    wl = W.ellipsoid_multirhs(int((1 << 21) * scale))
    nrhs = 64
    pts = torch.from_numpy(wl.points).cuda()
    plan = api.Plan(pts, wl.lo, wl.h, wl.ng, wl.k, max_nrhs=nrhs)
    lam_np = W.strengths(wl.n, nrhs, wl.seed)
    lam = torch.from_numpy(lam_np).cuda()
    out = torch.empty_like(lam)
    P = plan.pair_count()
    stream = torch.cuda.current_stream()
    res = {}
    for path, n_steps in (("tc_bf16x3", steps), ("tc_bf16x6", max(2, steps // 2)),
                          ("fp32_shared", max(2, steps // 4)), ("fp32_per_rhs", max(2, steps // 8))):
        med, _ = _events_time(lambda: plan.apply(lam, out=out, path=path), n_steps, 2, stream)
        res[path] = {"ms": med, "gpair_rhs_s": P * nrhs / med / 1e6, "steps": n_steps, "out": out.cpu().numpy()}
    # tensor-core path in two phases: strength pre-pack (k_tc_pack), then the pipelined kernel (k_p2p_tc)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for i in range(2 + steps):
        e = evs[i - 2] if i >= 2 else None
        if e:
            e[0].record(stream)
        C.p2p_apply_stage(plan._plan, lam, nrhs, nrhs, C.P2P_PATH_TC_BF16X3, stream)
        if e:
            e[1].record(stream)
        C.p2p_apply_staged(plan._plan, out, nrhs, nrhs, 0, C.P2P_PATH_TC_BF16X3, stream)
        if e:
            e[2].record(stream)
    torch.cuda.synchronize()
    status = plan.async_status()
    pack_ms = statistics.median(e[0].elapsed_time(e[1]) for e in evs)
    kern_ms = statistics.median(e[1].elapsed_time(e[2]) for e in evs)
    targets = _sample_targets(wl.n, samples, 5)
    ref, cpu_s = _oracle_sampled(wl, lam_np, targets)
    import oracle
    abs_sum = oracle.p2p_targets(wl.points, np.abs(lam_np).astype(np.float64), targets, wl.lo, wl.h, wl.ng, 0.0,
                                 kernel=oracle.LAPLACE).real
    for path in res:
        got = res[path].pop("out")[targets]
        e = _rel_l2_cols(got, ref)
        res[path]["max_per_target_err_over_abs_sum"] = float((np.abs(got - ref) / abs_sum).max())
        res[path]["rel_l2_max"] = float(e.max())
        res[path]["rel_l2_per_rhs_mean"] = float(e.mean())
        res[path]["rel_l2_per_rhs"] = [float(v) for v in e]
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    mufu_peak = props.multi_processor_count * 16 * f_max / 3 / 1e9        # G evaluations per second (G/s)
    tc_flops = 3 * 8 * P * nrhs                                           # hi.hi + hi.lo + lo.hi, realified complex
    t_tc = kern_ms * 1e-3                                                 # the pipelined kernel alone
    sizes = torch.diff(plan.structure.box_ptr.long())
    groups = int(((sizes + 15) // 16).sum().item())                      # 16-source groups of the pre-pack
    record = ((nrhs + 63) // 64) * (8192 + 16 * 16)                      # per 64-RHS chunk: hi/lo images + coordinates
    pack_bytes = wl.n * (nrhs * 8 + 16) + groups * record                 # strengths, coordinates read; records written
    rec = {"workload": "ellipsoid211_multirhs", "n_points": wl.n, "grid": wl.ng, "nrhs": nrhs, "pairs": P,
           "boxes": plan.num_boxes, "paths": res, "async_status": status,
           "speedup_tc_vs_fp32_per_rhs": res["fp32_per_rhs"]["ms"] / res["tc_bf16x3"]["ms"],
           "speedup_tc_vs_fp32_shared": res["fp32_shared"]["ms"] / res["tc_bf16x3"]["ms"],
           "speedup_tc6_vs_fp32_shared": res["fp32_shared"]["ms"] / res["tc_bf16x6"]["ms"],
           "tolerance": 1e-5,
           "roofline": {"bound": "alu", "kernel": "k_p2p_tc", "achieved": P / t_tc / 1e9, "peak": mufu_peak,
                        "unit": "G pair-evaluations/s", "frac": P / t_tc / 1e9 / mufu_peak,
                        "kernel_ms": kern_ms,
                        "tensor_tflops": tc_flops / t_tc / 1e12,
                        "tensor_frac_of_bf16_peak": tc_flops / t_tc / 1e12 / float(peaks["bf16_tflops"]),
                        "pack": {"kernel": "k_tc_pack", "ms": pack_ms, "bytes": pack_bytes,
                                 "gbs": pack_bytes / (pack_ms * 1e-3) / 1e9,
                                 "frac_of_hbm": pack_bytes / (pack_ms * 1e-3) / 1e9 / float(peaks["hbm_gbs"])}},
           "oracle_sample": {"targets": len(targets), "seconds": cpu_s}}
    del plan, lam, out, pts
    torch.cuda.empty_cache()
    return rec


def measure_redundant(wls, pts, structures, pairs, steps, flush, peaks, sms):
    """The redundant layout (Sec. 3.3: per-box copies of each neighbourhood's coordinates, strengths repacked
    every apply) on the occupancy sweep: per occupancy the repack and pair-kernel times (CUDA events, L2
    flushed before each apply), the apply rate, the pair kernel against R_MUFU, and the binding term of the
    whole apply: max(P / R_MUFU, bytes / HBM) with bytes = packed (16 + 8) + n (8 + 8) for the pair kernel and
    packed (4 + 8 + 8) for the repack."""
    import torch
    from paper_2403_01596_gb300 import _capi as C
    from paper_2403_01596_gb300 import api, workloads as W
    stream = torch.cuda.current_stream()
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    r_mufu = sms * MUFU_LANES_PER_SM_CLK * f_max / MUFU_PER_PAIR["helmholtz"]
    hbm = float(peaks["hbm_gbs"]) * 1e9
    path = C.P2P_PATH_FP32_SHARED
    rows = []
    for wl, st, P in zip(wls, structures, pairs):
        plan = api.Plan(pts, wl.lo, wl.h, wl.ng, wl.k, layout="redundant", structure=st)
        lam = torch.from_numpy(W.strengths(wl.n, 1, wl.seed)).to(pts.device)
        out = torch.empty_like(lam)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        for i in range(3 + steps):
            flush.zero_()
            e = evs[i - 3] if i >= 3 else None
            if e:
                e[0].record(stream)
            C.p2p_apply_stage(plan._plan, lam, 1, 1, path, stream)
            if e:
                e[1].record(stream)
            C.p2p_apply_staged(plan._plan, out, 1, 1, 0, path, stream)
            if e:
                e[2].record(stream)
        torch.cuda.synchronize()
        stage_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
        pair_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
        packed = int(st.sources)  # sum over boxes of the sources in each neighbourhood (the per-box copies)
        kbytes = packed * (16 + 8) + wl.n * (8 + 8)
        rbytes = packed * (4 + 8 + 8)
        t_mufu, t_hbm = P / r_mufu, (kbytes + rbytes) / hbm
        t_apply = (stage_ms + pair_ms) * 1e-3
        rows.append({"occupancy": wl.meta["target_occupancy"], "pairs": P, "packed": packed,
                     "repack_ms": stage_ms, "pair_kernel_ms": pair_ms, "apply_gpair_s": P / t_apply / 1e9,
                     "pair_kernel_frac_of_mufu": P / (pair_ms * 1e-3) / r_mufu,
                     "binding": "hbm" if t_hbm > t_mufu else "mufu",
                     "binding_us": 1e6 * max(t_mufu, t_hbm), "mufu_us": 1e6 * t_mufu, "hbm_us": 1e6 * t_hbm,
                     "apply_frac_of_binding": max(t_mufu, t_hbm) / t_apply,
                     "async_status": plan.async_status(), "tuning": plan.info["tuning"]})
        del plan
    tot_p = sum(r["pairs"] for r in rows)
    tot_ms = sum(r["repack_ms"] + r["pair_kernel_ms"] for r in rows)
    tot_k = sum(r["pair_kernel_ms"] for r in rows)
    return {"layout": "redundant", "steps": steps, "apply_gpair_s": tot_p / tot_ms / 1e6,
            "pair_kernel_frac_of_mufu": tot_p / (tot_k * 1e-3) / r_mufu, "per_occupancy": rows,
            "l2": "flushed before every apply"}


def run_multirhs(args):
    import torch
    torch.cuda.set_device(0)
    rec = measure_multirhs(args.scale, args.ext_steps, args.samples)
    res = rec["paths"]
    line = {"metric": METRIC + " [64-RHS: pair x RHS]", "value": res["tc_bf16x3"]["gpair_rhs_s"], "unit": UNIT,
            "n_gpus": 1, "steps": args.ext_steps, "warmup": 2, "ms_per_step": res["tc_bf16x3"]["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3/f32",
            "data": "synthetic",
            "config": {k: rec[k] for k in ("workload", "n_points", "grid", "nrhs", "pairs", "boxes")},
            "paths": res,
            "speedup_tc_vs_fp32_per_rhs": rec["speedup_tc_vs_fp32_per_rhs"],
            "speedup_tc_vs_fp32_shared": rec["speedup_tc_vs_fp32_shared"],
            "roofline": rec["roofline"],
            "cpu_baseline": {"value": rec["oracle_sample"]["targets"] * rec["nrhs"] * (rec["pairs"] / rec["n_points"])
                             / rec["oracle_sample"]["seconds"] / 1e9, "unit": UNIT, "cores": 1,
                             "kind": "oracle", "sample": f"{rec['oracle_sample']['targets']} targets x {rec['nrhs']} "
                                                         "RHS (pairs estimated from the mean neighbourhood), "
                                                         f"{rec['oracle_sample']['seconds']:.1f} s"}}
    print(json.dumps(line))
    return 0


def run_grad(args):
    import torch
    from paper_2403_01596_gb300 import api, workloads as W
    torch.cuda.set_device(0)
    wl = W.sphere_grad(int((1 << 18) * args.scale))
    pts = torch.from_numpy(wl.points).cuda().requires_grad_(True)
    plan = api.Plan(pts.detach(), wl.lo, wl.h, wl.ng, wl.k)
    lam = torch.from_numpy(W.strengths(wl.n, 1, wl.seed)).cuda().requires_grad_(True)
    b = torch.from_numpy(W.strengths(wl.n, 1, 4)).cuda()
    P = plan.pair_count()
    stream = torch.cuda.current_stream()

    def step():
        lam.grad = None
        pts.grad = None
        out = api.p2p(lam, pts, plan)
        loss = (out - b).abs().pow(2).sum()
        loss.backward()

    med, _ = _events_time(step, args.ext_steps, 3, stream)
    import oracle
    oracle.build()
    g = 2 * (plan.apply(lam.detach()) - b)
    t = time.perf_counter()
    ref_x = oracle.grad_points(wl.points, lam.detach().cpu().numpy(), g.cpu().numpy(), wl.lo, wl.h, wl.ng, wl.k)
    cpu_s = time.perf_counter() - t
    step()
    torch.cuda.synchronize()
    err_x = float(np.linalg.norm(pts.grad.cpu().numpy() - ref_x) / np.linalg.norm(ref_x))
    line = {"metric": METRIC + " [forward + adjoint + coordinate gradient: 3 sweeps per step]",
            "value": 3 * P / med / 1e6, "unit": UNIT, "n_gpus": 1, "steps": args.ext_steps, "warmup": 3,
            "ms_per_step": med, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "sphere_grad", "n_points": wl.n, "grid": wl.ng, "k": wl.k, "pairs": P,
                       "loss": "||A(x) lam - b||^2"},
            "grad_x_rel_l2_vs_fp64": err_x,
            "cpu_baseline": {"value": P / cpu_s / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"full FP64 coordinate gradient ({P} pairs, {cpu_s:.1f} s)"}}
    print(json.dumps(line))
    return 0


def run_batched(args):
    import torch
    from paper_2403_01596_gb300 import api, workloads as W
    torch.cuda.set_device(0)
    nrhs = 8
    plans, lams, geos, pairs = [], [], [], []
    t_plan = time.perf_counter()
    for g in range(len(W.BATCH_SIZES)):
        geo = W.batch_geometry(g, args.scale)
        pts = torch.from_numpy(geo["points"]).cuda()
        st = api.BoxStructure(pts, geo["lo"], geo["h"], geo["ng"])
        st.max_occupancy = int((st.box_ptr[1:] - st.box_ptr[:-1]).max().item())
        k = 2 * np.pi * geo["edge_wavelengths"] / st.h
        plan = api.Plan(pts, geo["lo"], st.h, st.ng, k, max_nrhs=nrhs, structure=st)
        plans.append(plan)
        geos.append(W.Workload(f"batch{g}", geo["points"], geo["lo"], st.h, st.ng, k, geo["seed"],
                               {"max_occupancy": st.max_occupancy}))
        lams.append(torch.from_numpy(W.strengths(plan.n, nrhs, geo["seed"])).cuda())
        pairs.append(plan.pair_count())
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t_plan
    batch = api.Batch(plans, nrhs=nrhs)
    outs = batch.capture(lams)
    stream = torch.cuda.current_stream()
    med, _ = _events_time(batch.replay, args.ext_steps, 3, stream)
    # the same work as separate per-plan applies, for comparison
    sep, _ = _events_time(lambda: [p.apply(l) for p, l in zip(plans, lams)], max(2, args.ext_steps // 2), 2, stream)
    batch.replay()
    torch.cuda.synchronize()
    errs, cpu_pairs, cpu_s = [], 0, 0.0
    for geo, plan, lam, out in zip(geos, plans, lams, outs):
        targets = _sample_targets(geo.n, args.samples // 8 + 1, 9)
        ref, dt = _oracle_sampled(geo, lam.cpu().numpy(), targets)
        errs.append(float(_rel_l2_cols(out.cpu().numpy()[targets], ref).max()))
        cpu_pairs += len(targets) * nrhs * pairs[len(errs) - 1] / geo.n
        cpu_s += dt
    P = sum(pairs) * nrhs
    line = {"metric": METRIC + " [8 geometries x 8 RHS, one persistent graph-launched kernel]",
            "value": P / med / 1e6, "unit": UNIT, "n_gpus": 1, "steps": args.ext_steps, "warmup": 3,
            "ms_per_step": med, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batched_cylinder_plates", "n_points": [g.n for g in geos],
                       "grids": [g.ng for g in geos], "max_occupancy": [g.meta["max_occupancy"] for g in geos],
                       "nrhs": nrhs, "pairs_per_rhs": pairs, "work_items": batch.info["work_items"],
                       "grid_ctas": batch.info["grid"], "setup_s": t_plan, "setup": "host generation of the 40 M points and strengths, copies, binning, neighbour lists and plans"},
            "separate_applies_ms": sep, "speedup_vs_separate_applies": sep / med,
            "rel_l2_vs_fp64_per_geometry": errs,
            "cpu_baseline": {"value": cpu_pairs / cpu_s / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.samples // 8 + 1} targets per geometry x {nrhs} RHS, {cpu_s:.1f} s "
                                       "(pairs estimated from the mean neighbourhood; includes the oracle's binning)"}}
    print(json.dumps(line))
    return 0


def _plate_points(n, seed):
    """n points uniform on the square z = 0.5 of the unit cube: the paper's random points on a square plate."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(np.concatenate([rng.random((n, 2)), np.full((n, 1), 0.5)], axis=1).astype(np.float32))


def run_tree_sweep(args):
    """The layout comparison of the paper's Fig. 6 (Sec. 4.6) on GB300: square plates of N = 4^L points, the
    CT = 15 tree level (4 points per box on average: N = 4 x boxes) raised or lowered by i in {-3 .. 3}, i.e. a
    plate grid of 2^(L - 1 + i) boxes per side, D = 4 / 4^i points per box.  Laplace kernel (the paper applies a
    potential kernel).  Per configuration: kernel-only time of the indexed layout (Sec. 3.2), the box-level
    redundant layout, the paper's per-target repetition layout (Sec. 3.3), the direct and box-group kernels and the plan's own choice, plus the
    repetition layout's per-apply strength repack; the speedup of repetition over indexing, X = T_indexed /
    T_repetition, next to the paper's kernel model (eq. 28), X = 55.3 lambda t / (N D), whose lambda is fitted
    by least squares in log space over the measured points."""
    import torch
    from paper_2403_01596_gb300 import _capi as C, api, workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    path = C.P2P_PATH_FP32_SHARED
    rows = []
    Ls = [int(v) for v in args.tree_levels.split(",")]
    for L in Ls:
        n = 4 ** L
        pts_np = _plate_points(n, 100 + L)
        pts = torch.from_numpy(pts_np).cuda()
        lam = torch.from_numpy(W.strengths(n, 1, 100 + L)).cuda()
        out = torch.empty_like(lam)
        for i in range(-3, 4):
            lev = L - 1 + i
            if lev < 0 or lev > 20:
                continue
            ng = 2 ** lev
            st = api.BoxStructure(pts, (0.0, 0.0, 0.0), 1.0 / ng, ng)
            sizes = torch.diff(st.box_ptr.long())
            t_max = int(sizes.max().item())
            D = n / st.num_boxes
            row = {"L": L, "i": i, "N": n, "ng": ng, "boxes": st.num_boxes, "D": D, "t": t_max, "ms": {}}
            for name, layout, tuning in (("indexed", "indexed", {"warp_boxes": -1}),
                                          ("redundant", "redundant", {"warp_boxes": -1}),
                                          ("repetition", "repetition", None),
                                          ("direct", "indexed", {"warp_boxes": 4 if D <= 12 else 1}),
                                          ("direct8", "indexed", {"warp_boxes": 8}),
                                          ("direct16", "indexed", {"warp_boxes": 16}),
                                          ("direct32", "indexed", {"warp_boxes": 32}),
                                          ("group", "indexed", {"warp_boxes": -2}),
                                          ("auto", "indexed", None)):
                try:
                    plan = api.Plan(pts, (0.0, 0.0, 0.0), 1.0 / ng, ng, 0.0, kernel="laplace", layout=layout,
                                    tuning=tuning, structure=st)
                except C.P2PError as e:  # records beyond 2^31 entries: not measured
                    row["ms"][name] = None
                    row.setdefault("skipped", {})[name] = str(e)
                    continue
                if "pairs" not in row:
                    row["pairs"] = plan.pair_count()
                evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.ext_steps)]
                for r in range(3 + args.ext_steps):
                    e = evs[r - 3] if r >= 3 else None
                    if e:
                        e[0].record(stream)
                    C.p2p_apply_stage(plan._plan, lam, 1, 1, path, stream)
                    if e:
                        e[1].record(stream)
                    C.p2p_apply_staged(plan._plan, out, 1, 1, 0, path, stream)
                    if e:
                        e[2].record(stream)
                torch.cuda.synchronize()
                row["ms"][name] = statistics.median(e[1].elapsed_time(e[2]) for e in evs)
                if name == "repetition":
                    row["repack_ms"] = statistics.median(e[0].elapsed_time(e[1]) for e in evs)
                    row["records"] = plan.records
                plan.close()
                del plan
            ms = row["ms"]
            if ms.get("repetition") and ms.get("indexed"):
                row["X_rep_over_indexed"] = ms["indexed"] / ms["repetition"]
            if ms.get("redundant") and ms.get("indexed"):
                row["X_redundant_over_indexed"] = ms["indexed"] / ms["redundant"]
            if ms.get("repetition") and ms.get("direct"):
                row["X_rep_over_direct"] = ms["direct"] / ms["repetition"]
            rows.append(row)
            torch.cuda.empty_cache()
    # fit of the paper's kernel model (eq. 28): X = 55.3 lambda t / (N D); log X = log lambda + log(55.3 t / (N D))
    pts_fit = [(r["X_rep_over_indexed"], 55.3 * r["t"] / (r["N"] * r["D"])) for r in rows if "X_rep_over_indexed" in r]
    fit = None
    if pts_fit:
        lx = np.log([p[0] for p in pts_fit])
        lm = np.log([p[1] for p in pts_fit])
        log_lam = float(np.mean(lx - lm))
        pred = lm + log_lam
        ss_res = float(np.sum((lx - pred) ** 2))
        ss_tot = float(np.sum((lx - lx.mean()) ** 2))
        fit = {"model": "X = 55.3 lambda t / (N D) (eq. 28)", "lambda_gpu": float(np.exp(log_lam)),
               "r2_log": 1.0 - ss_res / ss_tot if ss_tot > 0 else None,
               "corr_log": float(np.corrcoef(lx, lm)[0, 1]) if len(lx) > 2 else None,
               "points": len(pts_fit), "paper_lambda_gpu": 640.0}
        for r in rows:
            if "X_rep_over_indexed" in r:
                r["X_model"] = float(np.exp(log_lam) * 55.3 * r["t"] / (r["N"] * r["D"]))
    line = {"metric": METRIC + " [layout comparison, Fig. 6 analogue]", "value": None, "unit": UNIT, "n_gpus": 1,
            "steps": args.ext_steps, "warmup": 3, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "plate_tree_sweep", "levels": Ls, "i": list(range(-3, 4)), "CT": 15,
                       "kernel": "laplace", "nrhs": 1, "l2": "not flushed (kernel-only times of small problems)"},
            "rows": rows, "model_fit": fit}
    print(json.dumps(line))
    return 0


def run_pieces(args):
    """A problem cut into pieces of the size the paper recommends for its repetition kernel (Sec. 4.3: 50 000 -
    150 000 points): sixteen unit-sphere pieces of 65 536 points (32 points per box, leaf edge a quarter
    wavelength, Helmholtz, one RHS), applied as one graph-replayed persistent batch against sixteen separate
    applies (each a staging launch and a pair-kernel launch) issued eagerly, and against the same sixteen applies
    captured in one CUDA graph."""
    import torch
    from paper_2403_01596_gb300 import api, workloads as W
    torch.cuda.set_device(0)
    count, n, ng = 16, 1 << 16, 24
    plans, lams, pairs = [], [], []
    for g in range(count):
        pts = torch.from_numpy(W.unit_sphere(n, 200 + g)).cuda()
        h = 2.0 / ng
        plans.append(api.Plan(pts, (-1.0, -1.0, -1.0), h, ng, 2 * np.pi / (4 * h), tuning={"warp_boxes": -1}))
        lams.append(torch.from_numpy(W.strengths(n, 1, 200 + g)).cuda())
        pairs.append(plans[-1].pair_count())
    stream = torch.cuda.current_stream()
    outs_sep = [torch.empty_like(l) for l in lams]
    batch = api.Batch(plans, nrhs=1)
    outs = batch.capture(lams)
    med_b, _ = _events_time(batch.replay, args.ext_steps, 3, stream)
    med_s, _ = _events_time(lambda: [p.apply(l, out=o) for p, l, o in zip(plans, lams, outs_sep)], args.ext_steps, 3,
                            stream)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for p, l, o in zip(plans, lams, outs_sep):  # warm-up on the capture stream
            p.apply(l, out=o)
    stream.wait_stream(side)
    with torch.cuda.graph(graph):
        for p, l, o in zip(plans, lams, outs_sep):
            p.apply(l, out=o)
    med_g, _ = _events_time(graph.replay, args.ext_steps, 3, stream)
    batch.replay()
    torch.cuda.synchronize()
    diff = max(float((o.reshape(-1) - s.reshape(-1)).abs().max() / s.abs().max()) for o, s in zip(outs, outs_sep))
    # both against the FP64 oracle on sampled targets of two pieces
    errs = {}
    for g in (0, count - 1):
        wl = W.Workload(f"piece{g}", W.unit_sphere(n, 200 + g), (-1.0, -1.0, -1.0), 2.0 / ng, ng,
                        2 * np.pi / (4 * 2.0 / ng), 200 + g)
        targets = _sample_targets(n, 2000, g)
        ref, _ = _oracle_sampled(wl, lams[g].cpu().numpy(), targets)
        errs[f"piece{g}"] = {"batch": float(_rel_l2_cols(outs[g].reshape(-1).cpu().numpy()[targets], ref).max()),
                             "separate": float(_rel_l2_cols(outs_sep[g].reshape(-1).cpu().numpy()[targets], ref).max())}
    P = sum(pairs)
    line = {"metric": METRIC + " [16 pieces of 65 536 points: one batched launch vs separate applies]",
            "value": P / med_b / 1e6, "unit": UNIT, "n_gpus": 1, "steps": args.ext_steps, "warmup": 3,
            "ms_per_step": med_b, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "sphere_pieces", "pieces": count, "n_points_each": n, "grid": ng, "nrhs": 1,
                       "pairs": P, "work_items": batch.info["work_items"]},
            "batch_graph_ms": med_b, "separate_eager_ms": med_s, "separate_graph_ms": med_g,
            "speedup_vs_separate_eager": med_s / med_b, "speedup_vs_separate_graph": med_g / med_b,
            "max_rel_diff_batch_vs_separate": diff, "rel_l2_vs_fp64_sampled": errs}
    print(json.dumps(line))
    return 0


def run_cube(args):
    """Dense uniform cube (32 768 points, 8^3 boxes, k = 8 pi), both source layouts: device-timed applies
    (L2 flushed between them) and the full FP64 oracle on every target."""
    import torch
    from paper_2403_01596_gb300 import _capi as C, api, workloads as W
    import oracle
    torch.cuda.set_device(0)
    peaks = _peaks()
    props = torch.cuda.get_device_properties(0)
    wl = W.cube_dense(int(32768 * args.scale), 0)
    pts = torch.from_numpy(wl.points).cuda()
    lam_np = W.strengths(wl.n, 1, wl.seed)
    lam = torch.from_numpy(lam_np).cuda()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    oracle.build()
    t = time.perf_counter()
    ref = oracle.p2p(wl.points, lam_np, wl.lo, wl.h, wl.ng, wl.k)
    cpu_s = time.perf_counter() - t
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    peak = props.multi_processor_count * MUFU_LANES_PER_SM_CLK * f_max / MUFU_PER_PAIR["helmholtz"] / 1e9
    res = {}
    tuning = {k: v for k, v in (("chunk", args.chunk), ("warps_per_cta", args.warps),
                                ("target_group", args.target_group), ("warp_boxes", args.warp_boxes)) if v} or None
    for layout in ("indexed", "redundant"):
        plan = api.Plan(pts, wl.lo, wl.h, wl.ng, wl.k, layout=layout, tuning=tuning)
        out = torch.empty_like(lam)
        P = plan.pair_count()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.ext_steps)]
        for i in range(3 + args.ext_steps):
            flush.zero_()
            e = evs[i - 3] if i >= 3 else None
            if e:
                e[0].record(stream)
            C.p2p_apply_stage(plan._plan, lam, 1, 1, C.P2P_PATH_FP32_SHARED, stream)
            if e:
                e[1].record(stream)
            C.p2p_apply_staged(plan._plan, out, 1, 1, 0, C.P2P_PATH_FP32_SHARED, stream)
            if e:
                e[2].record(stream)
        torch.cuda.synchronize()
        apply_ms = statistics.median(e[0].elapsed_time(e[2]) for e in evs)
        kern_ms = statistics.median(e[1].elapsed_time(e[2]) for e in evs)
        err = float(np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref))
        res[layout] = {"ms": apply_ms, "pair_kernel_ms": kern_ms, "gpair_s": P / apply_ms / 1e6,
                       "pair_kernel_frac_of_mufu": P / kern_ms / 1e6 / peak, "rel_l2_vs_fp64": err}
    line = {"metric": METRIC + " [dense cube]", "value": res["indexed"]["gpair_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.ext_steps, "warmup": 3, "ms_per_step": res["indexed"]["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "cube_uniform_8x8x8", "n_points": wl.n, "grid": wl.ng, "k": wl.k, "pairs": P,
                       "tuning": tuning or "plan defaults", "l2": "flushed before every apply"},
            "layouts": res,
            "roofline": {"bound": "alu", "kernel": "k_pair", "achieved": P / res["indexed"]["pair_kernel_ms"] / 1e6,
                         "peak": peak, "unit": "Gpair/s", "frac": res["indexed"]["pair_kernel_frac_of_mufu"]},
            "cpu_baseline": {"value": P / cpu_s / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"full FP64 oracle on all {wl.n} targets ({P} pairs, {cpu_s:.1f} s)"}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--layout", choices=("auto", "indexed", "redundant", "symmetric"), default="indexed")
    ap.add_argument("--chunk", type=int, default=0, help="sources per work item (0: library default)")
    ap.add_argument("--warps", type=int, default=0, help="warps per block (0: library default)")
    ap.add_argument("--target-group", type=int, default=0, help="targets per sweep (0: library default)")
    ap.add_argument("--warp-boxes", type=int, default=0,
                    help="direct kernel boxes per warp (1, 2, 4), -1 for the staged pipeline, 0: library default")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tree-levels", default="5,6,7,8,9,10", help="tree_sweep: plate sizes N = 4^L")
    ap.add_argument("--workload", choices=("sweep", "cube", "multirhs", "grad", "batched", "tree_sweep", "pieces"),
                    default="sweep",
                    help="sweep (default): the occupancy sweep; the others measure the extension paths")
    ap.add_argument("--scale", type=float, default=1.0, help="point-count scale of the extension workloads")
    ap.add_argument("--ext-steps", type=int, default=20)
    ap.add_argument("--samples", type=int, default=400, help="oracle-checked targets of the extension workloads")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the redundant-layout and 64-RHS sub-records of the default run")
    ap.add_argument("--extra-steps", type=int, default=10, help="timed applies of each sub-record measurement")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: warmup raised to 3 (timing rule)", file=sys.stderr)
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "cube":
        return run_cube(args)
    if args.workload == "multirhs":
        return run_multirhs(args)
    if args.workload == "grad":
        return run_grad(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "tree_sweep":
        return run_tree_sweep(args)
    if args.workload == "pieces":
        return run_pieces(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
