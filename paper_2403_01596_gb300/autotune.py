"""Autotuner for the P2P launch configuration (layout, kernel, source chunk, warps per block).

For a point set and grid, every candidate configuration is built as a plan on
the shared box structure and timed with CUDA events on the current stream
(warm-up, then the median of a few applies).  The winner is cached in a JSON
file keyed by (GPU name, SM count, kernel, occupancy bucket, nrhs, layouts
searched), so a later plan for a similar workload on the same GPU reuses it
without timing.  The occupancy bucket is the power of two nearest to the mean
number of points per non-empty box.

The cache file defaults to $P2P_AUTOTUNE_CACHE, else
~/.cache/p2p_gb300/autotune.json.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading

# staged pipeline (warp_boxes -1) with several chunk / block shapes, the direct kernel with 1 - 32 boxes per warp
# and the box-group kernel (-2, indexed layout only) (one-RHS applies only; for several RHS a plan runs the staged
# pipeline whatever warp_boxes says)
DEFAULT_CANDIDATES = (
    {"chunk": 192, "warps_per_cta": 8, "target_group": 32, "warp_boxes": -1},
    {"chunk": 128, "warps_per_cta": 8, "target_group": 32, "warp_boxes": -1},
    {"chunk": 160, "warps_per_cta": 8, "target_group": 32, "warp_boxes": -1},
    {"chunk": 256, "warps_per_cta": 4, "target_group": 32, "warp_boxes": -1},
    {"chunk": 128, "warps_per_cta": 4, "target_group": 32, "warp_boxes": -1},
    {"chunk": 192, "warps_per_cta": 8, "target_group": 64, "warp_boxes": -1},
    {"chunk": 192, "warps_per_cta": 8, "target_group": 32, "warp_boxes": 1},
    {"chunk": 192, "warps_per_cta": 8, "target_group": 32, "warp_boxes": 2},
    {"chunk": 192, "warps_per_cta": 8, "target_group": 32, "warp_boxes": 4},
    {"chunk": 192, "warps_per_cta": 8, "target_group": 32, "warp_boxes": 8},
    {"chunk": 192, "warps_per_cta": 8, "target_group": 32, "warp_boxes": 16},
    {"chunk": 192, "warps_per_cta": 8, "target_group": 32, "warp_boxes": 32},
    {"chunk": 192, "warps_per_cta": 8, "target_group": 32, "warp_boxes": -2},
)

DEFAULT_LAYOUTS = ("indexed", "redundant", "symmetric")

_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("P2P_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "p2p_gb300", "autotune.json")


def occupancy_bucket(n_points: int, num_boxes: int) -> int:
    if num_boxes <= 0 or n_points <= 0:
        return 0
    d = n_points / num_boxes
    return int(2 ** round(math.log2(max(d, 1.0))))


def cache_key(gpu: str, sms: int, kernel: str, bucket: int, nrhs: int, layouts) -> str:
    return f"v3|{gpu}|{sms}|{kernel}|d{bucket}|r{nrhs}|{'+'.join(sorted(layouts))}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def select(timings: list[dict]) -> dict:
    """The fastest candidate (ties: the smaller chunk, then fewer warps, indexed before redundant)."""
    if not timings:
        raise ValueError("no candidate could be timed")
    return min(timings, key=lambda t: (t["ms"], t["tuning"]["chunk"], t["tuning"]["warps_per_cta"],
                                       t["layout"] != "indexed"))


def _time_plan(plan, lam, out, reps: int) -> float:
    import torch
    s = torch.cuda.current_stream()
    for _ in range(3):
        plan.apply(lam, out=out)
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        plan.apply(lam, out=out)
        e1.record(s)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def tune(structure, k: float, kernel: str = "helmholtz", nrhs: int = 1, layouts=DEFAULT_LAYOUTS,
         candidates=DEFAULT_CANDIDATES, reps: int = 7, use_cache: bool = True, path: str | None = None) -> dict:
    """Times every (layout, candidate) on `structure` and returns the best as
    {"layout", "tuning", "ms", "key", "cached"}."""
    import torch
    from .api import Plan
    dev = structure.points.device
    props = torch.cuda.get_device_properties(dev)
    key = cache_key(props.name, props.multi_processor_count, kernel,
                    occupancy_bucket(structure.n, structure.num_boxes), nrhs, layouts)
    with _lock:
        cache = load_cache(path) if use_cache else {}
    if use_cache and key in cache:
        hit = dict(cache[key])
        hit["cached"] = True
        hit["key"] = key
        return hit
    g = torch.Generator(device="cpu").manual_seed(0)
    lam = torch.complex(torch.randn(structure.n, nrhs, generator=g), torch.randn(structure.n, nrhs, generator=g))
    lam = lam.to(torch.complex64).to(dev)
    out = torch.empty_like(lam)
    timings = []
    for layout in layouts:
        for cand in candidates:
            if layout == "symmetric" and cand.get("warp_boxes", 0) > 0:
                continue  # the symmetric layout always runs the staged pipeline
            if layout != "indexed" and cand.get("warp_boxes", 0) == -2:
                continue  # the box-group kernel serves the indexed layout only
            plan = Plan(structure.points, structure.lo, structure.h, structure.ng, k, kernel=kernel, layout=layout,
                        max_nrhs=nrhs, tuning=dict(cand), structure=structure)
            timings.append({"layout": layout, "tuning": dict(cand), "ms": _time_plan(plan, lam, out, reps)})
            plan.close()
    best = select(timings)
    result = {"layout": best["layout"], "tuning": best["tuning"], "ms": best["ms"],
              "all": [(t["layout"], t["tuning"]["chunk"], t["tuning"]["warps_per_cta"],
                       t["tuning"].get("warp_boxes", 0), round(t["ms"], 5)) for t in timings]}
    if use_cache:
        with _lock:
            cache = load_cache(path)
            cache[key] = result
            save_cache(cache, path)
    result = dict(result)
    result["cached"] = False
    result["key"] = key
    return result


def best_config(wl, points=None, nrhs: int = 1, kernel: str = "helmholtz", **kw) -> dict:
    """Tunes a workload (workloads.Workload) on the current CUDA device."""
    import torch
    from .api import BoxStructure
    pts = points if points is not None else torch.from_numpy(wl.points).cuda()
    st = BoxStructure(pts, wl.lo, wl.h, wl.ng)
    return tune(st, wl.k, kernel=kernel, nrhs=nrhs, **kw)
