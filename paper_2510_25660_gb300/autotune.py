"""Launch-configuration autotuner for the render, backward and NLOS kernels.

Searches over threads per CTA, pixels (scan rows) per tile -- which sets the
shared-memory histogram size and hence the privatisation depth -- and CTAs per
SM, timing real launches with CUDA events.  Results are cached in a JSON file
(MT_AUTOTUNE_CACHE, default ~/.cache/mtr_autotune.json) keyed by device name,
kind and workload shape, and applied with mt_set_launch.
"""
from __future__ import annotations

import json
import os
import time

KINDS = {"render": 0, "backward": 1, "nlos": 2}


def cache_path() -> str:
    return os.environ.get("MT_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "mtr_autotune.json"))


def _key(kind, sc, film, spp, depth) -> str:
    import torch
    dev = torch.cuda.get_device_name()
    shape = f"T{film.T}xW{film.W}" if film is not None else "nlos"
    return f"{dev}|{kind}|n{sc.n_tris}|{shape}|spp{spp}|d{depth}|med{int(sc.medium is not None)}"


def _load() -> dict:
    p = cache_path()
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except (OSError, ValueError):
            return {}
    return {}


def _store(d: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    json.dump(d, open(tmp, "w"), indent=1)
    os.replace(tmp, p)


def apply(scene, kind, sc, film, spp, depth) -> dict | None:
    """Apply a cached configuration, if any; returns it."""
    cfg = _load().get(_key(kind, sc, film, spp, depth))
    if cfg:
        scene.set_launch(KINDS[kind], cfg["threads"], cfg["tile"], cfg["ctas_per_sm"])
    return cfg


def tune(scene, kind, sc, film, spp, depth, run, candidates, reps=3, budget_s=60.0) -> dict:
    """Time `run()` (one launch of the kernel) under each candidate
    (threads, tile, ctas_per_sm); keep and cache the fastest."""
    import torch
    best = None
    t_end = time.time() + budget_s
    results = []
    for threads, tile, cps in candidates:
        if time.time() > t_end:
            break
        scene.set_launch(KINDS[kind], threads, tile, cps)
        try:
            run()
            torch.cuda.synchronize()
        except Exception as e:  # a configuration that does not fit is skipped
            results.append({"threads": threads, "tile": tile, "ctas_per_sm": cps, "error": str(e)[:80]})
            continue
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        results.append({"threads": threads, "tile": tile, "ctas_per_sm": cps, "ms": ms})
        if best is None or ms < best["ms"]:
            best = {"threads": threads, "tile": tile, "ctas_per_sm": cps, "ms": ms}
    if best is None:
        raise RuntimeError("no launch configuration ran")
    scene.set_launch(KINDS[kind], best["threads"], best["tile"], best["ctas_per_sm"])
    d = _load()
    d[_key(kind, sc, film, spp, depth)] = dict(best, results=results)
    _store(d)
    return best
