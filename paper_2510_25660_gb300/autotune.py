"""Launch-configuration autotuner for the render, backward and NLOS kernels.

Searches over threads per CTA, pixels (scan rows) per tile -- which sets the
shared-memory histogram size and hence the privatisation depth -- CTAs per
SM, the kernel form and option bits, and, for the wavefront form, the paths
in flight per thread (the path-pool size divided by the threads of one
wavefront launch, 8 CTAs of 256 threads per SM), timing real launches with
CUDA events.  Results are cached in a JSON file (MT_AUTOTUNE_CACHE, default
~/.cache/mtr_autotune.json) keyed by device name, kind and workload shape,
and applied with mt_set_launch and mt_set_wavefront_pool.
"""
from __future__ import annotations

import json
import os
import time

KINDS = {"render": 0, "backward": 1, "nlos": 2}


TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "launch_table.json")


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
    """Apply a cached configuration (user cache first, then the table shipped
    with the package), if any; returns it."""
    key = _key(kind, sc, film, spp, depth)
    cfg = _load().get(key)
    if cfg is None and os.path.exists(TABLE):
        cfg = json.load(open(TABLE)).get(key)
    if cfg:
        scene.set_launch(KINDS[kind], cfg["threads"], cfg["tile"], cfg["ctas_per_sm"], cfg.get("priv", -1),
                         cfg.get("options", 0))
        if kind != "nlos":
            scene.set_wavefront_pool(pool_paths(cfg.get("paths_per_thread", 0)))
    return cfg


WF_CTAS_PER_SM, WF_THREADS = 8, 256  # the grid of every wavefront launch


def pool_paths(paths_per_thread) -> int:
    """Path-pool size for `paths_per_thread` paths per thread of a wavefront
    launch on this GPU (0 = the library's default pool)."""
    if not paths_per_thread:
        return 0
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return int(min(1 << 22, max(32, paths_per_thread * sms * WF_CTAS_PER_SM * WF_THREADS)))


def tune(scene, kind, sc, film, spp, depth, run, candidates, reps=3, budget_s=60.0) -> dict:
    """Time `run()` (one launch of the kernel) under each candidate
    (threads, tile, ctas_per_sm, priv_bins[, options[, paths_per_thread]]);
    keep and cache the fastest."""
    import torch
    best = None
    t_end = time.time() + budget_s
    results = []
    for cand in candidates:
        threads, tile, cps, priv = cand[:4]
        opts = cand[4] if len(cand) > 4 else 0
        ppt = cand[5] if len(cand) > 5 else 0
        if time.time() > t_end:
            break
        rec = {"threads": threads, "tile": tile, "ctas_per_sm": cps, "priv": priv, "options": opts,
               "paths_per_thread": ppt}
        scene.set_launch(KINDS[kind], threads, tile, cps, priv, opts)
        if kind != "nlos":
            scene.set_wavefront_pool(pool_paths(ppt))
        try:
            run()
            torch.cuda.synchronize()
        except Exception as e:  # a configuration that does not fit is skipped
            results.append(dict(rec, error=str(e)[:80]))
            continue
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        results.append(dict(rec, ms=ms))
        if best is None or ms < best["ms"]:
            best = dict(rec, ms=ms)
    if best is None:
        raise RuntimeError("no launch configuration ran")
    scene.set_launch(KINDS[kind], best["threads"], best["tile"], best["ctas_per_sm"], best["priv"], best["options"])
    if kind != "nlos":
        scene.set_wavefront_pool(pool_paths(best["paths_per_thread"]))
    d = _load()
    d[_key(kind, sc, film, spp, depth)] = dict(best, results=results)
    _store(d)
    return best


TILES = (1, 2, 4, 8, 16)          # pixels per warp tile (renders) or scan rows per CTA tile (NLOS)
PATHS_PER_THREAD = (1, 2, 4, 8, 0)  # wavefront form; 0 = the default pool (about 13 paths per thread)
CTAS_PER_SM = (0, 4)              # 0 = as many as fit (occupancy), else a cap on resident CTAs per SM


def candidates(kind, film_T, wavefront_only=False):
    """The search space, as (threads, tile, ctas_per_sm, priv_bins, options[,
    paths_per_thread]) tuples.  NLOS: threads x scan rows per CTA tile x
    CTAs per SM x privatisation (all bins / none) x warp-aggregated atomics.
    Renders: first the wavefront form at 1, 2, 4 and 8 paths per thread and
    the default pool (so that a time budget never cuts off the form that wins
    on large workloads), then the persistent kernel's threads x pixels per
    warp tile x CTAs per SM x privatisation depth (all that fit, none, T/4,
    T/2) x options (aggregation, deferred refill).  Tiles or depths whose
    shared memory does not fit fail to launch and are skipped by `tune`."""
    return _candidates(kind, film_T, wavefront_only)


def _candidates(kind, film_T, wavefront_only=False):
    out = []
    if kind == "nlos":
        for threads in (128, 256):
            for tile in TILES:
                for cps in CTAS_PER_SM:
                    for priv in (-1, 0):
                        for opt in (0, 1):
                            out.append((threads, tile, cps, priv, opt))
        return out
    for ppt in PATHS_PER_THREAD:
        out.append((256, 1, 0, 0, 4, ppt))
    if not wavefront_only:
        for threads in (128, 256):
            for tile in TILES:
                for cps in CTAS_PER_SM:
                    for priv in (-1, 0, film_T // 4, film_T // 2):
                        for opt in (0, 1, 16 << 8):
                            out.append((threads, tile, cps, priv, opt, 0))
    return out


def main():
    """Tune the benchmark workloads on this GPU and print the table entries."""
    import sys
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2510_25660_gb300 import api, scenes
    from paper_2510_25660_gb300 import build as b
    b.build()
    api.load()
    found = {}
    which = sys.argv[1:] or ["render", "backward", "nlos"]
    if "render" in which:
        sc = scenes.large_scene()
        f = scenes.LARGE_FILM
        s = api.Scene(sc)
        film, steady = api.new_film(f.H, f.W, f.T)
        run = lambda: api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, 256, 1, 8, out=(film, steady))
        best = tune(s, "render", sc, f, 256, 8, run, _candidates("render", f.T), reps=2, budget_s=120)
        found[_key("render", sc, f, 256, 8)] = best
        del s, film, steady
    if "backward" in which:
        sc = scenes.diff_scene()
        f = scenes.DIFF_FILM
        s = api.Scene(sc)
        film, steady = api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, 64, 1, 8)
        g = torch.randn_like(film)
        out = (torch.zeros((sc.n_tris, 3), device="cuda"), torch.zeros((len(sc.emitters), 3), device="cuda"),
               torch.zeros(1, device="cuda"))
        run = lambda: api.render_backward(s, f.T, f.start_opl, f.bin_width, 64, 1, 8, g, out=out)
        best = tune(s, "backward", sc, f, 64, 8, run, _candidates("backward", f.T), reps=2, budget_s=60)
        found[_key("backward", sc, f, 64, 8)] = best
        del s
    if "nlos" in which:
        sc = scenes.nlos_scene()
        s = api.Scene(sc)
        lasers = torch.from_numpy(scenes.wall_grid(64, 64)).cuda()
        nf = [None]

        def run():
            nf[0] = api.render_nlos(s, lasers, None, api.MT_CONFOCAL, scenes.NLOS_T, scenes.NLOS_START,
                                    scenes.NLOS_W, 1024, 1, out=nf[0])
        best = tune(s, "nlos", sc, None, 1024, 0, run, _candidates("nlos", scenes.NLOS_T), reps=3, budget_s=60)
        found[_key("nlos", sc, None, 1024, 0)] = best
    print(json.dumps(found, indent=1))


if __name__ == "__main__":
    main()
