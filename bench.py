"""Benchmark: time-resolved path tracing on GB300 (arXiv 2510.25660).

One step = one transient render of the large static scene (1.16M triangles,
512x512 pixels, T = 2048 bins of 0.005 m, 256 spp, max_depth 8, NEE + MIS),
through the C ABI, with the scene resident in HBM.  Prints one JSON line:
value = path vertices/s (whole job), roofline of the render kernel, e2e
through host buffers, the oracle timed on the host cores as cpu_baseline,
and secondary figures (backward grads/s on the differentiable scene, batched
NLOS connections/s).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# row bands of the end-to-end render, as fractions of the frame height: later bands are smaller so
# that the one copy that cannot overlap a render is short (measured on the 512-row frame with a 31-ms
# scene creation: one band 153 ms, 2 equal bands 147, 4 equal bands 130.5, 8 equal bands 130.3;
# with the current kernels: 160/144/128/80 rows 111.0 ms, 144/128/112/80/48 108.4,
# 128/112/96/80/64/32 108.3, 112/96/96/80/64/40/24 108.9)
# end-to-end step: the frame as three windows (472, 32 and 8 of 512 rows), each copied to the host in
# bands of 8 rows as its bands finish (mt_render_to_host), so a window's last copies overlap the next
E2E_WINDOWS = (472 / 512, 32 / 512, 8 / 512)
E2E_BAND_ROWS = 8
METRIC = "time-resolved path vertices/s on 1 GB300"  # both arms report the same metric
L2_FLUSH_BYTES = 512 << 20
WORKLOAD = "large static scene: 1,164,296-triangle fBm heightfield + 200 icospheres, 4 area lights, " \
           "512x512 px, T=2048 bins x 0.005 m from 12 m, 256 spp, max_depth 8, NEE+MIS, FP32 film"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
                power.append(float(p[3]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


def _kernel_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2510_25660_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def _profile(kernel_hash, name):
    """The committed ncu summary profiles/<name>.json, or None if the kernel
    sources changed since it was captured."""
    p = os.path.join(ROOT, "profiles", name + ".json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    return d if d.get("kernel_hash") == kernel_hash else None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def aggregate_ranks(seconds, vertices, world_size, device):
    """Whole-job figures over ranks: the slowest rank's time and the sum of
    the path vertices all ranks traced (replicas: no data exchange)."""
    if world_size <= 1:
        return seconds, vertices
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    v = torch.tensor([vertices], dtype=torch.float64, device=device)
    dist.all_reduce(v)
    return float(t.item()), float(v.item())


_ORACLE = {}


def _oracle_worker_init():
    """Pool worker: the oracle's copy of the benchmark scene, built once."""
    from paper_2510_25660_gb300 import scenes
    from oracle import oracle as O
    sc = scenes.large_scene()
    _ORACLE["osc"] = O.OracleScene(sc)
    _ORACLE["film"] = scenes.LARGE_FILM


def _oracle_segment(task):
    """Render pixel segments (x0, x1, y) of the benchmark frame at full spp and
    depth until `budget_s` of work is done; returns (vertices, seconds, pixels)."""
    segs, spp, depth, budget_s = task
    osc, f = _ORACLE["osc"], _ORACLE["film"]
    v, t, px = 0, 0.0, 0
    for (x0, x1, y) in segs:
        if t >= budget_s:
            break
        t0 = time.perf_counter()
        r = osc.render(f.H, f.W, 16, f.start_opl, f.bin_width, spp, 25660, depth, crop=(x0, x1, y, y + 1))
        t += time.perf_counter() - t0
        v += r["counters"]["vertices"]
        px += x1 - x0
    return v, t, px


def _oracle_pool():
    import multiprocessing as mp
    n = max(1, os.cpu_count() or 1)
    return mp.get_context("spawn").Pool(n, initializer=_oracle_worker_init), n


def cpu_baseline(sc, film_spec, spp, depth, budget_s=12.0):
    """The oracle as it stands on every host core: one spawned process per core,
    each rendering its own 8-pixel row segments of the benchmark frame at full
    spp and depth for ~budget_s; throughput = all vertices / the longest worker."""
    from oracle import oracle as O
    O.build()
    f = film_spec
    pool, n = _oracle_pool()
    try:
        cx, cy = f.W // 2, f.H // 2
        tasks = []
        for w in range(n):
            segs = [(cx - 128 + 8 * ((w + n * k) % 32), cx - 120 + 8 * ((w + n * k) % 32), cy + (w + n * k) // 32)
                    for k in range(256 // n * 32)]
            tasks.append((segs, spp, depth, budget_s))
        res = pool.map(_oracle_segment, tasks)
    finally:
        pool.close()
        pool.join()
    v = sum(r[0] for r in res)
    t = max(r[1] for r in res)
    px = sum(r[2] for r in res)
    one = res[0][0] / res[0][1]
    return {"value": v / t, "unit": "path vertices/s", "cores": n, "kind": "oracle",
            "sample": f"{px} pixels below the centre of the 512x512 frame (8-pixel row segments, disjoint per "
                      f"process) x {spp} spp, max_depth {depth}, FP64, {n} processes for {t:.1f} s; one process "
                      f"alone {one:.0f} vertices/s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2510_25660_gb300 import scenes
    from oracle import oracle as O
    O.build()
    f = scenes.LARGE_FILM
    spp, depth = 256, 8
    pool, n = _oracle_pool()
    times, verts = [], []
    cx, cy = f.W // 2, f.H // 2
    try:
        pool.map(_oracle_segment, [([(cx, cx + 1, cy)], 1, 1, 1.0)] * n)   # workers built and warm
        for k in range(args.warmup + args.steps):
            # one step: 4 x 8 pixels x 256 spp per process, disjoint across processes and steps
            tasks = [([(cx - 128 + 8 * w, cx - 120 + 8 * w, cy + 8 + 4 * k + j) for j in range(4)], spp, depth, 1e9)
                     for w in range(n)]
            t0 = time.perf_counter()
            res = pool.map(_oracle_segment, tasks)
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                times.append(dt)
                verts.append(sum(r[0] for r in res))
    finally:
        pool.close()
        pool.join()
    v = sum(verts) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "path vertices/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"32 pixels x 256 spp per process per step, {n} processes"},
            "cpu_baseline": {"value": v, "unit": "path vertices/s", "cores": n, "kind": "oracle",
                             "sample": f"{args.steps} steps of 32 pixels x 256 spp on each of {n} processes, "
                                       f"max_depth 8, FP64"},
            "e2e": {"value": v, "unit": "path vertices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile", default="", help="small | trace: launches of the hot kernels on reduced sizes (for ncu)")
    ap.add_argument("--profile-summary", nargs=2, metavar=("CSV", "LOG"),
                    help="write profiles/k_wf_trace_large_scene.json from the ncu CSV and log of --profile trace")
    ap.add_argument("--compare", action="store_true",
                    help="batched NLOS vs per-scan-point launches; adjoint vs finite differences")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_summary:
        return profile_summary(args.profile_summary[0], args.profile_summary[1],
                               os.path.join(ROOT, "profiles", "k_wf_trace_large_scene.json"))
    if args.profile:
        return profile_case(args.profile)
    if args.compare:
        return compare()

    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2510_25660_gb300 import api, autotune, scenes
    from paper_2510_25660_gb300 import build as b
    if rank == 0 or ws == 1:
        b.build()
    if ws > 1:
        torch.distributed.barrier()
    api.load()

    sc = scenes.large_scene()
    f = scenes.LARGE_FILM
    spp, depth, seed = 256, 8, scenes.RENDER_SEED
    s = api.Scene(sc)
    cfg = autotune.apply(s, "render", sc, f, spp, depth)
    wavefront = bool(cfg and cfg.get("options", 0) & api.MT_OPT_WAVEFRONT)
    if wavefront:
        # CUDA events at the stage boundaries time the traversal kernels inside the timed region
        s.set_launch(api.MT_LAUNCH_RENDER, cfg["threads"], cfg["tile"], cfg["ctas_per_sm"], cfg.get("priv", -1),
                     cfg["options"] | api.MT_OPT_STAGE_TIMING)
    film, steady = api.new_film(f.H, f.W, f.T)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, spp, seed, depth, out=(film, steady))

    for _ in range(max(3, args.warmup)):
        step()
    s.sync()
    # algorithmic traffic per launch from the counters of one identical launch
    s.read_counters(reset=True)
    api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, spp, seed, depth, flags=api.MT_COUNTERS,
               out=(film, steady))
    cnt = s.read_counters(reset=True)
    s.sync()
    film_bytes = film.numel() * 4 + steady.numel() * 4
    trav_bytes = cnt["node_bytes"] + cnt["tri_tests"] * 48
    alg_bytes = trav_bytes + cnt["vertices"] * 32 + film_bytes
    # timed region
    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    s.read_counters(reset=True)
    s.stage_times(reset=True)
    launches0 = s.stats()["launches"]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        flush.fill_(float(k))                 # write > L2 between timed iterations
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    s.sync()
    run_cnt = s.read_counters(reset=True)
    stages = s.stage_times(reset=True)
    launches = s.stats()["launches"] - launches0
    step_ms = [a.elapsed_time(b_) for a, b_ in ev]
    total_s, total_vertices = aggregate_ranks(sum(step_ms) / 1000.0, float(run_cnt["vertices"]), ws, "cuda")
    value = total_vertices / total_s
    mean_ms = 1000.0 * total_s / args.steps
    hbm_peak, hbm_kind = _peaks()
    render_achieved = alg_bytes / (mean_ms / 1000.0) / 1e9
    khash = _kernel_hash()
    # measured rates of the traversal pass's own access patterns on this GPU (the roofline's denominators)
    l2_gbs = api.microbench(api.MT_MICRO_GATHER32, 64 << 20, 256)
    red_gops = api.microbench(api.MT_MICRO_RED_GLOBAL, 1 << 30, 64)
    red_shared_gops = api.microbench(api.MT_MICRO_RED_SHARED, 1 << 20, 1024)
    prof = _profile(khash, "k_wf_trace_large_scene") if wavefront else None
    if wavefront:
        # dominant kernel: the BVH traversal pass k_wf_trace (extension rays, then the shadow rays
        # of the previous shading pass; the last shading pass's shadow rays in k_wf_shadow),
        # timed by its own events on the render stream
        trav_ms = (stages["extend_ms"] + stages["shadow_ms"]) / args.steps
        achieved = trav_bytes / (trav_ms / 1000.0) / 1e9
        kernel_name = ("k_wf_trace (+ k_wf_shadow for the last pass): BVH traversal of extension and "
                       "shadow rays, with the film splats of unoccluded shadow rays")
        per_unit = "per ray: BVH node bytes fetched (32 B per node) + 48 B per triangle tested"
        stage_ms = {k: v / args.steps for k, v in stages.items() if k.endswith("_ms")}
        stage_ms["share_of_step"] = {k: v / mean_ms for k, v in stage_ms.items()}
        # DRAM bytes per render: the ncu capture of every k_wf_trace launch of one 256x256-px render
        # of the same scene, scaled by rays to this render (null once the kernels changed)
        traffic = None
        if prof:
            traffic = prof["dram_bytes_per_ray"] * cnt["rays"]
        n_atom = cnt["gmem_splats"] * 3  # three colour channels per splat
        terms = {"l2_gather_ms": trav_bytes / (l2_gbs * 1e9) * 1e3,
                 "atomic_ms": n_atom / (red_gops * 1e9) * 1e3,
                 "hbm_ms": (traffic if traffic is not None else film_bytes) / (hbm_peak * 1e9) * 1e3}
        binding = max(terms, key=terms.get)
        t_star = terms[binding]
        roofline = {
            "bound": "l2", "achieved": achieved, "peak": l2_gbs, "unit": "GB/s", "frac": achieved / l2_gbs,
            "traffic": traffic,
            "peak_kind": "measured in this run: mt_microbench random 32-B loads from a 64 MB (L2-resident) "
                         "buffer on this GPU",
            "kernel": kernel_name, "algorithmic_bytes_per_launch": trav_bytes,
            "launch": "one render's traversal pass (all its k_wf_trace launches); bytes and time per render",
            "per_unit": per_unit, "units_per_launch": cnt["rays"],
            "time_ms_per_launch": trav_ms,
            "terms_ms": terms, "binding_term": binding, "t_star_ms": t_star, "t_star_frac": t_star / trav_ms,
            "terms_note": "T* = max(B_L2 / measured L2 gather rate, N_atomic / measured red.global rate, "
                          "B_DRAM / measured HBM copy rate); N_atomic counts every film and steady-image "
                          "splat of the render (3 atomics each, an upper bound for this pass); B_DRAM from "
                          "the ncu capture (film bytes when it is stale)",
            "hbm": {"dram_bytes_per_launch": traffic,
                    "achieved": traffic / (trav_ms / 1000.0) / 1e9 if traffic is not None else None,
                    "peak": hbm_peak, "peak_kind": hbm_kind + " (MEASURED_PEAKS.json hbm_gbs)" if hbm_kind ==
                    "measured" else hbm_kind, "unit": "GB/s",
                    "frac": traffic / (trav_ms / 1000.0) / 1e9 / hbm_peak if traffic is not None else None},
            "alu_issue": prof.get("issue") if prof else None,
            "rates": {"l2_gather32_gbs": l2_gbs, "red_global_gops": red_gops, "red_shared_gops": red_shared_gops},
            "stage_ms_per_step": stage_ms,
            "whole_render": {"algorithmic_bytes": alg_bytes, "achieved_gbs": render_achieved},
            "counts": cnt, "kernel_hash": khash,
        }
    else:
        roofline = {"bound": "l2", "achieved": render_achieved, "peak": l2_gbs, "unit": "GB/s",
                    "frac": render_achieved / l2_gbs, "traffic": None, "kernel": "k_render (forward megakernel)",
                    "algorithmic_bytes_per_launch": alg_bytes, "counts": cnt, "kernel_hash": khash}

    # e2e: host arrays in, film out, through the public API (scene load + render + read-back)
    e2e = None
    if rank == 0 or ws == 1:
        pin = torch.empty(film.shape, dtype=torch.float32, pin_memory=True)
        pin_s = torch.empty(steady.shape, dtype=torch.float32, pin_memory=True)
        h2d = sc.tris.nbytes + sc.n_tris * 20 + len(sc.emitters) * 36
        # the step's inputs live in pinned host memory (numpy views of page-locked tensors)
        sc_host = dataclasses.replace(sc, **{k: torch.from_numpy(getattr(sc, k)).pin_memory().numpy()
                                             for k in ("tris", "albedo", "roughness", "mtype")})
        # the frame renders as film windows; within each, every band of E2E_BAND_ROWS rows is copied to
        # the host on a second stream as soon as its paths have finished (mt_render_to_host)
        win_rows = [int(round(x * f.H)) for x in E2E_WINDOWS]
        win_rows[-1] = f.H - sum(win_rows[:-1])
        copy_stream = torch.cuda.Stream()
        e_times, e_verts = [], 0
        for k in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s2 = api.Scene(sc_host)
            autotune.apply(s2, "render", sc_host, f, spp, depth)
            r0 = 0
            for rows in win_rows:
                api.render_to_host(s2, rows, f.W, f.T, f.start_opl, f.bin_width, spp, seed, depth,
                                   pin[r0:r0 + rows], pin_s[r0:r0 + rows], E2E_BAND_ROWS, copy_stream,
                                   out=(film[r0:r0 + rows], steady[r0:r0 + rows]), window=(f.H, r0))
                r0 += rows
            torch.cuda.synchronize()
            e_times.append(time.perf_counter() - t0)
            e_verts = s2.read_counters(reset=True)["vertices"]
            del s2
        e2e = {"value": e_verts / min(e_times), "unit": "path vertices/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(film_bytes), "ms_per_step": 1000 * min(e_times),
               "note": f"scene arrays from pinned host memory (BVH build included) + render as film windows of "
                       f"{win_rows} rows, each with its film and steady image copied to pinned host memory in bands "
                       f"of {E2E_BAND_ROWS} rows on a second stream as the bands finish (mt_render_to_host); best of 3"}

    extras = {}
    if not args.no_extras and (rank == 0 or ws == 1):
        extras = secondary(api, autotune, scenes)
        extras["comparisons"] = comparisons(api, autotune, scenes)

    line = {
        "metric": METRIC,
        "value": value, "unit": "path vertices/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": "replicas" if ws > 1 else "single GPU",
                   "l2": f"{L2_FLUSH_BYTES >> 20} MB buffer written between timed steps; film output "
                         f"{film_bytes / 1e9:.2f} GB per step",
                   "bvh": s.stats()},
        "roofline": roofline,
        "clocks": clk,
        "gpu_launches": launches,
        "e2e": e2e,
        "step_ms": step_ms,
    }
    line.update(extras)
    if (rank == 0 or ws == 1) and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(sc, f, spp, depth)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def profile_case(which):
    """Launches of the hot kernels for ncu captures (small cases only).
    small: the large scene (full geometry) at 256x256 px, 256 spp (16.7M paths:
    four fills of the path pool, so mid-render passes run with a full pool;
    1.6 GB film) with the launch configuration of the benchmark, three times;
    the differentiable scene's backward at 64x64; a 16x16 confocal NLOS grid.
    trace: one 256x256-px, 256-spp render of the large scene in the
    benchmark's configuration (every k_wf_trace launch of it, for one-pass DRAM
    counters), then the same render with MT_COUNTERS, whose ray count it
    prints for scaling the bytes to other renders."""
    import torch
    from paper_2510_25660_gb300 import api, scenes
    from paper_2510_25660_gb300 import build as b
    b.build()
    api.load()
    from paper_2510_25660_gb300 import autotune
    sc = scenes.large_scene()
    f = scenes.LARGE_FILM
    s = api.Scene(sc)
    autotune.apply(s, "render", sc, f, 256, 8)
    film, steady = api.new_film(256, 256, f.T)
    if which == "trace":
        api.render(s, 256, 256, f.T, f.start_opl, f.bin_width, 256, scenes.RENDER_SEED, 8, out=(film, steady))
        s.sync()
        s.read_counters(reset=True)
        api.render(s, 256, 256, f.T, f.start_opl, f.bin_width, 256, scenes.RENDER_SEED, 8, flags=api.MT_COUNTERS,
                   out=(film, steady))
        c = s.read_counters(reset=True)
        print(json.dumps({"profile_case": "trace", "rays": c["rays"], "paths": c["paths"],
                          "node_bytes": c["node_bytes"], "tri_tests": c["tri_tests"]}), flush=True)
        return
    for _ in range(3):
        api.render(s, 256, 256, f.T, f.start_opl, f.bin_width, 256, 1, 8, out=(film, steady))
    s.sync()
    del s
    sc = scenes.diff_scene()
    f = scenes.DIFF_FILM
    s = api.Scene(sc)
    film, steady = api.render(s, 64, 64, f.T, f.start_opl, f.bin_width, 16, 1, 8)
    for _ in range(2):
        api.render_backward(s, f.T, f.start_opl, f.bin_width, 16, 1, 8, torch.randn_like(film))
    s.sync()
    del s
    sc = scenes.nlos_scene()
    s = api.Scene(sc)
    lasers = torch.from_numpy(scenes.wall_grid(16, 16)).cuda()
    for _ in range(2):
        api.render_nlos(s, lasers, None, api.MT_CONFOCAL, scenes.NLOS_T, 0.0, scenes.NLOS_W, 1024, 1)
    s.sync()
    print("profile case done")


def profile_summary(csv_path, log_path, out_path):
    """profiles/k_wf_trace_large_scene.json from the ncu CSV of the `trace`
    profile case (dram__bytes_read.sum, dram__bytes_write.sum and
    gpu__time_duration.sum of every k_wf_trace launch) and that run's log (ray
    count of the render).  Only the launches of the timed form (no counters)
    are summed."""
    import csv
    rows = [r for r in csv.reader(l for l in open(csv_path) if not l.startswith("=="))]
    head = rows[0]
    ki, mi, vi = head.index("Kernel Name"), head.index("Metric Name"), head.index("Metric Value")
    idi = head.index("ID")
    launches = {}
    for r in rows[1:]:
        if len(r) <= vi or "k_wf_trace<" not in r[ki]:
            continue
        targs = r[ki].split("k_wf_trace<", 1)[1].split(">", 1)[0].replace(" ", "")
        if targs.split(",")[1] not in ("0", "false"):  # CNT = true: the counting render
            continue
        v = float(r[vi].replace(",", ""))
        unit = r[head.index("Metric Unit")] if "Metric Unit" in head else ""
        if r[mi].startswith("dram__bytes"):
            v *= {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(unit, 1)
        elif r[mi] == "gpu__time_duration.sum":
            v *= {"nsecond": 1e-6, "usecond": 1e-3, "msecond": 1.0}.get(unit, 1e-6)
        launches.setdefault(r[idi], {})[r[mi]] = v
    info = None
    for l in open(log_path):
        if l.startswith("{") and "profile_case" in l:
            info = json.loads(l)
    rd = sum(x.get("dram__bytes_read.sum", 0) for x in launches.values())
    wr = sum(x.get("dram__bytes_write.sum", 0) for x in launches.values())
    ms = sum(x.get("gpu__time_duration.sum", 0) for x in launches.values())
    d = {"kernel": "k_wf_trace (timed form)", "kernel_hash": _kernel_hash(),
         "workload": "one render of the 1,164,296-triangle scene, 256x256 px, 256 spp, max_depth 8, T = 2048, "
                     "benchmark launch configuration (16.7 M paths, 4 fills of the path pool)",
         "command": "python bench.py --profile trace > trace.log && ncu --metrics "
                    "dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none "
                    "-k regex:k_wf_trace --csv --log-file trace_dram.csv python bench.py --profile trace",
         "launches": len(launches), "rays": info["rays"], "dram_bytes_read": rd, "dram_bytes_write": wr,
         "gpu_time_ms_serialised": ms, "dram_bytes_per_ray": (rd + wr) / info["rays"]}
    old = json.load(open(out_path)) if os.path.exists(out_path) else {}
    if "issue" in old:
        d["issue"] = old["issue"]
    json.dump(d, open(out_path, "w"), indent=1)
    print(json.dumps(d))


def comparisons(api, autotune, scenes, per_point=256):
    """The two comparisons the method's own claims set up, at equal sample
    counts.  (1) Batched NLOS (Sec. 4.5): all 4096 confocal scan points of the
    64x64 grid in one graph launch against one launch per scan point, timed
    over `per_point` points and scaled to 4096, with the film error of each
    against a 16x-spp reference over those points.  (2) Adjoint (Sec. 4.4):
    one path-replay backward pass (every albedo's gradient) against central
    differences of forward renders for 32 parameters (two renders each), with
    the relative difference of the two gradients."""
    import numpy as np
    import torch
    out = {}
    sc = scenes.nlos_scene()
    s = api.Scene(sc)
    cfg = autotune.apply(s, "nlos", sc, None, 1024, 0) or {}
    pts = torch.from_numpy(scenes.wall_grid(64, 64)).cuda()
    T, W0, spp = scenes.NLOS_T, scenes.NLOS_W, 1024
    film = torch.empty((4096, T), device="cuda")
    steady = torch.empty(4096, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        api.render_nlos(s, pts, None, api.MT_CONFOCAL, T, 0.0, W0, spp, 1, out=(film, steady))
    torch.cuda.synchronize()
    e0.record()
    api.render_nlos(s, pts, None, api.MT_CONFOCAL, T, 0.0, W0, spp, 1, out=(film, steady))
    e1.record()
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1)
    # reference for the error: the same points at 16x the samples (another seed)
    sub = pts[:per_point].contiguous()
    ref, ref_s = api.render_nlos(s, sub, None, api.MT_CONFOCAL, T, 0.0, W0, 16 * spp, 99)
    # one plain launch per scan point through the same API, same kernel and launch configuration
    s.set_launch(api.MT_LAUNCH_NLOS, cfg.get("threads", 0), cfg.get("tile", 0), 0, cfg.get("priv", -1),
                 cfg.get("options", 0) | api.MT_OPT_NO_GRAPH)
    pf = torch.empty((per_point, T), device="cuda")
    ps = torch.empty(per_point, device="cuda")
    rows = [(pf[i:i + 1], ps[i:i + 1]) for i in range(per_point)]
    pt_rows = [pts[i:i + 1].contiguous() for i in range(per_point)]
    for i in range(min(32, per_point)):
        api.render_nlos(s, pt_rows[i], None, api.MT_CONFOCAL, T, 0.0, W0, spp, 1, out=rows[i])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record()
    for i in range(per_point):
        api.render_nlos(s, pt_rows[i], None, api.MT_CONFOCAL, T, 0.0, W0, spp, 1, out=rows[i])
    e1.record()
    torch.cuda.synchronize()
    loop_wall_ms = 1000 * (time.perf_counter() - t0)
    loop_ms = e0.elapsed_time(e1)

    def err(a, b):
        return float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))

    def coarse(x):  # 64 time bins of 19.2 cm (64 of the film's bins each)
        return x.reshape(x.shape[0], 64, -1).sum(2)

    out["nlos_batched_vs_per_point"] = {
        "workload": "64x64 confocal scan, 1024 spp, T=4096 x 3 mm, 49.4k hidden triangles; per point: one "
                    f"direct launch per scan point (timed over the first {per_point} points, scaled to 4096), "
                    "same kernel and launch configuration",
        "batched_ms_4096_points": batched_ms, "per_point_loop_ms_4096_points": loop_ms * 4096 / per_point,
        "per_point_loop_wall_ms_4096_points": loop_wall_ms * 4096 / per_point,
        "speedup": loop_ms * 4096 / per_point / batched_ms,
        "film_rel_err_batched": err(coarse(film[:per_point]), coarse(ref)),
        "film_rel_err_per_point": err(coarse(pf), coarse(ref)),
        "steady_rel_err_batched": err(steady[:per_point], ref_s), "steady_rel_err_per_point": err(ps, ref_s),
        "film_rel_err_full_resolution_batched": err(film[:per_point], ref),
        "film_rel_err_full_resolution_per_point": err(pf, ref),
        "error_reference": f"the first {per_point} points at 16384 spp (another seed); film errors on 64 time "
                           "bins of 19.2 cm (at the film's 3 mm bins each bin holds a few samples at 1024 spp)"}
    del s, film, steady, ref, pf, ps
    # adjoint vs finite differences on the differentiable scene, 32 parameters
    sc = scenes.diff_scene()
    f = scenes.DIFF_FILM
    s = api.Scene(sc)
    autotune.apply(s, "backward", sc, f, 64, 8)
    autotune.apply(s, "render", sc, f, 64, 8)
    spp, depth = 64, 8
    alb0 = torch.from_numpy(sc.albedo).cuda()
    s.set_params(albedo=torch.from_numpy(scenes.perturbed_albedo(sc)).cuda())
    target, _ = api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, spp, 7, depth)
    target = target.clone()
    s.set_params(albedo=alb0)
    film, steady = api.new_film(f.H, f.W, f.T)

    def loss():
        api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, spp, 1, depth, out=(film, steady))
        return float(((film.double() - target.double()) ** 2).sum())

    L0 = loss()
    g = (2 * (film - target)).contiguous()
    outg = (torch.zeros((sc.n_tris, 3), device="cuda"), torch.zeros((len(sc.emitters), 3), device="cuda"),
            torch.zeros(1, device="cuda"))
    api.render_backward(s, f.T, f.start_opl, f.bin_width, spp, 1, depth, g, out=outg)
    torch.cuda.synchronize()
    outg[0].zero_()
    e0.record()
    api.render_backward(s, f.T, f.start_opl, f.bin_width, spp, 1, depth, g, out=outg)
    e1.record()
    torch.cuda.synchronize()
    adj_ms = e0.elapsed_time(e1)
    ga = outg[0].cpu().numpy()
    rng = np.random.default_rng(3)
    # parameters the loss depends on noticeably
    cand = np.argsort(-np.abs(ga).reshape(-1))[:2000]
    pick = rng.choice(cand, 32, replace=False)
    h = 1e-3
    fd = []
    e0.record()
    for k in pick:
        t, c = divmod(int(k), 3)
        vals = []
        for sgn in (1, -1):
            a = alb0.clone()
            a[t, c] += sgn * h
            s.set_params(albedo=a)
            vals.append(loss())
        fd.append((vals[0] - vals[1]) / (2 * h))
    e1.record()
    torch.cuda.synchronize()
    s.set_params(albedo=alb0)
    fd_ms = e0.elapsed_time(e1)
    adj = ga.reshape(-1)[pick]
    fd = np.array(fd)
    rel = np.abs(adj - fd) / np.maximum(np.abs(fd), 1e-30)
    out["adjoint_vs_finite_differences"] = {
        "workload": "97k-triangle scene, 256x256x512 film, 64 spp, depth 8, L2 loss vs a target with albedos "
                    "x U[0.8,1.2]; finite differences: step 1e-3, common random numbers, 32 parameters",
        "adjoint_ms_all_params": adj_ms, "n_params_adjoint": int(sc.n_tris * 3),
        "fd_ms_32_params": fd_ms, "fd_launches": 64, "loss": L0,
        "adjoint_vs_fd_rel_err_median": float(np.median(rel)), "adjoint_vs_fd_rel_err_max": float(rel.max()),
        "speedup_per_param": (fd_ms / 32) / (adj_ms / (sc.n_tris * 3)),
        "speedup_for_32_params": fd_ms / adj_ms}
    return out


def compare():
    """The comparisons of the default run with the per-point loop over all 4096 points."""
    from paper_2510_25660_gb300 import api, autotune, scenes
    from paper_2510_25660_gb300 import build as b
    b.build()
    api.load()
    print(json.dumps(comparisons(api, autotune, scenes, per_point=4096)), flush=True)


def _timed(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def secondary(api, autotune, scenes):
    """Throughput of the other workloads: backward grads/s on the differentiable
    scene, batched NLOS, the Cornell box and participating-media forward renders,
    the media backward pass and the frequency-space (phasor) film."""
    import torch
    out = {}
    # Cornell box: 64x64, T=256, 16 spp, depth 4 (65,536 paths)
    sc = scenes.cornell_box()
    f = scenes.CORNELL_FILM
    s = api.Scene(sc)
    film, steady = api.new_film(f.H, f.W, f.T)
    ms = _timed(lambda: api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, 16, 1, 4, out=(film, steady)), 20)
    s.read_counters(reset=True)
    api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, 16, 1, 4, out=(film, steady))
    c = s.read_counters(reset=True)
    out["cornell"] = {"vertices_per_s": c["vertices"] / (ms / 1000.0), "ms_per_render": ms,
                      "workload": "36-triangle Cornell box, 64x64 px, T=256 x 0.01 m, 16 spp, max_depth 4"}
    del s, film, steady
    # participating media: Cornell box + 128^3 heterogeneous medium, 256x256, T=1024, 128 spp, depth 16
    sc = scenes.media_scene()
    f = scenes.MEDIA_FILM
    s = api.Scene(sc)
    autotune.apply(s, "render", sc, f, 128, 16)   # the wavefront form (482 -> 59 ms measured)
    film, steady = api.new_film(f.H, f.W, f.T)
    ms = _timed(lambda: api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, 128, 1, 16, out=(film, steady)), 3)
    s.read_counters(reset=True)
    api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, 128, 1, 16, out=(film, steady))
    c = s.read_counters(reset=True)
    g = torch.randn_like(film)
    outg = (torch.zeros((sc.n_tris, 3), device="cuda"), torch.zeros((len(sc.emitters), 3), device="cuda"),
            torch.zeros(1, device="cuda"))
    autotune.apply(s, "backward", sc, f, 128, 16)
    bms = _timed(lambda: api.render_backward(s, f.T, f.start_opl, f.bin_width, 128, 1, 16, g, out=outg), 3)
    s.read_counters(reset=True)
    api.render_backward(s, f.T, f.start_opl, f.bin_width, 128, 1, 16, g, out=outg)
    cb = s.read_counters(reset=True)
    s.sync()
    out["media"] = {"vertices_per_s": c["vertices"] / (ms / 1000.0), "ms_per_render": ms,
                    "backward_vertices_per_s": cb["vertices"] / (bms / 1000.0), "ms_per_backward": bms,
                    "workload": "Cornell box in a 128^3 heterogeneous medium (sigma_t 0.1-2 /m, albedo 0.9, HG 0.3), "
                                "256x256 px, T=1024 x 0.005 m, 128 spp, max_depth 16; backward = surface and "
                                "medium albedo gradients"}
    del s, film, steady, g
    # frequency-space film of the benchmark frame: 4 wavelengths instead of 2048 time bins
    sc = scenes.large_scene()
    f = scenes.LARGE_FILM
    s = api.Scene(sc)
    # the benchmark frame with scattering delays on every surface (Exp, mean 0-5 cm per triangle)
    # and a Gaussian source pulse (mean 3 cm, deviation 1 cm), benchmark launch configuration
    autotune.apply(s, "render", sc, f, 256, 8)
    tau = torch.rand(sc.n_tris, device="cuda", generator=torch.Generator("cuda").manual_seed(7)) * 0.05
    s.set_delays(tau)
    s.set_pulse(api.MT_PULSE_GAUSSIAN, 0.03, 0.01)
    film, steady = api.new_film(f.H, f.W, f.T)
    ms = _timed(lambda: api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, 256, 1, 8, out=(film, steady)), 3)
    s.read_counters(reset=True)
    api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, 256, 1, 8, out=(film, steady))
    c = s.read_counters(reset=True)
    s.sync()
    out["delays"] = {"vertices_per_s": c["vertices"] / (ms / 1000.0), "ms_per_render": ms,
                     "workload": "benchmark frame with per-triangle exponential scattering delays (mean U[0, 5 cm]) "
                                 "and a Gaussian emission pulse (3 cm, 1 cm)"}
    s.set_delays(None)
    s.set_pulse(api.MT_PULSE_DELTA)
    del film, steady
    lam = [0.4, 0.2, 0.1, 0.05]
    ms = _timed(lambda: api.render_phasor(s, f.H, f.W, lam, 256, 1, 8), 3)
    s.read_counters(reset=True)
    api.render_phasor(s, f.H, f.W, lam, 256, 1, 8)
    c = s.read_counters(reset=True)
    s.sync()
    # transient polarization of the benchmark frame at 64 spp (Stokes film [512][512][2048][4][3] would be
    # 25.8 GB; T = 512 bins x 0.02 m keeps it at 6.4 GB)
    pf, pst = (torch.empty((f.H, f.W, 512, 4, 3), device="cuda"), torch.empty((f.H, f.W, 4, 3), device="cuda"))
    pms = _timed(lambda: api.render_polarized(s, f.H, f.W, 512, f.start_opl, 0.02, 64, 1, 8, out=(pf, pst)), 2)
    s.read_counters(reset=True)
    api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, 64, 1, 8)
    cp = s.read_counters(reset=True)
    s.sync()
    out["polarized"] = {"vertices_per_s": cp["vertices"] / (pms / 1000.0), "ms_per_render": pms,
                        "workload": "large static scene, 512x512 px, 64 spp, max_depth 8, Stokes film "
                                    "[512][512][512 bins x 0.02 m][4][3] (vertices counted by the scalar render "
                                    "of the same paths)"}
    del pf, pst
    out["phasor"] = {"vertices_per_s": c["vertices"] / (ms / 1000.0), "ms_per_render": ms,
                     "workload": "large static scene, 512x512 px, 256 spp, max_depth 8, K=4 wavelengths "
                                 "(0.4, 0.2, 0.1, 0.05 m), phasor film [H][W][K][2][3], benchmark launch "
                                 "configuration"}
    del s
    # backward: 97k-triangle scene, 256x256x512 film, 64 spp, depth 8
    sc = scenes.diff_scene()
    f = scenes.DIFF_FILM
    s = api.Scene(sc)
    autotune.apply(s, "backward", sc, f, 64, 8)
    autotune.apply(s, "render", sc, f, 64, 8)
    film, steady = api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, 64, 1, 8)
    g = torch.randn_like(film)
    gs = torch.randn_like(steady)
    outg = (torch.zeros((sc.n_tris, 3), device="cuda"), torch.zeros((len(sc.emitters), 3), device="cuda"),
            torch.zeros(1, device="cuda"))
    for _ in range(2):
        api.render_backward(s, f.T, f.start_opl, f.bin_width, 64, 1, 8, g, gs, out=outg)
    s.sync()
    s.read_counters(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        api.render_backward(s, f.T, f.start_opl, f.bin_width, 64, 1, 8, g, gs, out=outg)
    e1.record()
    s.sync()
    c = s.read_counters(reset=True)
    ms = e0.elapsed_time(e1) / 3
    fwd0, fwd1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fwd0.record()
    for _ in range(3):
        api.render(s, f.H, f.W, f.T, f.start_opl, f.bin_width, 64, 1, 8, out=(film, steady))
    fwd1.record()
    s.sync()
    out["backward"] = {"grads_per_s": c["vertices"] / 3 / (ms / 1000.0), "unit": "adjoint path vertices/s",
                       "ms_per_backward": ms, "forward_ms": fwd0.elapsed_time(fwd1) / 3,
                       "params_per_s": sc.n_tris * 3 / (ms / 1000.0),
                       "workload": "97k-triangle scene, 256x256x512 film, 64 spp, max_depth 8"}
    # forward-mode derivative film on the same scene and paths (tangent over every albedo)
    dalb = torch.randn((sc.n_tris, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    tfilm, tsteady = api.new_film(f.H, f.W, f.T)
    tms = _timed(lambda: api.render_tangent(s, f.H, f.W, f.T, f.start_opl, f.bin_width, 64, 1, 8, dalb, None,
                                            out=(tfilm, tsteady)), 3)
    s.sync()
    out["tangent"] = {"vertices_per_s": c["vertices"] / 3 / (tms / 1000.0), "ms_per_tangent": tms,
                      "workload": "97k-triangle scene, 256x256x512 film, 64 spp, max_depth 8, one tangent "
                                  "direction over all albedos (forward mode)"}
    del tfilm, tsteady
    del s
    # NLOS confocal 64x64 x 1024 spp, T=4096
    sc = scenes.nlos_scene()
    s = api.Scene(sc)
    lasers = torch.from_numpy(scenes.wall_grid(64, 64)).cuda()
    autotune.apply(s, "nlos", sc, None, 1024, 0)
    nf = None
    for _ in range(2):
        nf = api.render_nlos(s, lasers, None, api.MT_CONFOCAL, scenes.NLOS_T, scenes.NLOS_START, scenes.NLOS_W,
                             1024, 1, out=nf)
    s.sync()
    e0.record()
    for _ in range(5):
        nf = api.render_nlos(s, lasers, None, api.MT_CONFOCAL, scenes.NLOS_T, scenes.NLOS_START, scenes.NLOS_W,
                             1024, 1, out=nf)
    e1.record()
    s.sync()
    ms = e0.elapsed_time(e1) / 5
    out["nlos"] = {"confocal_connections_per_s": 4096 * 1024 / (ms / 1000.0), "ms_per_capture": ms,
                   "workload": "64x64 confocal grid x 1024 spp, T=4096 x 0.003 m, 49.4k hidden triangles, "
                               "one graph launch"}
    del nf
    # exhaustive grid: 16x16 lasers x 64x64 sensors, 1024 hidden samples per laser shared by its sensors
    las = torch.from_numpy(scenes.wall_grid(16, 16)).cuda()
    sen = torch.from_numpy(scenes.wall_grid(64, 64)).cuda()
    ef = (torch.empty((256 * 4096, scenes.NLOS_T), device="cuda"), torch.empty(256 * 4096, device="cuda"))
    api.render_nlos(s, las, sen, api.MT_EXHAUSTIVE, scenes.NLOS_T, scenes.NLOS_START, scenes.NLOS_W, 1024, 1, out=ef)
    s.sync()
    e0.record()
    api.render_nlos(s, las, sen, api.MT_EXHAUSTIVE, scenes.NLOS_T, scenes.NLOS_START, scenes.NLOS_W, 1024, 1, out=ef)
    e1.record()
    s.sync()
    ms = e0.elapsed_time(e1)
    out["nlos"]["exhaustive_connections_per_s"] = 256 * 4096 * 1024 / (ms / 1000.0)
    out["nlos"]["exhaustive_ms"] = ms
    out["nlos"]["exhaustive_workload"] = ("16x16 lasers x 64x64 sensors x 1024 shared hidden samples per laser, "
                                          "film 1,048,576 x 4096 (17.2 GB)")
    del ef
    return out


if __name__ == "__main__":
    main()
