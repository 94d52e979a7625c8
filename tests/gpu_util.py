"""Helpers for the GPU parity tests: load the CUDA path and compare it with the oracle."""
import os

import numpy as np

# (test id, matched records, divergent records, values off by more than rel, bin mismatches)
# of every per-contribution comparison in this session; printed at the end of the run
PARITY = []


def build_and_load():
    from paper_2510_25660_gb300 import build as b
    b.build()
    from paper_2510_25660_gb300 import api
    api.load()
    return api


def match_contribs(gpu, ora, rel=1e-4, start=None, width=None, edge=1e-5):
    """Match per-contribution records by (pixel, sample, depth, kind) and
    compare values; records present on one side only count as divergent.
    Returns (n_matched, n_divergent, worst relative error, values off by more
    than rel, time-bin mismatches of contributions whose OPL lies more than
    `edge` metres from a bin edge, |OPL differences|)."""
    def key(r):
        return (r["pixel"].astype(np.int64) << 32) | (r["sample"].astype(np.int64) << 12) | \
               (r["depth"].astype(np.int64) << 2) | r["kind"].astype(np.int64)

    kg, ko = key(gpu), key(ora)
    assert len(np.unique(kg)) == len(kg), "duplicate GPU records"
    assert len(np.unique(ko)) == len(ko), "duplicate oracle records"
    common, ig, io = np.intersect1d(kg, ko, return_indices=True)
    div = len(kg) + len(ko) - 2 * len(common)
    g, o = gpu[ig], ora[io]
    same_tri = g["tri"] == o["tri"]
    div += int((~same_tri).sum())
    g, o = g[same_tri], o[same_tri]
    cg = g["c"].astype(np.float64)
    co = o["c"]
    scale = np.maximum(np.abs(co).max(axis=1, keepdims=True), 1e-30)
    err = np.abs(cg - co) / scale
    worst = float(err.max()) if len(err) else 0.0
    bad_val = int((err.max(axis=1) > rel).sum()) if len(err) else 0
    # time bins must agree unless a bin edge lies within `edge` metres of the
    # span between the two OPLs (FP32 OPL error grows along a path)
    assert start is not None and width is not None
    dopl = np.abs(g["opl"].astype(np.float64) - o["opl"])
    x = (o["opl"] - start) / width
    away = np.abs(x - np.round(x)) * width > dopl + edge
    bin_bad = int(((g["bin"] != o["bin"]) & away).sum())
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    PARITY.append((test, len(common), div, bad_val, bin_bad, worst))
    return len(common), div, worst, bad_val, bin_bad, dopl


def divergent_pixels(gpu, ora, rel=1e-4):
    """Pixels with a contribution on one side only, a different triangle, a
    value off by more than rel, or a different time bin (allowed only within
    FP32 rounding of a bin edge, which match_contribs checks): the pixels whose
    films may legitimately differ by more than rounding."""
    def key(r):
        return (r["pixel"].astype(np.int64) << 32) | (r["sample"].astype(np.int64) << 12) | \
               (r["depth"].astype(np.int64) << 2) | r["kind"].astype(np.int64)

    kg, ko = key(gpu), key(ora)
    common, ig, io = np.intersect1d(kg, ko, return_indices=True)
    only = np.setxor1d(kg, ko)
    px = set((only >> 32).tolist())
    g, o = gpu[ig], ora[io]
    scale = np.maximum(np.abs(o["c"]).max(axis=1), 1e-30)
    off = (g["tri"] != o["tri"]) | (g["bin"] != o["bin"]) | \
        (np.abs(g["c"].astype(np.float64) - o["c"]).max(axis=1) / scale > rel)
    px |= set(g["pixel"][off].tolist())
    return px


def rel_l2(a, b, mask=None):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
