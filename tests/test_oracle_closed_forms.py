"""Pins of the oracle estimator against closed forms and invariants.

* single bounce of a point emitter on a Lambertian plane: the transient is a
  single spike of height rho I cos / (pi d1^2) at time of flight d1 + d2
  (Sec. 3: Eqs. 3-4 tof, Eq. 8 impulse response, path reuse binning);
  with camera unwarping the spike moves to d1 (Sec. 3, "Camera warp");
* the time-summed film plus what falls outside the window equals the steady
  image (Sec. 2 listing returns both; Sec. 3 path reuse);
* white furnace: inside a closed uniformly emitting enclosure of albedo rho the
  steady radiance is Le * sum_k rho^k (Eq. 9 is unbiased);
* transient furnace: one bounce inside a sphere adds a chord 2R cos(theta) with
  density l / (2 R^2) on [0, 2R]; mean chord 4V/S (Cauchy);
* MIS consistency: light-only, BSDF-only and MIS estimators agree;
* resumable rendering: two half-spp calls with a sample offset equal one call.
"""
import numpy as np
import pytest


def _plane_case(oracle_mod, scenes_mod, flags):
    sc = scenes_mod.point_light_plane(albedo=0.6, intensity=5.0, light_pos=(0.3, 1.2, -0.2))
    osc = oracle_mod.OracleScene(sc)
    H = W = 16
    T, start, width = 600, 0.0, 0.01
    r = osc.render(H, W, T, start, width, spp=1, seed=7, max_depth=2,
                   flags=oracle_mod.PIXEL_CENTER | flags, want_dropped=True)
    return sc, osc, r, (H, W, T, start, width)


@pytest.mark.parametrize("unwarp", [False, True])
def test_point_light_plane_single_bounce(oracle_mod, scenes_mod, unwarp):
    sc, osc, r, (H, W, T, start, width) = _plane_case(oracle_mod, scenes_mod, oracle_mod.UNWARP if unwarp else 0)
    rho, I = 0.6, 5.0
    p = np.array([0.3, 1.2, -0.2])
    film = r["film"]
    checked = 0
    for py in range(H):
        for px in range(W):
            o, d = osc.camera_ray(W, H, px, py)
            assert d[1] < 0
            t = -o[1] / d[1]
            x = o + t * d
            d1 = np.linalg.norm(p - x)
            cos = (p[1] - x[1]) / d1
            L = rho * I * cos / (np.pi * d1 * d1)
            opl = d1 + (0.0 if unwarp else t)
            kf = (opl - start) / width
            assert abs(r["steady"][py, px] - L).max() < 5e-4 * L
            nz = np.nonzero(film[py, px, :, 0])[0]
            assert len(nz) == 1  # a single spike: everything else is exactly zero
            if abs(kf - round(kf)) > 0.05:
                assert nz[0] == int(np.floor(kf)), (px, py, nz, kf)
                checked += 1
            assert np.allclose(film[py, px, nz[0]], L, rtol=5e-4)
    assert checked > 200
    # the 1/r^2 cosine falloff makes the pixel nearest the light the brightest
    iy, ix = np.unravel_index(np.argmax(r["steady"][..., 0]), (H, W))
    best = None
    for py in range(H):
        for px in range(W):
            o, d = osc.camera_ray(W, H, px, py)
            x = o + (-o[1] / d[1]) * d
            v = (1.2 - x[1]) / np.linalg.norm(p - x) ** 3
            if best is None or v > best[0]:
                best = (v, py, px)
    assert (iy, ix) == best[1:]


def test_tsum_equals_steady_cornell(oracle_mod, scenes_mod):
    sc = scenes_mod.cornell_box()
    osc = oracle_mod.OracleScene(sc)
    f = scenes_mod.CORNELL_FILM
    r = osc.render(f.H, f.W, f.T, f.start_opl, f.bin_width, spp=4, seed=25660, max_depth=4,
                   crop=(16, 48, 16, 48), want_dropped=True)
    lhs = r["film"].sum(2) + r["dropped"]
    assert np.allclose(lhs, r["steady"], rtol=1e-12, atol=1e-14)
    assert r["film"].sum() > 0 and r["dropped"].sum() > 0


def test_white_furnace_steady(oracle_mod, scenes_mod):
    rho, Le, D = 0.5, 1.0, 4
    sc = scenes_mod.furnace_sphere(level=3, radius=1.0, albedo=rho, radiance=Le)
    osc = oracle_mod.OracleScene(sc)
    r = osc.render(8, 8, 16, 0.0, 1.0, spp=256, seed=3, max_depth=D)
    expect = Le * sum(rho ** k for k in range(D))
    s = r["steady"][..., 0].reshape(-1)
    se = s.std() / np.sqrt(len(s))
    assert abs(s.mean() - expect) < max(4 * se, 2e-3 * expect), (s.mean(), expect, se)
    assert np.allclose(r["steady"][..., 0], r["steady"][..., 1])


def test_transient_furnace_chord_distribution(oracle_mod, scenes_mod):
    """Energy of one-bounce paths is rho Le spread over OPL = R + l with
    density l / (2 R^2) on [0, 2R] (chord of a cosine-distributed direction in a
    sphere); its mean increment is 4R/3 = 4V/S."""
    R, rho, Le = 1.0, 0.5, 1.0
    sc = scenes_mod.furnace_sphere(level=5, radius=R, albedo=rho, radiance=Le)
    osc = oracle_mod.OracleScene(sc)
    T, start, width = 25, 0.9, 0.1
    kw = dict(spp=256, seed=11)
    r2 = osc.render(6, 6, T, start, width, max_depth=2, **kw)
    r1 = osc.render(6, 6, T, start, width, max_depth=1, **kw)
    h = (r2["film"] - r1["film"])[..., 0].mean((0, 1))  # one-bounce energy per bin
    edges = start + width * np.arange(T + 1)
    l = np.clip(edges - R, 0.0, 2 * R)
    expect = rho * Le * np.diff(l ** 2 / (4 * R * R))
    assert abs(h.sum() - rho * Le) < 0.01 * rho * Le
    big = expect > 0.02 * rho * Le
    assert np.all(np.abs(h[big] - expect[big]) < 0.06 * expect[big] + 2e-3), np.c_[h, expect]
    centers = edges[:-1] + width / 2
    mean_inc = (h * (centers - R)).sum() / h.sum()
    assert abs(mean_inc - 4 * R / 3) < 0.03, mean_inc


def test_mis_consistency(oracle_mod, scenes_mod):
    sc = scenes_mod.cornell_box()
    osc = oracle_mod.OracleScene(sc)
    f = scenes_mod.CORNELL_FILM
    out = {}
    for name, strat in (("mis", oracle_mod.STRAT_MIS), ("nee", oracle_mod.STRAT_NEE_ONLY),
                        ("bsdf", oracle_mod.STRAT_BSDF_ONLY)):
        r = osc.render(f.H, f.W, 32, 3.5, 0.1, spp=48, seed=5, max_depth=3, crop=(12, 52, 12, 52), strategy=strat)
        s = r["steady"].sum(-1).reshape(-1)
        t = r["film"].sum((0, 1, 3))
        out[name] = (s.mean(), s.std() / np.sqrt(len(s)), t)
    m, sm, tm = out["mis"]
    for other in ("nee", "bsdf"):
        o, so, to = out[other]
        assert abs(m - o) < 4.5 * np.sqrt(sm ** 2 + so ** 2), (other, m, o, sm, so)
    # the time profiles agree too (coarse 10 cm bins)
    tm_n, tn_n = out["mis"][2], out["nee"][2]
    big = tm_n > 0.05 * tm_n.max()
    assert np.all(np.abs(tm_n[big] - tn_n[big]) < 0.1 * tm_n[big])


def test_resume_with_sample_offset(oracle_mod, scenes_mod):
    sc = scenes_mod.cornell_box()
    osc = oracle_mod.OracleScene(sc)
    kw = dict(H=64, W=64, T=256, start=3.5, width=0.01, seed=9, max_depth=4, crop=(20, 28, 20, 28))
    full = osc.render(spp=8, flags=oracle_mod.ACCUMULATE, **kw)
    a = osc.render(spp=3, flags=oracle_mod.ACCUMULATE, **kw)
    b = osc.render(spp=5, flags=oracle_mod.ACCUMULATE, sample_offset=3, **kw)
    assert np.array_equal(a["film"] + b["film"], full["film"]) or np.allclose(a["film"] + b["film"], full["film"], rtol=1e-13, atol=1e-15)
    norm = osc.render(spp=8, **kw)
    assert np.allclose(norm["film"] * 8, full["film"], rtol=1e-13, atol=1e-15)


def test_max_depth_one_is_direct_view_only(oracle_mod, scenes_mod):
    sc = scenes_mod.cornell_box()
    osc = oracle_mod.OracleScene(sc)
    r = osc.render(64, 64, 256, 3.5, 0.01, spp=2, seed=1, max_depth=1, dump_cap=100000)
    d = r["dump"]
    assert len(d) > 0 and np.all(d["depth"] == 1) and np.all(d["kind"] == 0)
    assert np.all(np.isin(d["tri"], [34, 35]))
    assert np.allclose(d["c"], 10.0)
