"""Pins of the oracle's participating-media transport (Sec. 4.1, tof inside
media per Eq. 3 with eta = 1): trilinear density lookup, Beer-Lambert
transmittance of a directly seen emitter, delta and ratio tracking against the
ray-marched optical depth, and single scattering against 1-D quadrature."""
import numpy as np
import pytest


def _dummy_geometry(scenes_mod):
    # one tiny black triangle far away so the scene is not empty
    t = np.array([[[50, 50, 50], [50.01, 50, 50], [50, 50.01, 50]]], np.float32)
    return t


def test_trilinear_reproduces_linear_fields(oracle_mod, scenes_mod):
    rx, ry, rz = 4, 5, 6
    lo, hi = np.array([-1.0, -0.5, 0.0]), np.array([1.0, 1.5, 3.0])
    hs = (hi - lo) / np.array([rx, ry, rz])
    xc = lo[0] + (np.arange(rx) + 0.5) * hs[0]
    yc = lo[1] + (np.arange(ry) + 0.5) * hs[1]
    zc = lo[2] + (np.arange(rz) + 0.5) * hs[2]
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    f = lambda x, y, z: 0.7 + 0.3 * x - 0.2 * y + 0.1 * z
    dens = f(X, Y, Z).astype(np.float32)
    sc = scenes_mod.cornell_box()
    sc.medium = dict(lo=tuple(lo), hi=tuple(hi), density=dens, albedo=0.9, g=0.0)
    osc = oracle_mod.OracleScene(sc)
    rng = np.random.default_rng(0)
    for _ in range(200):
        p = rng.uniform(lo + hs / 2, hi - hs / 2)
        assert abs(osc.density(p) - f(*p)) < 1e-6  # grid values are float32
    assert abs(osc.majorant() - dens.max()) == 0


def test_beer_lambert_direct_view(oracle_mod, scenes_mod):
    sigma, Le = 0.8, 3.0
    em = scenes_mod.quad((-2, -2, -0.5), (2, -2, -0.5), (2, 2, -0.5), (-2, 2, -0.5))  # normal +z
    tris = em.astype(np.float32)
    sc = scenes_mod.Scene(tris, np.zeros((2, 3), np.float32), np.zeros(2, np.float32), np.zeros(2, np.uint32),
                          [dict(type=0, first_tri=0, n_tris=2, radiance=(Le,) * 3, position=(0, 0, 0))],
                          dict(origin=(0, 0, 3.5), target=(0, 0, 0), up=(0, 1, 0), fov_x_deg=10.0))
    sc.medium = scenes_mod.homogeneous_medium(sigma, albedo=0.0)
    osc = oracle_mod.OracleScene(sc)
    N = 6000
    T, start, width = 200, 3.5, 0.01
    out = osc.render(2, 2, T, start, width, spp=N, seed=99, max_depth=1, flags=oracle_mod.PIXEL_CENTER)
    for py in range(2):
        for px in range(2):
            o, d = osc.camera_ray(2, 2, px, py)
            path_in = 1.5 / abs(d[2])
            p = np.exp(-sigma * path_in)
            est = out["steady"][py, px, 0] / Le
            assert abs(est - p) < 4 * np.sqrt(p * (1 - p) / N), (est, p)
            opl = 4.0 / abs(d[2])
            assert out["film"][py, px, int(np.floor((opl - start) / width)), 0] == out["steady"][py, px, 0]


def test_tracking_matches_optical_depth(oracle_mod, scenes_mod):
    sc = scenes_mod.media_scene(res=32)
    osc = oracle_mod.OracleScene(sc)
    rng = np.random.default_rng(5)
    for k in range(3):
        o = rng.uniform(-0.9, 0.9, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        dist = 1.2
        ts = (np.arange(4000) + 0.5) / 4000 * dist
        inside = lambda p: bool(np.all(np.abs(p) <= 1.0))
        tau = sum(osc.density(o + t * d) for t in ts if inside(o + t * d)) * dist / 4000
        Tx = np.exp(-tau)
        N = 4000
        ratio = np.array([osc.track(o, d, dist, 1234 + k, i, 7, 0) for i in range(N)])
        delta = np.array([osc.track(o, d, dist, 1234 + k, i, 7, 1) for i in range(N)])
        assert abs(ratio.mean() - Tx) < 4 * ratio.std() / np.sqrt(N) + 1e-4, (ratio.mean(), Tx)
        assert abs(delta.mean() - Tx) < 4 * np.sqrt(Tx * (1 - Tx) / N), (delta.mean(), Tx)


def test_single_scatter_matches_quadrature(oracle_mod, scenes_mod):
    sigma, alb, g, I = 0.6, 0.9, 0.3, 2.0
    light = np.array([0.0, 0.3, 0.0])
    tris = _dummy_geometry(scenes_mod)
    sc = scenes_mod.Scene(tris, np.zeros((1, 3), np.float32), np.zeros(1, np.float32), np.zeros(1, np.uint32),
                          [dict(type=1, first_tri=0, n_tris=0, radiance=(I,) * 3, position=tuple(light))],
                          dict(origin=(0, 0, 3.5), target=(0, 0, 0), up=(0, 1, 0), fov_x_deg=20.0))
    sc.medium = scenes_mod.homogeneous_medium(sigma, albedo=alb, g=g)
    osc = oracle_mod.OracleScene(sc)
    N = 20000
    T, start, width = 40, 3.0, 0.1
    out = osc.render(2, 2, T, start, width, spp=N, seed=4, max_depth=2, flags=oracle_mod.PIXEL_CENTER)
    for py in range(2):
        for px in range(2):
            o, d = osc.camera_ray(2, 2, px, py)
            a = (1.0 - o[2]) / d[2]
            b = (-1.0 - o[2]) / d[2]
            # exits through the box side if earlier
            for ax in (0, 1):
                if d[ax] != 0:
                    tb = ((1.0 if d[ax] > 0 else -1.0) - o[ax]) / d[ax]
                    b = min(b, tb)
            n = 20000
            t = a + (np.arange(n) + 0.5) / n * (b - a)
            x = o + t[:, None] * d
            v = light - x
            r = np.linalg.norm(v, axis=1)
            cos = (v @ d) / r
            ph = (1 - g * g) / (4 * np.pi * (1 + g * g - 2 * g * cos) ** 1.5)
            f = sigma * np.exp(-sigma * (t - a)) * alb * ph * I * np.exp(-sigma * r) / r ** 2
            ref = f.sum() * (b - a) / n
            est = out["steady"][py, px, 0]
            assert abs(est - ref) < 0.04 * ref, (est, ref)
            opl = t + r
            hist = np.bincount(np.clip(np.floor((opl - start) / width).astype(int), 0, T - 1),
                               weights=f * (b - a) / n, minlength=T)
            big = hist > 0.1 * hist.max()
            assert np.all(np.abs(out["film"][py, px, big, 0] - hist[big]) < 0.15 * hist[big])
