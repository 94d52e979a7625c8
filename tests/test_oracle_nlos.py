"""Pins of the oracle's relay-wall NLOS estimator (Sec. 4.5): the impulse
response H(x_l, x_s, t) of a small hidden patch against brute-force quadrature
of the third-bounce transport integral, exact reciprocity under swapping laser
and sensor, and occlusion."""
import numpy as np
import pytest


def _patch_scene(scenes_mod, r=0.5, a=0.05, albedo=0.5, blocker=False):
    wall = scenes_mod.quad((-0.5, -0.5, 0.0), (0.5, -0.5, 0.0), (0.5, 0.5, 0.0), (-0.5, 0.5, 0.0))
    h = a / 2
    # patch centred at (0.05, -0.03, r), facing the wall (normal -z)
    c = np.array([0.05, -0.03, r])
    patch = scenes_mod.quad(c + (-h, -h, 0), c + (-h, h, 0), c + (h, h, 0), c + (h, -h, 0))
    parts = [wall, patch]
    if blocker:
        parts.append(scenes_mod.quad((-0.2, -0.2, 0.25), (-0.2, 0.2, 0.25), (0.3, 0.2, 0.25), (0.3, -0.2, 0.25)))
    tris = np.concatenate(parts).astype(np.float32)
    n = len(tris)
    alb = np.full((n, 3), 0.8, np.float32)
    alb[2:4] = albedo
    sc = scenes_mod.Scene(tris, alb, np.zeros(n, np.float32), np.zeros(n, np.uint32), [],
                          dict(origin=(0, 0, 2), target=(0, 0, 0), up=(0, 1, 0), fov_x_deg=40),
                          hidden=(2, 2), wall=dict(center=(0, 0, 0), size=1.0, normal=(0, 0, 1), albedo=0.8))
    return sc, c, h


def _quadrature(xl, xs, c, h, rho_w=0.8, rho_h=0.5, n=300):
    """Midpoint quadrature of the third-bounce integrand over the square patch;
    returns the integral and the OPL samples with their weights."""
    g = (np.arange(n) + 0.5) / n * 2 * h - h
    X, Y = np.meshgrid(g, g, indexing="ij")
    P = np.stack([c[0] + X, c[1] + Y, np.full_like(X, c[2])], -1).reshape(-1, 3)
    dA = (2 * h / n) ** 2
    nw = np.array([0, 0, 1.0])
    ny = np.array([0, 0, -1.0])
    v1 = P - xl
    v2 = xs - P
    d1 = np.linalg.norm(v1, axis=1)
    d2 = np.linalg.norm(v2, axis=1)
    cl = v1 @ nw / d1
    cs = -(v2 @ nw) / d2
    cy1 = -(v1 @ ny) / d1
    cy2 = (v2 @ ny) / d2
    f = (rho_w / np.pi) ** 2 * (rho_h / np.pi) * cl * cs * cy1 * cy2 / (d1 ** 2 * d2 ** 2)
    return f.sum() * dA, d1 + d2, f * dA


@pytest.mark.parametrize("exhaustive", [False, True])
def test_small_patch_matches_quadrature(oracle_mod, scenes_mod, exhaustive):
    sc, c, h = _patch_scene(scenes_mod)
    osc = oracle_mod.OracleScene(sc)
    xl = np.array([[0.0, 0.0, 0.0]], np.float32)
    xs = np.array([[0.25, 0.1, 0.0]], np.float32) if exhaustive else None
    T, start, width = 4096, 0.0, 0.003
    out = osc.render_nlos(xl, xs, exhaustive, T, start, width, spp=4096, seed=17)
    ref, opl, w = _quadrature(xl[0].astype(np.float64), (xs if exhaustive else xl)[0].astype(np.float64), c, h)
    assert abs(out["steady"][0] - ref) < 2e-3 * ref, (out["steady"][0], ref)
    assert abs(out["film"][0].sum() - ref) < 2e-3 * ref
    # binned time profile: all energy where the quadrature puts it
    hist = np.bincount(np.floor((opl - start) / width).astype(int), weights=w, minlength=T)[:T]
    nz = hist > 0.05 * hist.max()
    assert np.all(out["film"][0][~(hist > 0)] == 0)
    assert np.all(np.abs(out["film"][0][nz] - hist[nz]) < 0.1 * hist[nz] + 0.01 * ref)


def test_confocal_small_patch_limit(oracle_mod, scenes_mod):
    """Tiny fronto-parallel patch straight in front of x: H -> (rho_w/pi)^2 (rho_h/pi) A / r^4 at OPL 2r."""
    r, a = 0.6, 0.01
    sc, c, h = _patch_scene(scenes_mod, r=r, a=a)
    osc = oracle_mod.OracleScene(sc)
    xl = np.array([c[:2].tolist() + [0.0]], np.float32)
    out = osc.render_nlos(xl, None, False, 1000, 0.0, 0.003, spp=1024, seed=3)
    lim = (0.8 / np.pi) ** 2 * (0.5 / np.pi) * a * a / r ** 4
    assert abs(out["steady"][0] - lim) < 2e-3 * lim
    assert out["film"][0].argmax() == int(np.floor(2 * r / 0.003))


def test_reciprocity_exact(oracle_mod, scenes_mod):
    """The third-bounce integrand is symmetric in (x_l, x_s); with the same y
    samples (laser index 0 in both calls) H(a, b, t) = H(b, a, t)."""
    sc, c, h = _patch_scene(scenes_mod, a=0.2)
    osc = oracle_mod.OracleScene(sc)
    A = np.array([[-0.3, 0.2, 0.0]], np.float32)
    B = np.array([[0.35, -0.1, 0.0]], np.float32)
    ab = osc.render_nlos(A, B, True, 2000, 0.0, 0.003, spp=512, seed=8)
    ba = osc.render_nlos(B, A, True, 2000, 0.0, 0.003, spp=512, seed=8)
    assert ab["steady"][0] > 0
    assert np.allclose(ab["film"], ba["film"], rtol=1e-10, atol=0)


def test_occluder_blocks(oracle_mod, scenes_mod):
    sc, c, h = _patch_scene(scenes_mod, blocker=True)
    osc = oracle_mod.OracleScene(sc)
    xl = np.array([[0.0, 0.0, 0.0]], np.float32)
    out = osc.render_nlos(xl, None, False, 1000, 0.0, 0.003, spp=256, seed=1)
    assert out["steady"][0] == 0.0
