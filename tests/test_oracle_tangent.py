"""Pins of the oracle's forward-mode derivative (Sec. 4.4, forward mode: the
film of dI/dpi for one direction in parameter space).

Reading: parameters are per-triangle albedos, emitter radiances and the medium
albedo; with colour-independent sampling and no Russian roulette a contribution
is a polynomial in the albedos and linear in the radiance for fixed random
numbers, so central differences with common random numbers are exact up to
O(h^2) and forward mode must equal reverse mode transposed."""
import numpy as np
import pytest

KW = dict(spp=4, seed=13, max_depth=4)
CROP = (26, 38, 26, 38)
H = W = 64
T, START, WIDTH = 96, 3.5, 0.03


@pytest.fixture(scope="module")
def cornell(oracle_mod, scenes_mod):
    sc = scenes_mod.cornell_box()
    return sc, oracle_mod.OracleScene(sc)


def _dirs(sc, seed):
    rng = np.random.default_rng(seed)
    dalb = rng.normal(size=(sc.n_tris, 3))
    drad = rng.normal(size=(len(sc.emitters), 3))
    return dalb, drad


def test_tangent_equals_central_differences(cornell):
    sc, osc = cornell
    dalb, drad = _dirs(sc, 1)
    t = osc.render_tangent(H, W, T, START, WIDTH, dalb=dalb, drad=drad, crop=CROP, **KW)
    alb0 = sc.albedo.astype(np.float64)
    rad0 = np.array([e["radiance"] for e in sc.emitters], np.float64)
    h = 1e-3
    films = []
    for sgn in (1, -1):
        osc.set_params(albedo=alb0 + sgn * h * dalb, radiance=rad0 + sgn * h * drad)
        films.append(osc.render(H, W, T, START, WIDTH, crop=CROP, **KW))
    osc.set_params(albedo=alb0, radiance=rad0)
    fd = (films[0]["film"] - films[1]["film"]) / (2 * h)
    fds = (films[0]["steady"] - films[1]["steady"]) / (2 * h)
    scale = np.abs(t["film"]).max()
    assert scale > 0
    assert np.abs(t["film"] - fd).max() < 1e-5 * scale
    assert np.abs(t["steady"] - fds).max() < 1e-5 * np.abs(t["steady"]).max()


def test_tangent_is_the_transposed_adjoint(cornell):
    """<g, J dtheta> = <J^T g, dtheta> for random g and dtheta."""
    sc, osc = cornell
    dalb, drad = _dirs(sc, 2)
    rng = np.random.default_rng(3)
    g = rng.normal(size=(CROP[3] - CROP[2], CROP[1] - CROP[0], T, 3))
    gs = rng.normal(size=(CROP[3] - CROP[2], CROP[1] - CROP[0], 3))
    t = osc.render_tangent(H, W, T, START, WIDTH, dalb=dalb, drad=drad, crop=CROP, **KW)
    b = osc.render_backward(H, W, T, START, WIDTH, grad_film=g, grad_steady=gs, crop=CROP, **KW)
    lhs = (g * t["film"]).sum() + (gs * t["steady"]).sum()
    rhs = (b["albedo"] * dalb).sum() + (b["radiance"] * drad).sum()
    assert lhs == pytest.approx(rhs, rel=1e-10)


def test_tangent_homogeneity_closed_forms(cornell, oracle_mod):
    """Scaling every radiance (drad = L_e) gives the film itself (C is linear
    in L_e); scaling every Lambertian albedo (dalb = albedo) multiplies each
    contribution by its number of surface vertices (C is homogeneous of that
    degree), which the per-contribution dump gives independently."""
    sc, osc = cornell
    assert np.all(sc.mtype == 0)  # all Lambertian
    rad0 = np.array([e["radiance"] for e in sc.emitters], np.float64)
    base = osc.render(H, W, T, START, WIDTH, crop=CROP, dump_cap=500000, **KW)
    t = osc.render_tangent(H, W, T, START, WIDTH, drad=rad0, crop=CROP, **KW)
    assert np.allclose(t["film"], base["film"], rtol=1e-12, atol=1e-15)
    t2 = osc.render_tangent(H, W, T, START, WIDTH, dalb=sc.albedo.astype(np.float64), crop=CROP, **KW)
    d = base["dump"]
    nv = np.where(d["kind"] == 1, d["depth"], d["depth"] - 1)
    expect = np.zeros_like(base["film"])
    inb = (d["bin"] >= 0) & (d["bin"] < T)
    py = d["pixel"] // W - CROP[2]
    px = d["pixel"] % W - CROP[0]
    np.add.at(expect, (py[inb], px[inb], d["bin"][inb]), (nv[inb, None] * d["c"][inb]) / KW["spp"])
    assert np.allclose(t2["film"], expect, rtol=1e-10, atol=1e-14)


def test_tangent_medium_albedo(oracle_mod, scenes_mod):
    """Medium albedo direction against central differences in a heterogeneous medium."""
    sc = scenes_mod.media_scene(res=16)
    osc = oracle_mod.OracleScene(sc)
    kw = dict(spp=2, seed=4, max_depth=6, crop=(28, 36, 28, 36))
    t = osc.render_tangent(64, 64, 64, 3.5, 0.05, dmed=1.0, **kw)
    a0 = sc.medium["albedo"]
    h = 1e-4
    osc.set_params(medium_albedo=a0 + h)
    fp = osc.render(64, 64, 64, 3.5, 0.05, **kw)["film"]
    osc.set_params(medium_albedo=a0 - h)
    fm = osc.render(64, 64, 64, 3.5, 0.05, **kw)["film"]
    osc.set_params(medium_albedo=a0)
    fd = (fp - fm) / (2 * h)
    assert np.abs(t["film"]).max() > 0
    assert np.abs(t["film"] - fd).max() < 1e-5 * np.abs(t["film"]).max()
