"""Pins of the oracle's backward mode (Sec. 4.4, Eqs. 13-15) against central
finite differences with common random numbers.

With no Russian roulette and colour-independent sampling, every contribution
is a polynomial in the per-triangle albedos (Lambert rho, Schlick F0) and the
medium albedo, and linear in the emitter radiance, for fixed random numbers;
sampling tables stay fixed when parameters change.  Central differences with
step 1e-3 therefore match the exact gradient up to O(h^2) and rounding.
"""
import numpy as np
import pytest

H = W = 64
CROP = (24, 40, 24, 40)


def _scene(scenes_mod, ggx=True):
    sc = scenes_mod.cornell_box()
    if ggx:
        rng = np.random.default_rng(4)
        sc.mtype[10:22] = 1           # short block: GGX conductor
        sc.roughness[10:22] = 0.3
        sc.albedo[10:22] = rng.uniform(0.5, 1.0, (12, 3))
    return sc


def _loss(out, target, w_steady):
    return ((out["film"] - target) ** 2).sum() + (w_steady * out["steady"]).sum()


@pytest.mark.parametrize("ggx", [False, True])
def test_albedo_and_radiance_gradients_match_fd(oracle_mod, scenes_mod, ggx):
    sc = _scene(scenes_mod, ggx)
    osc = oracle_mod.OracleScene(sc)
    kw = dict(H=H, W=W, T=64, start=3.5, width=0.04, spp=4, seed=321, max_depth=4, crop=CROP)
    rng = np.random.default_rng(0)
    base = osc.render(**kw)
    target = base["film"] * rng.uniform(0.7, 1.3, base["film"].shape)
    w_steady = rng.uniform(-1, 1, base["steady"].shape)
    g = osc.render_backward(grad_film=2 * (base["film"] - target), grad_steady=w_steady, **kw)
    alb0 = sc.albedo.astype(np.float64).copy()
    params = [(int(t), int(c)) for t, c in zip(rng.integers(0, 34, 32), rng.integers(0, 3, 32))]
    h = 1e-3
    gmax = np.abs(g["albedo"]).max()
    checked = 0
    for t, c in params:
        vals = []
        for s in (+1, -1):
            a = alb0.copy()
            a[t, c] += s * h
            osc.set_params(albedo=a)
            vals.append(_loss(osc.render(**kw), target, w_steady))
        osc.set_params(albedo=alb0)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g["albedo"][t, c]) <= 2e-4 * max(abs(fd), 1e-3 * gmax), (t, c, fd, g["albedo"][t, c])
        checked += abs(fd) > 1e-3 * gmax
    assert checked >= 16
    rad0 = np.array([sc.emitters[0]["radiance"]], np.float64)
    for c in range(3):
        vals = []
        for s in (+1, -1):
            r = rad0.copy()
            r[0, c] += s * h
            osc.set_params(radiance=r)
            vals.append(_loss(osc.render(**kw), target, w_steady))
        osc.set_params(radiance=rad0)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g["radiance"][0, c]) <= 1e-4 * abs(fd), (c, fd, g["radiance"][0, c])


def test_gradient_of_linear_loss_is_film_derivative(oracle_mod, scenes_mod):
    """For L = <w, I>, the gradient w.r.t. the emitter radiance is exactly
    <w, I> / Le (the film is linear in the radiance of the only emitter)."""
    sc = _scene(scenes_mod, ggx=True)
    osc = oracle_mod.OracleScene(sc)
    kw = dict(H=H, W=W, T=64, start=3.5, width=0.04, spp=2, seed=5, max_depth=3, crop=CROP)
    out = osc.render(**kw)
    w = np.random.default_rng(1).uniform(0, 1, out["film"].shape)
    g = osc.render_backward(grad_film=w, **kw)
    L = (w * out["film"]).sum(axis=(0, 1, 2))
    assert np.allclose(g["radiance"][0], L / 10.0, rtol=1e-10)


def test_medium_albedo_gradient_matches_fd(oracle_mod, scenes_mod):
    sc = scenes_mod.cornell_box()
    sc.medium = scenes_mod.homogeneous_medium(0.5, albedo=0.8, g=0.3)
    osc = oracle_mod.OracleScene(sc)
    kw = dict(H=32, W=32, T=64, start=3.5, width=0.05, spp=8, seed=77, max_depth=6, crop=(8, 24, 8, 24))
    base = osc.render(**kw)
    rng = np.random.default_rng(2)
    target = base["film"] * rng.uniform(0.5, 1.5, base["film"].shape)
    g = osc.render_backward(grad_film=2 * (base["film"] - target), **kw)
    h = 1e-3
    vals = []
    for s in (+1, -1):
        osc.set_params(medium_albedo=0.8 + s * h)
        vals.append(((osc.render(**kw)["film"] - target) ** 2).sum())
    osc.set_params(medium_albedo=0.8)
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(fd) > 0
    assert abs(fd - g["medium_albedo"]) <= 1e-4 * abs(fd), (fd, g["medium_albedo"])
    # surface albedo inside the medium, two parameters
    alb0 = sc.albedo.astype(np.float64).copy()
    for t, c in ((4, 0), (21, 2)):
        vals = []
        for s in (+1, -1):
            a = alb0.copy()
            a[t, c] += s * h
            osc.set_params(albedo=a)
            vals.append(((osc.render(**kw)["film"] - target) ** 2).sum())
        osc.set_params(albedo=alb0)
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - g["albedo"][t, c]) <= 1e-4 * abs(fd) + 1e-12, (t, c, fd, g["albedo"][t, c])
