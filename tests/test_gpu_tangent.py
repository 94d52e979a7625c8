"""GPU forward-mode derivative (Sec. 4.4, forward mode) against the oracle on
the same Philox stream, against the GPU's own reverse mode (transpose
identity) and against central differences of the GPU forward render."""
import numpy as np
import pytest

from gpu_util import build_and_load, rel_l2

pytestmark = pytest.mark.gpu

H = W = 64
T, START, WIDTH = 128, 3.5, 0.02
SPP, SEED, DEPTH = 8, 31, 4


@pytest.fixture(scope="module")
def cornell(oracle_mod, scenes_mod):
    api = build_and_load()
    sc = scenes_mod.cornell_box()
    rng = np.random.default_rng(6)
    dalb = rng.normal(size=(sc.n_tris, 3)).astype(np.float32)
    drad = rng.normal(size=(len(sc.emitters), 3)).astype(np.float32)
    return api, sc, api.Scene(sc), oracle_mod.OracleScene(sc), dalb, drad


def test_tangent_matches_oracle(cornell):
    import torch
    api, sc, s, osc, dalb, drad = cornell
    tf, ts = api.render_tangent(s, H, W, T, START, WIDTH, SPP, SEED, DEPTH, torch.from_numpy(dalb).cuda(),
                                torch.from_numpy(drad).cuda())
    s.sync()
    crop = (24, 40, 24, 40)
    ref = osc.render_tangent(H, W, T, START, WIDTH, SPP, SEED, DEPTH, dalb=dalb, drad=drad, crop=crop)
    g = tf.cpu().numpy()[24:40, 24:40]
    assert np.abs(ref["film"]).max() > 0
    assert rel_l2(g, ref["film"]) < 2e-3
    assert rel_l2(ts.cpu().numpy()[24:40, 24:40], ref["steady"]) < 1e-3


def test_tangent_is_transposed_backward_on_gpu(cornell):
    import torch
    api, sc, s, osc, dalb, drad = cornell
    da, dr = torch.from_numpy(dalb).cuda(), torch.from_numpy(drad).cuda()
    tf, ts = api.render_tangent(s, H, W, T, START, WIDTH, SPP, SEED, DEPTH, da, dr)
    gen = torch.Generator("cuda").manual_seed(1)
    g = torch.randn(tf.shape, device="cuda", generator=gen)
    gs = torch.randn(ts.shape, device="cuda", generator=gen)
    ga, gr, gm = api.render_backward(s, T, START, WIDTH, SPP, SEED, DEPTH, g, gs)
    lhs = (g.double() * tf.double()).sum() + (gs.double() * ts.double()).sum()
    rhs = (ga.double() * da.double()).sum() + (gr.double() * dr.double()).sum()
    assert abs(lhs.item() - rhs.item()) < 1e-3 * max(abs(rhs.item()), 1e-12)


def test_tangent_matches_central_differences(cornell):
    import torch
    api, sc, s, osc, dalb, drad = cornell
    da = torch.from_numpy(dalb).cuda() * 0.1
    tf, _ = api.render_tangent(s, H, W, T, START, WIDTH, SPP, SEED, DEPTH, da, None)
    alb0 = torch.from_numpy(sc.albedo.astype(np.float32)).cuda()
    h = 1e-2
    s.set_params(albedo=alb0 + h * da)
    fp, _ = api.render(s, H, W, T, START, WIDTH, SPP, SEED, DEPTH)
    fp = fp.clone()
    s.set_params(albedo=alb0 - h * da)
    fm, _ = api.render(s, H, W, T, START, WIDTH, SPP, SEED, DEPTH)
    s.set_params(albedo=alb0)
    s.sync()
    fd = (fp.double() - fm.double()) / (2 * h)
    assert rel_l2(tf.cpu().numpy(), fd.cpu().numpy()) < 5e-3


def test_medium_tangent_matches_oracle(oracle_mod, scenes_mod):
    api = build_and_load()
    sc = scenes_mod.media_scene(res=32)
    s = api.Scene(sc)
    osc = oracle_mod.OracleScene(sc)
    tf, ts = api.render_tangent(s, H, W, 256, 3.5, 0.01, 4, 3, 6, None, None, dmedium=1.0)
    s.sync()
    crop = (28, 36, 28, 36)
    ref = osc.render_tangent(H, W, 256, 3.5, 0.01, 4, 3, 6, dmed=1.0, crop=crop)
    assert rel_l2(ts.cpu().numpy()[28:36, 28:36], ref["steady"]) < 0.02
    assert rel_l2(tf.cpu().numpy()[28:36, 28:36].sum(2), ref["film"].sum(2)) < 0.02


@pytest.mark.parametrize("which", ["cornell_ggx", "media"])
def test_wavefront_tangent_equals_megakernel(scenes_mod, which):
    """The wavefront form carries the same prefix sums per path: equal tangent
    films up to the order of floating-point additions."""
    import torch
    api = build_and_load()
    if which == "media":
        sc = scenes_mod.media_scene(res=32)
        kw = dict(dmedium=0.7)
    else:
        sc = scenes_mod.cornell_box()
        sc.mtype[10:22] = 1
        sc.roughness[10:22] = 0.3
        kw = {}
    s = api.Scene(sc)
    gen = torch.Generator("cuda").manual_seed(4)
    da = torch.randn((sc.n_tris, 3), device="cuda", generator=gen)
    dr = torch.randn((len(sc.emitters), 3), device="cuda", generator=gen)
    a, sa = api.render_tangent(s, H, W, T, START, WIDTH, SPP, SEED, 6, da, dr, **kw)
    a, sa = a.clone(), sa.clone()
    s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT)
    try:
        b, sb = api.render_tangent(s, H, W, T, START, WIDTH, SPP, SEED, 6, da, dr, **kw)
        s.sync()
    finally:
        s.set_launch(api.MT_LAUNCH_RENDER)
    assert a.abs().max().item() > 0
    assert rel_l2(b.cpu().numpy(), a.cpu().numpy()) < 1e-4
    assert rel_l2(sb.cpu().numpy(), sa.cpu().numpy()) < 1e-4
