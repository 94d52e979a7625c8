"""GPU path-replay gradients (Sec. 4.4) against the oracle's gradient on the
same Philox stream and against central finite differences of the GPU forward
render (step 1e-3, 32 random parameters), within 2% relative."""
import numpy as np
import pytest

from gpu_util import build_and_load

pytestmark = pytest.mark.gpu

H = W = 64
T, START, WIDTH = 64, 3.5, 0.04


def _scene(scenes_mod):
    sc = scenes_mod.cornell_box()
    rng = np.random.default_rng(4)
    sc.mtype[10:22] = 1
    sc.roughness[10:22] = 0.3
    sc.albedo[10:22] = rng.uniform(0.5, 1.0, (12, 3))
    return sc


@pytest.fixture(scope="module")
def setup(oracle_mod, scenes_mod):
    api = build_and_load()
    sc = _scene(scenes_mod)
    return api, sc, api.Scene(sc), oracle_mod.OracleScene(sc)


def test_gradient_matches_oracle(setup):
    """L2 loss against a target rendered with albedos perturbed by +-20%:
    GPU and oracle gradients (same Philox stream) agree within 2%."""
    import torch
    api, sc, s, osc = setup
    spp, seed, depth = 8, 321, 4
    rng = np.random.default_rng(0)
    alb0 = torch.from_numpy(sc.albedo.astype(np.float32)).cuda()
    s.set_params(albedo=torch.from_numpy(np.clip(sc.albedo * rng.uniform(0.8, 1.2, (sc.n_tris, 1)), 0, 1)
                                         .astype(np.float32)).cuda())
    target, target_s = api.render(s, H, W, T, START, WIDTH, spp, seed + 1, depth)
    s.set_params(albedo=alb0)
    film, steady = api.render(s, H, W, T, START, WIDTH, spp, seed, depth)
    gfilm = (2 * (film - target)).contiguous()
    gsteady = (2 * (steady - target_s)).contiguous()
    ga, gr, gm = api.render_backward(s, T, START, WIDTH, spp, seed, depth, gfilm, gsteady)
    s.sync()
    ref = osc.render_backward(H, W, T, START, WIDTH, spp, seed, depth, gfilm.cpu().numpy().astype(np.float64),
                              gsteady.cpu().numpy().astype(np.float64))
    ga = ga.cpu().numpy()
    ra = ref["albedo"]
    err = np.linalg.norm(ga - ra) / np.linalg.norm(ra)
    assert err < 0.02, err
    big = np.abs(ra) > 0.02 * np.abs(ra).max()
    rel = np.abs(ga - ra)[big] / np.abs(ra)[big]
    assert np.median(rel) < 0.005 and rel.max() < 0.05, (np.median(rel), rel.max())
    assert np.allclose(gr.cpu().numpy()[:1], ref["radiance"], rtol=0.02)


@pytest.mark.parametrize("which", ["steady", "film"])
def test_gradient_per_term_matches_oracle_tightly(setup, which):
    """Random dL/dsteady (every contribution, also those outside the time
    window, e.g. light found at the last vertex) or random dL/dfilm alone:
    the replay's albedo and radiance gradients equal the oracle's to FP32
    accuracy, not merely within a few percent."""
    import torch
    api, sc, s, osc = setup
    spp, seed, depth = 4, 77, 4
    gen = torch.Generator("cuda").manual_seed(2)
    gf = torch.randn((H, W, T, 3), device="cuda", generator=gen)
    gs = torch.randn((H, W, 3), device="cuda", generator=gen)
    if which == "steady":
        gf.zero_()
    else:
        gs.zero_()
    ga, gr, gm = api.render_backward(s, T, START, WIDTH, spp, seed, depth, gf, gs)
    s.sync()
    ref = osc.render_backward(H, W, T, START, WIDTH, spp, seed, depth, gf.cpu().numpy().astype(np.float64),
                              gs.cpu().numpy().astype(np.float64))
    ra = ref["albedo"]
    assert np.linalg.norm(ga.cpu().numpy() - ra) < 2e-3 * np.linalg.norm(ra)
    assert np.linalg.norm(gr.cpu().numpy()[:1] - ref["radiance"]) < 2e-3 * np.linalg.norm(ref["radiance"])


def test_gradient_matches_gpu_finite_differences(setup):
    import torch
    api, sc, s, osc = setup
    spp, seed, depth = 8, 77, 4
    base_alb = torch.from_numpy(sc.albedo.astype(np.float32)).cuda()
    film0, steady0 = api.render(s, H, W, T, START, WIDTH, spp, seed, depth)
    rng = np.random.default_rng(1)
    target = (film0 * torch.from_numpy(rng.uniform(0.7, 1.3, film0.shape).astype(np.float32)).cuda()).double()

    def loss():
        f, _ = api.render(s, H, W, T, START, WIDTH, spp, seed, depth)
        return float(((f.double() - target) ** 2).sum())

    g = 2 * (film0.double() - target)
    ga, gr, _ = api.render_backward(s, T, START, WIDTH, spp, seed, depth, g.float().contiguous())
    ga = ga.cpu().numpy()
    h = 1e-3
    params = [(int(t), int(c)) for t, c in zip(rng.integers(0, 34, 32), rng.integers(0, 3, 32))]
    gmax = np.abs(ga).max()
    ok = 0
    for t, c in params:
        vals = []
        for sgn in (1, -1):
            a = base_alb.clone()
            a[t, c] += sgn * h
            s.set_params(albedo=a)
            vals.append(loss())
        s.set_params(albedo=base_alb)
        fd = (vals[0] - vals[1]) / (2 * h)
        if abs(fd) > 1e-2 * gmax:
            assert abs(fd - ga[t, c]) <= 0.02 * abs(fd), (t, c, fd, ga[t, c])
            ok += 1
    assert ok >= 8


def test_autograd_function(setup):
    import torch
    api, sc, s, osc = setup
    TR = api.TransientRender
    alb = torch.from_numpy(sc.albedo.astype(np.float32)).cuda().requires_grad_(True)
    rad = torch.tensor([[10.0, 10.0, 10.0]], device="cuda", requires_grad=True)
    film, steady = TR.apply(alb, rad, s, H, W, T, START, WIDTH, 4, 9, 4)
    loss = (film ** 2).sum() + steady.sum()
    loss.backward()
    g = 2 * film.detach()
    ga, gr, _ = api.render_backward(s, T, START, WIDTH, 4, 9, 4, g.contiguous(), torch.ones_like(steady))
    assert torch.allclose(alb.grad, ga, rtol=1e-4, atol=1e-7)
    assert torch.allclose(rad.grad, gr[:1], rtol=1e-4)


@pytest.mark.parametrize("which", ["cornell_ggx", "media"])
def test_wavefront_backward_equals_megakernel(setup, scenes_mod, which):
    """The wavefront replay (vertex records in the path pool, suffix sums when a
    path ends) gives the megakernel's gradients on the same paths."""
    import torch
    api = setup[0]
    if which == "media":
        sc = scenes_mod.media_scene(res=32)
        depth = 8
    else:
        sc = setup[1]
        depth = 4
    s = api.Scene(sc)
    gen = torch.Generator("cuda").manual_seed(5)
    gf = torch.randn((H, W, T, 3), device="cuda", generator=gen)
    gs = torch.randn((H, W, 3), device="cuda", generator=gen)
    a = api.render_backward(s, T, START, WIDTH, 8, 21, depth, gf, gs)
    a = [x.clone() for x in a]
    s.set_launch(api.MT_LAUNCH_BACKWARD, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT)
    try:
        b = api.render_backward(s, T, START, WIDTH, 8, 21, depth, gf, gs)
        s.sync()
    finally:
        s.set_launch(api.MT_LAUNCH_BACKWARD)
    ga, gb = a[0].cpu().numpy(), b[0].cpu().numpy()
    assert np.abs(ga).max() > 0
    assert np.linalg.norm(gb - ga) < 1e-4 * np.linalg.norm(ga)
    assert np.linalg.norm(b[1].cpu().numpy() - a[1].cpu().numpy()) < 1e-4 * np.linalg.norm(a[1].cpu().numpy())
    if which == "media":
        assert abs(b[2].item() - a[2].item()) < 1e-4 * abs(a[2].item())
