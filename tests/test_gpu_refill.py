"""The wavefront form in its pool-refill regime, against the oracle.

The wavefront tracer keeps at most P paths in flight (mt_set_wavefront_pool);
a render of more paths restarts finished slots from the free-slot stack, so
every path of the estimator (Sec. 3, Eq. 9 with path reuse) must still be
traced exactly once.  Here the pool is cut to a few thousand slots so that a
65,536-path Cornell render refills it in every iteration, and every form that
keeps state in the pool is compared with the oracle on the same Philox stream
and with the same render in a pool that holds all its paths: the forward
render (per-contribution dump and fused film), the path replay (vertex
records), the forward-mode derivative (prefix sums), the phasor film, media
and transient polarization (Mueller matrices in the pool).
"""
import numpy as np
import pytest

from gpu_util import build_and_load, divergent_pixels, match_contribs, rel_l2

pytestmark = pytest.mark.gpu

H = W = 64
T, START, WIDTH = 256, 3.5, 0.01
POOL = 4096  # 65,536 paths at 16 spp: each slot carries ~16 paths


@pytest.fixture(scope="module")
def cornell(oracle_mod, scenes_mod):
    api = build_and_load()
    sc = scenes_mod.cornell_box()
    rng = np.random.default_rng(4)
    sc.mtype[10:22] = 1  # one GGX block, so both BSDFs run in the refilled slots
    sc.roughness[10:22] = 0.3
    sc.albedo[10:22] = rng.uniform(0.5, 1.0, (12, 3))
    s = api.Scene(sc)
    s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT | api.MT_OPT_STAGE_TIMING)
    s.set_launch(api.MT_LAUNCH_BACKWARD, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT)
    return api, sc, s, oracle_mod.OracleScene(sc)


def _pool(s, n):
    s.set_wavefront_pool(n)


def test_refill_forward_per_path_and_film(cornell):
    api, sc, s, osc = cornell
    spp, seed, depth = 16, 25660, 4
    _pool(s, POOL)
    try:
        s.stage_times(reset=True)
        s.read_counters(reset=True)
        film, steady, rec, n = api.render_dump(s, H, W, T, START, WIDTH, spp, seed, depth, cap=4_000_000)
        paths = s.read_counters(reset=True)["paths"]
        f2, s2 = api.render(s, H, W, T, START, WIDTH, spp, seed, depth)
        s.sync()
        iters = s.stage_times(reset=True)["iterations"]
    finally:
        _pool(s, 0)
    f_full, s_full = api.render(s, H, W, T, START, WIDTH, spp, seed, depth)
    s.sync()
    # 65,536 paths through 4,096 slots: the pool was refilled many times
    assert iters >= H * W * spp // POOL, iters  # one pool holding every path would need <= depth + 1
    assert n <= 4_000_000
    # every path of the frame started exactly once, each with a (pixel, sample) of this frame
    assert paths == H * W * spp, paths
    ps = rec["pixel"].astype(np.int64) * spp + rec["sample"]
    assert ps.min() >= 0 and ps.max() < H * W * spp
    crop = (16, 48, 16, 48)
    ref = osc.render(H, W, T, START, WIDTH, spp, seed, depth, crop=crop, dump_cap=4_000_000)
    px, py = rec["pixel"] % W, rec["pixel"] // W
    sel = (px >= crop[0]) & (px < crop[1]) & (py >= crop[2]) & (py < crop[3])
    nm, div, worst, bad, bin_bad, _ = match_contribs(rec[sel], ref["dump"], start=START, width=WIDTH)
    assert nm > 20000 and bin_bad == 0, (nm, bin_bad)
    assert div <= 1e-4 * nm and bad <= 1e-3 * nm, f"divergent {div}/{nm} = {div / nm:.1e}, off {bad} (worst {worst:.1e})"
    # the fused film of the capped pool: equal to the oracle on pixels without divergent paths,
    # and to the same render with all paths in flight up to the order of additions
    g = f2.cpu().numpy()[crop[2]:crop[3], crop[0]:crop[1]]
    bad_px = divergent_pixels(rec[sel], ref["dump"])
    keep = np.ones(g.shape[:2], bool)
    for p in bad_px:
        keep[p // W - crop[2], p % W - crop[0]] = False
    assert keep.mean() > 0.95
    assert rel_l2(g[keep], ref["film"][keep]) < 1e-4
    assert rel_l2(s2.cpu().numpy()[crop[2]:crop[3], crop[0]:crop[1]][keep], ref["steady"][keep]) < 1e-4
    assert rel_l2(f2.cpu().numpy(), f_full.cpu().numpy()) < 1e-5
    assert rel_l2(s2.cpu().numpy(), s_full.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("pool", [32, 1000])
def test_refill_tiny_and_ragged_pools(cornell, pool):
    """A 32-slot pool (one warp of paths) and a pool that is not a multiple of
    the warp size give the same film as a pool holding every path."""
    api, sc, s, osc = cornell
    spp, seed, depth = 4, 9, 4
    f_full, s_full = api.render(s, 32, 32, T, START, WIDTH, spp, seed, depth)
    _pool(s, pool)
    try:
        f, st = api.render(s, 32, 32, T, START, WIDTH, spp, seed, depth)
        s.sync()
    finally:
        _pool(s, 0)
    assert rel_l2(f.cpu().numpy(), f_full.cpu().numpy()) < 1e-5
    assert rel_l2(st.cpu().numpy(), s_full.cpu().numpy()) < 1e-5


def test_refill_backward_matches_oracle(cornell):
    """Path replay with vertex records in a 1,024-slot pool: per-term gradients
    equal the oracle's to FP32 accuracy and the uncapped replay's."""
    import torch
    api, sc, s, osc = cornell
    Tb, Wb = 64, 0.04
    spp, seed, depth = 4, 77, 4
    gen = torch.Generator("cuda").manual_seed(2)
    gf = torch.randn((H, W, Tb, 3), device="cuda", generator=gen)
    gs = torch.randn((H, W, 3), device="cuda", generator=gen)
    full = [x.clone() for x in api.render_backward(s, Tb, START, Wb, spp, seed, depth, gf, gs)]
    _pool(s, 1024)
    try:
        ga, gr, gm = api.render_backward(s, Tb, START, Wb, spp, seed, depth, gf, gs)
        s.sync()
    finally:
        _pool(s, 0)
    ref = osc.render_backward(H, W, Tb, START, Wb, spp, seed, depth, gf.cpu().numpy().astype(np.float64),
                              gs.cpu().numpy().astype(np.float64))
    ra = ref["albedo"]
    assert np.linalg.norm(ga.cpu().numpy() - ra) < 2e-3 * np.linalg.norm(ra)
    assert np.linalg.norm(gr.cpu().numpy()[:1] - ref["radiance"]) < 2e-3 * np.linalg.norm(ref["radiance"])
    fa = full[0].cpu().numpy()
    assert np.linalg.norm(ga.cpu().numpy() - fa) < 1e-5 * np.linalg.norm(fa)


def test_refill_tangent_and_phasor(cornell):
    import torch
    api, sc, s, osc = cornell
    spp, seed, depth = 8, 31, 4
    rng = np.random.default_rng(6)
    da = torch.from_numpy(rng.normal(size=(sc.n_tris, 3)).astype(np.float32)).cuda()
    lam = np.array([0.2, 0.066])
    a = [x.clone() for x in api.render_tangent(s, H, W, 128, START, 0.02, spp, seed, depth, da, None)]
    pa = [x.clone() for x in api.render_phasor(s, H, W, lam, spp, seed, depth)]
    _pool(s, 2048)
    try:
        b = api.render_tangent(s, H, W, 128, START, 0.02, spp, seed, depth, da, None)
        pb = api.render_phasor(s, H, W, lam, spp, seed, depth)
        s.sync()
    finally:
        _pool(s, 0)
    assert np.abs(a[0].cpu().numpy()).max() > 0
    assert rel_l2(b[0].cpu().numpy(), a[0].cpu().numpy()) < 1e-5
    assert rel_l2(b[1].cpu().numpy(), a[1].cpu().numpy()) < 1e-5
    assert rel_l2(pb[0].cpu().numpy(), pa[0].cpu().numpy()) < 1e-5
    crop = (24, 40, 24, 40)
    ref = osc.render_tangent(H, W, 128, START, 0.02, spp, seed, depth, dalb=da.cpu().numpy(), crop=crop)
    assert rel_l2(b[0].cpu().numpy()[24:40, 24:40], ref["film"]) < 2e-3


def test_refill_polarized_matches_oracle(cornell):
    api, sc, s, osc = cornell
    Tp, Sp, Wp = 200, 3.0, 0.02
    spp, seed, depth = 16, 5, 6
    a = [x.clone() for x in api.render_polarized(s, H, W, Tp, Sp, Wp, spp, seed, depth)]
    _pool(s, 2048)
    try:
        pf, ps = api.render_polarized(s, H, W, Tp, Sp, Wp, spp, seed, depth)
        s.sync()
    finally:
        _pool(s, 0)
    assert rel_l2(pf.cpu().numpy(), a[0].cpu().numpy()) < 1e-5
    assert rel_l2(ps.cpu().numpy(), a[1].cpu().numpy()) < 1e-5
    crop = (24, 40, 24, 40)
    ref = osc.render_polarized(H, W, Tp, Sp, Wp, spp, seed, depth, crop=crop)
    assert rel_l2(ps.cpu().numpy()[24:40, 24:40], ref["steady"]) < 1e-3


def test_refill_media(scenes_mod):
    """Delta tracking and ratio-tracked shadow rays in a 2,048-slot pool give the
    film of the persistent megakernel on the same paths."""
    api = build_and_load()
    sc = scenes_mod.media_scene(res=32)
    s = api.Scene(sc)
    a, sa = api.render(s, H, W, 512, START, 0.01, 16, 9, 12)
    s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT)
    s.set_wavefront_pool(2048)
    b, sb = api.render(s, H, W, 512, START, 0.01, 16, 9, 12)
    s.sync()
    assert rel_l2(b.cpu().numpy(), a.cpu().numpy()) < 1e-4
    assert rel_l2(sb.cpu().numpy(), sa.cpu().numpy()) < 1e-4


def test_pool_size_argument_checks(cornell):
    api, sc, s, osc = cornell
    for bad in (-1, 1, 31, (1 << 22) + 1):
        with pytest.raises(api.MtError) as e:
            s.set_wavefront_pool(bad)
        assert e.value.status == api.MT_ERR_INVALID_ARGUMENT
    s.set_wavefront_pool(0)
