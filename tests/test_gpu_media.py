"""GPU parity of transient volumetric path tracing (Sec. 4.1): delta tracking
with the optical path length accumulated through the medium, ratio-tracked
next-event estimation, medium-albedo gradients, and the bounded tracking loop
reporting MT_ERR_TIMEOUT instead of hanging."""
import numpy as np
import pytest

from gpu_util import build_and_load, divergent_pixels, match_contribs, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def media(oracle_mod, scenes_mod):
    api = build_and_load()
    sc = scenes_mod.media_scene(res=32)
    return api, sc, api.Scene(sc), oracle_mod.OracleScene(sc)


@pytest.fixture(scope="module")
def media128(oracle_mod, scenes_mod):
    """The medium of the volumetric workload: a 128^3 fBm density grid."""
    api = build_and_load()
    sc = scenes_mod.media_scene(res=128)
    return api, sc, api.Scene(sc), oracle_mod.OracleScene(sc)


@pytest.mark.parametrize("form", ["megakernel", "wavefront"])
def test_media_contributions_and_film(media128, scenes_mod, form):
    """Per contribution (value, time bin) and per time bin of the film, on the
    128^3 grid with the volumetric workload's window (T = 1024 bins of 5 mm
    from 3.5 m) and depth 16 (Sec. 4.1 volumetric scattering; time of flight
    through the medium, Sec. 3 Eq. 3)."""
    api, sc, s, osc = media128
    fm = scenes_mod.MEDIA_FILM
    H = W = 64
    T, start, width = fm.T, fm.start_opl, fm.bin_width
    spp, seed, depth = 32, 25660, 16
    if form == "wavefront":
        s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT)
    try:
        film, steady, rec, n = api.render_dump(s, H, W, T, start, width, spp, seed, depth, cap=8_000_000)
        f2, s2 = api.render(s, H, W, T, start, width, spp, seed, depth)
        s.sync()
    finally:
        s.set_launch(api.MT_LAUNCH_RENDER)
    assert n <= 8_000_000
    crop = (16, 48, 16, 48)
    ref = osc.render(H, W, T, start, width, spp, seed, depth, crop=crop, dump_cap=8_000_000)
    px = rec["pixel"] % W
    py = rec["pixel"] // W
    sel = (px >= crop[0]) & (px < crop[1]) & (py >= crop[2]) & (py < crop[3])
    nm, div, worst, bad, bin_bad, _ = match_contribs(rec[sel], ref["dump"], start=start, width=width)
    assert nm > 20000
    assert bin_bad == 0, bin_bad
    assert div <= 5e-4 * nm and bad <= 5e-3 * nm, \
        f"divergent {div}/{nm} = {div / nm:.1e}, off {bad} (worst {worst:.1e})"
    for fg, sg in ((film, steady), (f2, s2)):  # dump form and the timed form
        g = fg.cpu().numpy()[crop[2]:crop[3], crop[0]:crop[1]]
        gs = sg.cpu().numpy()[crop[2]:crop[3], crop[0]:crop[1]]
        # per bin, on pixels whose paths all agree with the oracle's
        keep = np.ones(g.shape[:2], bool)
        for p in divergent_pixels(rec[sel], ref["dump"], rel=1e-3):
            keep[p // W - crop[2], p % W - crop[0]] = False
        assert keep.mean() > 0.8, keep.mean()
        assert rel_l2(g[keep], ref["film"][keep]) < 1e-3
        assert rel_l2(gs[keep], ref["steady"][keep]) < 1e-3
        # per bin of the crop's transient (summed over its pixels) where a bin holds >= 100 samples
        d = ref["dump"]
        inb = (d["bin"] >= 0) & (d["bin"] < T)
        cnt = np.bincount(d["bin"][inb], minlength=T)
        m = cnt >= 100
        assert m.sum() > 200
        assert rel_l2(g.sum((0, 1))[m], ref["film"].sum((0, 1))[m]) < 0.01


def test_media_wavefront_equals_megakernel(media):
    """Same estimator and random numbers in both forms: equal films up to the
    order of floating-point additions."""
    api, sc, s, osc = media
    H = W = 64
    T, start, width = 512, 3.5, 0.01
    a, sa = api.render(s, H, W, T, start, width, 16, 9, 12)
    s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT)
    try:
        b, sb = api.render(s, H, W, T, start, width, 16, 9, 12)
        s.sync()
    finally:
        s.set_launch(api.MT_LAUNCH_RENDER)
    assert rel_l2(b.cpu().numpy(), a.cpu().numpy()) < 1e-4
    assert rel_l2(sb.cpu().numpy(), sa.cpu().numpy()) < 1e-4


def test_medium_albedo_gradient(media):
    import torch
    api, sc, s, osc = media
    H = W = 32
    T, start, width = 64, 3.5, 0.05
    spp, seed, depth = 4, 5, 6
    rng = np.random.default_rng(3)
    g = rng.uniform(-1, 1, (H, W, T, 3))
    ga, gr, gm = api.render_backward(s, T, start, width, spp, seed, depth, torch.from_numpy(g.astype(np.float32)).cuda())
    ref = osc.render_backward(H, W, T, start, width, spp, seed, depth, g)
    assert abs(gm.item() - ref["medium_albedo"]) < 0.02 * abs(ref["medium_albedo"])
    ra = ref["albedo"]
    assert np.linalg.norm(ga.cpu().numpy() - ra) < 0.02 * np.linalg.norm(ra)


def test_bounded_tracking_reports_timeout(api_free_scene=None):
    """A medium whose majorant is far above its typical density makes the
    free-flight loop exceed its step cap; the kernel drops those paths, sets the
    error word, and mt_sync reports MT_ERR_TIMEOUT (no hang, no fault)."""
    import torch
    from paper_2510_25660_gb300 import scenes
    api = build_and_load()
    sc = scenes.cornell_box()
    dens = np.zeros((8, 8, 8), np.float32)
    dens[0, 0, 0] = 5000.0  # majorant 5000 /m, a 2 m segment takes ~10^4 null steps
    sc.medium = dict(lo=(-1, -1, -1), hi=(1, 1, 1), density=dens, albedo=0.9, g=0.0)
    s = api.Scene(sc)
    api.render(s, 8, 8, 16, 3.5, 0.1, 1, 1, 2)
    with pytest.raises(api.MtError) as e:
        s.sync()
    assert e.value.status == api.MT_ERR_TIMEOUT
    # the context stays usable
    api.render(s, 8, 8, 16, 3.5, 0.1, 1, 1, 1)
    torch.cuda.synchronize()
    # the wavefront form reports the same
    s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT)
    api.render(s, 8, 8, 16, 3.5, 0.1, 1, 1, 2)
    with pytest.raises(api.MtError) as e:
        s.sync()
    assert e.value.status == api.MT_ERR_TIMEOUT
    api.render(s, 8, 8, 16, 3.5, 0.1, 1, 1, 1)
    torch.cuda.synchronize()
