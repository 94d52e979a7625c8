"""GPU transient polarization (Sec. 4.2) against the oracle on the same Philox
stream: the Lambertian limit, a single conductor reflection, a Cornell box
with conductor blocks (multiple reflections, circular light), physical
Stokes vectors."""
import numpy as np
import pytest

from gpu_util import build_and_load, rel_l2

pytestmark = pytest.mark.gpu


def test_lambertian_limit(scenes_mod):
    api = build_and_load()
    sc = scenes_mod.cornell_box()
    s = api.Scene(sc)
    pf, ps = api.render_polarized(s, 64, 64, 128, 3.5, 0.02, 8, 5, 4)
    f, st = api.render(s, 64, 64, 128, 3.5, 0.02, 8, 5, 4)
    s.sync()
    assert (pf[:, :, :, 1:, :] == 0).all().item() and (ps[:, :, 1:, :] == 0).all().item()
    assert rel_l2(pf[:, :, :, 0, :].cpu().numpy(), f.cpu().numpy()) < 1e-5
    assert rel_l2(ps[:, :, 0, :].cpu().numpy(), st.cpu().numpy()) < 1e-5


def test_single_conductor_reflection_matches_oracle(oracle_mod, scenes_mod):
    api = build_and_load()
    sc = scenes_mod.point_light_plane()
    sc.mtype[:] = 1
    sc.roughness[:] = 0.3
    sc.albedo[:] = np.array([0.9, 0.6, 0.3], np.float32)
    s = api.Scene(sc)
    n = 16
    pf, ps = api.render_polarized(s, n, n, 4, 0.0, 100.0, 1, 3, 2, flags=api.MT_PIXEL_CENTER)
    s.sync()
    ref = oracle_mod.OracleScene(sc).render_polarized(n, n, 4, 0.0, 100.0, 1, 3, 2, flags=oracle_mod.PIXEL_CENTER)
    g, r = ps.cpu().numpy(), ref["steady"]
    assert np.abs(r[:, :, 1:]).max() > 1e-3 * r[:, :, 0].max()
    assert np.abs(g - r).max() < 2e-4 * np.abs(r).max()


@pytest.fixture(scope="module")
def conductor_box(oracle_mod, scenes_mod):
    sc = scenes_mod.cornell_box()
    sc.mtype[10:34] = 1
    sc.roughness[10:34] = 0.08
    sc.albedo[10:34] = np.clip(sc.albedo[10:34] + 0.3, 0, 0.95)
    return sc, oracle_mod.OracleScene(sc)


def test_conductor_box_matches_oracle(conductor_box):
    api = build_and_load()
    sc, osc = conductor_box
    s = api.Scene(sc)
    T, start, width = 200, 3.0, 0.02
    pf, ps = api.render_polarized(s, 64, 64, T, start, width, 16, 5, 6)
    s.sync()
    crop = (24, 40, 24, 40)
    ref = osc.render_polarized(64, 64, T, start, width, 16, 5, 6, crop=crop)
    g = ps.cpu().numpy()[24:40, 24:40]
    r = ref["steady"]
    assert rel_l2(g[:, :, 0], r[:, :, 0]) < 0.01
    assert np.linalg.norm(g[:, :, 1:] - r[:, :, 1:]) < 0.02 * np.linalg.norm(r[:, :, 1:])
    assert np.abs(r[:, :, 3]).max() > 0
    gf = pf.cpu().numpy()[24:40, 24:40]
    assert rel_l2(gf[..., 0, :], ref["film"][..., 0, :]) < 0.01
    # physical Stokes vectors everywhere (FP32 slack)
    S = ps.cpu().numpy()
    assert np.all(S[:, :, 0] + 1e-6 >= np.sqrt((S[:, :, 1:] ** 2).sum(2)) * (1 - 1e-5))


def test_media_rejected(scenes_mod):
    api = build_and_load()
    s = api.Scene(scenes_mod.media_scene(res=8))
    with pytest.raises(api.MtError) as e:
        api.render_polarized(s, 8, 8, 4, 0.0, 1.0, 1, 1, 2)
    assert e.value.status == api.MT_ERR_UNSUPPORTED


def test_two_reflections_match_oracle(oracle_mod, scenes_mod):
    """Conductor floor and back wall before a Lambertian ceiling (the frames of
    two polarising reflections chained on the continuation path)."""
    api = build_and_load()
    sc = scenes_mod.mirror_corner()
    s = api.Scene(sc)
    n = 24
    pf, ps = api.render_polarized(s, n, n, 4, 0.0, 100.0, 1, 4, 4, flags=api.MT_PIXEL_CENTER)
    s.sync()
    ref = oracle_mod.OracleScene(sc).render_polarized(n, n, 4, 0.0, 100.0, 1, 4, 4, flags=oracle_mod.PIXEL_CENTER)
    g, r = ps.cpu().numpy(), ref["steady"]
    lit = r[:, :, 0, :] > 1e-3 * r[:, :, 0, :].max()
    assert lit.sum() > 100
    ratio_g = g[:, :, 1:, :] / np.where(lit, g[:, :, 0, :], 1.0)[:, :, None, :]
    ratio_r = r[:, :, 1:, :] / np.where(lit, r[:, :, 0, :], 1.0)[:, :, None, :]
    err = np.abs(ratio_g - ratio_r).max(axis=2)[lit]
    assert np.quantile(err, 0.95) < 1e-3 and err.max() < 2e-2, (np.quantile(err, 0.95), err.max())
    assert rel_l2(g[:, :, 0, :], r[:, :, 0, :]) < 1e-3


@pytest.mark.parametrize("which", ["conductor_box", "mirror_corner"])
def test_wavefront_polarized_equals_path_kernel(scenes_mod, which):
    """The wavefront form keeps each path's Mueller matrices and frame in the
    path pool: the same Stokes films as the path-per-thread kernel up to the
    order of floating-point additions, whole frame and band by band."""
    import torch
    api = build_and_load()
    if which == "mirror_corner":
        sc = scenes_mod.mirror_corner()
    else:
        sc = scenes_mod.cornell_box()
        sc.mtype[10:34] = 1
        sc.roughness[10:34] = 0.08
        sc.albedo[10:34] = np.clip(sc.albedo[10:34] + 0.3, 0, 0.95)
    s = api.Scene(sc)
    H = W = 48
    T, start, width = 160, 3.0, 0.025
    a, sa = api.render_polarized(s, H, W, T, start, width, 8, 9, 6)
    a, sa = a.clone(), sa.clone()
    s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT)
    try:
        b, sb = api.render_polarized(s, H, W, T, start, width, 8, 9, 6)
        bf = torch.empty_like(b)
        bs = torch.empty_like(sb)
        for r0 in range(0, H, 16):
            api.render_polarized(s, 16, W, T, start, width, 8, 9, 6, out=(bf[r0:r0 + 16], bs[r0:r0 + 16]),
                                 window=(H, r0))
        s.sync()
    finally:
        s.set_launch(api.MT_LAUNCH_RENDER)
    assert sa[:, :, 1:].abs().max().item() > 0
    for x, y in ((b, a), (sb, sa), (bf, a), (bs, sa)):
        assert rel_l2(x.cpu().numpy(), y.cpu().numpy()) < 1e-4
