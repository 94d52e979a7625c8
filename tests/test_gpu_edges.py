"""Edge cases of the path tracer, in both forms (persistent megakernel and
wavefront stages), through the C ABI: ragged frame sizes with a single time bin
and one sample per pixel, paths of one segment, a scene without emitters,
zero-area triangles, and camera rays with exactly zero direction components."""
import dataclasses

import numpy as np
import pytest

from gpu_util import build_and_load, rel_l2

pytestmark = pytest.mark.gpu

FORMS = {"megakernel": 0, "wavefront": None}


def _scene(api, sc, form):
    s = api.Scene(sc)
    opts = api.MT_OPT_WAVEFRONT if form == "wavefront" else 0
    s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, opts)
    return s


def _close_per_pixel(g, r, tol=1e-4, frac=0.99):
    """Relative steady-image error per lit pixel: all but a few pixels (paths
    whose FP32 and FP64 branch decisions differ) within tol."""
    lit = r.sum(-1) > 1e-6 * r.sum(-1).max()
    err = np.abs(g - r).sum(-1)[lit] / r.sum(-1)[lit]
    return lit.sum() > 0 and np.quantile(err, frac) < tol


@pytest.mark.parametrize("form", list(FORMS))
def test_ragged_frame_single_bin_single_sample(oracle_mod, scenes_mod, form):
    api = build_and_load()
    sc = scenes_mod.cornell_box()
    s = _scene(api, sc, form)
    H, W, T, start, width = 23, 37, 1, 3.5, 5.0
    f, st = api.render(s, H, W, T, start, width, 1, 7, 4)
    s.sync()
    ref = oracle_mod.OracleScene(sc).render(H, W, T, start, width, 1, 7, 4)
    assert f.shape == (H, W, T, 3)
    assert _close_per_pixel(st.cpu().numpy(), ref["steady"])
    assert rel_l2(f.cpu().numpy(), ref["film"]) < 1e-2


@pytest.mark.parametrize("form", list(FORMS))
def test_one_segment_sees_only_emitters(oracle_mod, scenes_mod, form):
    """max_depth = 1: only emitters seen directly, each sample adding L_e
    (weight 1) at the camera-to-emitter distance."""
    api = build_and_load()
    sc = scenes_mod.cornell_box()
    s = _scene(api, sc, form)
    H = W = 48
    f, st = api.render(s, H, W, 64, 3.5, 0.02, 4, 3, 1)
    s.sync()
    ref = oracle_mod.OracleScene(sc).render(H, W, 64, 3.5, 0.02, 4, 3, 1)
    g = st.cpu().numpy()
    # samples grazing the light's edge may land on either side in FP32 and FP64
    differ = np.abs(g - ref["steady"]).max(-1) > 1e-5 * max(1.0, ref["steady"].max())
    assert differ.sum() <= 2, differ.sum()
    le = np.asarray(sc.emitters[0]["radiance"], np.float32)
    seen = g[..., 0] > 0
    assert seen.sum() > 0
    # every value is a multiple of L_e / spp
    k = g[seen] / (le / 4.0)
    assert np.allclose(k, np.round(k), atol=1e-4)


@pytest.mark.parametrize("form", list(FORMS))
def test_scene_without_emitters_is_black(scenes_mod, form):
    api = build_and_load()
    sc = dataclasses.replace(scenes_mod.cornell_box(), emitters=[])
    s = _scene(api, sc, form)
    f, st = api.render(s, 32, 32, 32, 3.5, 0.05, 4, 1, 6)
    s.sync()
    assert f.abs().max().item() == 0.0 and st.abs().max().item() == 0.0


@pytest.mark.parametrize("form", list(FORMS))
def test_zero_area_triangles_change_nothing(scenes_mod, form):
    """Triangles with coincident vertices (points and segments) are never hit:
    appending 64 of them inside the box leaves every path, so the film, as it
    was (up to the order of the film's floating-point additions)."""
    import torch
    api = build_and_load()
    sc = scenes_mod.cornell_box()
    rng = np.random.default_rng(5)
    p = rng.uniform(-0.9, 0.9, (64, 3)).astype(np.float32)
    q = rng.uniform(-0.9, 0.9, (64, 3)).astype(np.float32)
    deg = np.stack([p, p, q], 1)
    deg[:32, 2] = p[:32]  # points
    sc2 = dataclasses.replace(
        sc, tris=np.concatenate([sc.tris, deg]).astype(np.float32),
        albedo=np.concatenate([sc.albedo, np.full((64, 3), 0.5, np.float32)]),
        roughness=np.concatenate([sc.roughness, np.zeros(64, np.float32)]),
        mtype=np.concatenate([sc.mtype, np.zeros(64, np.uint32)]))
    a, sa = api.render(_scene(api, sc, form), 48, 48, 128, 3.5, 0.02, 8, 9, 6)
    a, sa = a.clone(), sa.clone()
    s2 = _scene(api, sc2, form)
    b, sb = api.render(s2, 48, 48, 128, 3.5, 0.02, 8, 9, 6)
    s2.sync()
    torch.cuda.synchronize()
    assert a.abs().max().item() > 0
    assert rel_l2(b.cpu().numpy(), a.cpu().numpy()) < 1e-5
    assert rel_l2(sb.cpu().numpy(), sa.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("form", list(FORMS))
def test_axis_parallel_camera_rays(oracle_mod, scenes_mod, form):
    """Pixel centres of an odd frame: the middle pixel's ray is exactly (0, 0, -1),
    so the slab test meets zero direction components.  Compared over the central
    19 x 19 pixels, whose camera rays reach the back wall before any side wall:
    pixel centres on the diagonals of the frame aim exactly at the box's concave
    corner edges, where an FP32 hit point can land an ulp behind the adjacent
    wall (a measure-zero case that the normal offset does not cover)."""
    api = build_and_load()
    sc = scenes_mod.cornell_box()
    s = _scene(api, sc, form)
    n = 33
    f, st = api.render(s, n, n, 64, 3.5, 0.05, 4, 2, 4, flags=api.MT_PIXEL_CENTER)
    s.sync()
    ref = oracle_mod.OracleScene(sc).render(n, n, 64, 3.5, 0.05, 4, 2, 4, flags=oracle_mod.PIXEL_CENTER)
    g = st.cpu().numpy()
    c = n // 2
    assert ref["steady"][c, c].sum() > 0
    assert np.abs(g[c, c] - ref["steady"][c, c]).max() < 1e-4 * ref["steady"][c, c].max()
    assert _close_per_pixel(g[7:26, 7:26], ref["steady"][7:26, 7:26])


@pytest.mark.parametrize("bad", ["nan_vertex", "inf_vertex", "ggx_roughness", "albedo", "type"])
def test_large_scene_inputs_checked_on_the_device(scenes_mod, bad):
    """Scenes above 65,536 triangles have their vertices and materials checked on
    the device after the upload; an invalid one fails with the same error (and
    the same message, naming the triangle) as the host check of small scenes,
    and leaves nothing allocated behind."""
    import torch
    api = build_and_load()
    sc = scenes_mod.diff_scene()  # 96,776 triangles
    assert sc.n_tris > 1 << 16
    k = sc.n_tris - 1234
    kw = {}
    if bad in ("nan_vertex", "inf_vertex"):
        tris = sc.tris.copy()
        tris[k, 1, 2] = np.nan if bad == "nan_vertex" else np.inf
        kw["tris"] = tris
        msg = f"non-finite vertex coordinate at triangle {k}"
    elif bad == "ggx_roughness":
        mt, ro = sc.mtype.copy(), sc.roughness.copy()
        mt[k], ro[k] = api.MT_GGX_CONDUCTOR, 0.0
        kw.update(mtype=mt, roughness=ro)
        msg = f"triangle {k}: GGX roughness"
    elif bad == "albedo":
        al = sc.albedo.copy()
        al[k, 2] = -0.5
        kw["albedo"] = al
        msg = f"triangle {k}: bad albedo"
    else:
        mt = sc.mtype.copy()
        mt[k] = 7
        kw["mtype"] = mt
        msg = f"triangle {k}: unknown material type 7"
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(api.MtError) as e:
        api.Scene(dataclasses.replace(sc, **kw))
    assert e.value.status == api.MT_ERR_INVALID_ARGUMENT
    assert msg in str(e.value), str(e.value)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    s = api.Scene(sc)  # the valid scene still loads
    assert s.stats()["n_tris"] == sc.n_tris
