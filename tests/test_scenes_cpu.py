"""The seeded synthetic inputs (no GPU): the scenes, films and scan grids that
stand in for the paper's workloads have the sizes, materials, lights and
value ranges the input recipe states, and are reproducible from their seeds.

Stand-ins for the paper's scenes (Cornell box of Sec. 4, the large static
scene of the transient renders of Sec. 3, the NLOS relay-wall setup of Sec.
4.5, the differentiable scene of Sec. 4.4, the participating medium of Sec.
4.1); no dataset or public benchmark is used.
"""
import hashlib
import math

import numpy as np
import pytest

from paper_2510_25660_gb300 import scenes


def _digest(sc):
    h = hashlib.sha256()
    for a in (sc.tris, sc.albedo, sc.roughness, sc.mtype):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def _normals(tris):
    t = tris.astype(np.float64)
    return np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0])


@pytest.fixture(scope="module")
def large():
    return scenes.large_scene()


def test_triangle_counts_and_types():
    for make, n in ((scenes.cornell_box, 36), (scenes.diff_scene, 96776), (scenes.nlos_scene, 49410)):
        sc = make()
        assert sc.n_tris == n
        assert sc.tris.dtype == np.float32 and sc.tris.shape == (n, 3, 3)
        assert sc.albedo.dtype == np.float32 and sc.albedo.shape == (n, 3)
        assert sc.roughness.dtype == np.float32 and sc.mtype.dtype == np.uint32
        assert np.isfinite(sc.tris).all()


def test_large_scene_recipe(large):
    sc = large
    assert sc.n_tris == 1164296
    hf = 2 * 512 * 512  # 513^2-vertex heightfield
    ggx = sc.mtype == scenes.GGX
    # 30 % GGX conductors per heightfield patch and per sphere
    assert 0.2 < ggx[:hf].mean() < 0.4 and 0.2 < ggx[hf:-8].mean() < 0.4
    assert (sc.roughness[ggx] >= 0.05).all() and (sc.roughness[ggx] <= 0.5).all()
    assert (sc.albedo[ggx] >= 0.5).all() and (sc.albedo[ggx] <= 1.0).all()
    lam = ~ggx
    lam[-8:] = False
    assert (sc.albedo[lam] >= 0.2).all() and (sc.albedo[lam] <= 0.8).all() and (sc.roughness[lam] == 0).all()
    # the heightfield spans 20 x 20 m with a 2 m amplitude
    v = sc.tris[:hf].reshape(-1, 3)
    assert np.allclose(v[:, 0].min(), -10) and np.allclose(v[:, 0].max(), 10)
    assert np.allclose(v[:, 2].min(), -10) and np.allclose(v[:, 2].max(), 10)
    assert np.abs(v[:, 1]).max() <= 2.0 + 1e-6
    assert (_normals(sc.tris[:hf])[:, 1] > 0).all()  # wound with +y normals
    # four 1 m quad lights 8 m up, radiance 20, facing down
    assert len(sc.emitters) == 4
    for e in sc.emitters:
        lt = sc.tris[e["first_tri"]:e["first_tri"] + e["n_tris"]]
        assert e["n_tris"] == 2 and e["radiance"] == (20.0, 20.0, 20.0)
        assert np.allclose(lt[..., 1], 8.0)
        assert (_normals(lt)[:, 1] < 0).all()
        assert math.isclose(0.5 * np.linalg.norm(_normals(lt), axis=1).sum(), 1.0, rel_tol=1e-6)
    assert sc.emitters[-1]["first_tri"] + 2 == sc.n_tris
    # camera 6 m up, 12 m out, 30 degrees down, 50 degrees horizontal field of view
    cam = sc.camera
    d = np.subtract(cam["target"], cam["origin"])
    assert cam["origin"] == (0.0, 6.0, 12.0) and cam["fov_x_deg"] == 50.0
    assert math.isclose(math.degrees(math.asin(-d[1] / np.linalg.norm(d))), 30.0, rel_tol=1e-9)


def test_scenes_are_reproducible_from_their_seeds(large):
    assert _digest(scenes.large_scene()) == _digest(large)
    assert _digest(scenes.cornell_box()) == _digest(scenes.cornell_box())
    assert _digest(scenes.cornell_box(seed=1)) != _digest(scenes.cornell_box())


def test_cornell_box_recipe():
    sc = scenes.cornell_box()
    assert (sc.albedo[:-2] >= 0.2).all() and (sc.albedo[:-2] <= 0.8).all() and (sc.mtype == scenes.LAMBERT).all()
    v = sc.tris.reshape(-1, 3)
    assert v.min() >= -1.0 and v.max() <= 1.0
    (e,) = sc.emitters
    lt = sc.tris[e["first_tri"]:e["first_tri"] + e["n_tris"]]
    assert e["radiance"] == (10.0, 10.0, 10.0) and e["first_tri"] == 34
    assert math.isclose(0.5 * np.linalg.norm(_normals(lt), axis=1).sum(), 0.25, rel_tol=1e-6)  # 0.5 m quad
    assert (_normals(lt)[:, 1] < 0).all()
    assert sc.camera["origin"] == (0.0, 0.0, 3.5) and sc.camera["fov_x_deg"] == 40.0


def test_nlos_scene_recipe():
    sc = scenes.nlos_scene()
    first, n = sc.hidden
    assert (first, n) == (2, sc.n_tris - 2) and sc.emitters == []
    wall = sc.tris[:2]
    assert np.allclose(wall[..., 2], 0.0) and (_normals(wall)[:, 2] > 0).all()
    assert math.isclose(0.5 * np.linalg.norm(_normals(wall), axis=1).sum(), 1.0, rel_tol=1e-6)
    assert sc.wall["albedo"] == 0.8 and sc.wall["normal"] == (0.0, 0.0, 1.0)
    z = sc.tris[first:first + n][..., 2]
    assert 0.53 < z.min() < 0.55 and 1.51 < z.max() < 1.53  # hidden mesh 0.54-1.52 m in front of the wall


def test_media_scene_recipe():
    sc = scenes.media_scene()
    m = sc.medium
    assert m["density"].shape == (128, 128, 128) and m["density"].dtype == np.float32
    assert math.isclose(float(m["density"].min()), 0.1, rel_tol=1e-6)
    assert math.isclose(float(m["density"].max()), 2.0, rel_tol=1e-6)
    assert m["albedo"] == 0.9 and m["g"] == 0.3 and m["lo"] == (-1.0, -1.0, -1.0) and m["hi"] == (1.0, 1.0, 1.0)
    assert _digest(sc) == _digest(scenes.cornell_box())  # the Cornell box's geometry


def test_film_windows():
    f = scenes.CORNELL_FILM
    assert (f.H, f.W, f.T, f.start_opl, f.bin_width) == (64, 64, 256, 3.5, 0.01)
    f = scenes.LARGE_FILM
    assert (f.H, f.W, f.T, f.start_opl, f.bin_width) == (512, 512, 2048, 12.0, 0.005)
    f = scenes.DIFF_FILM
    assert (f.H, f.W, f.T, f.start_opl, f.bin_width) == (256, 256, 512, 15.0, 0.005)
    f = scenes.MEDIA_FILM
    assert (f.H, f.W, f.T, f.start_opl, f.bin_width) == (256, 256, 1024, 3.5, 0.005)
    assert (scenes.NLOS_T, scenes.NLOS_W, scenes.NLOS_START) == (4096, 0.003, 0.0)


def test_wall_grid_is_cell_centred_and_row_major():
    g = scenes.wall_grid(4, 2)
    assert g.shape == (8, 3) and g.dtype == np.float32
    assert np.allclose(g[:4, 0], [-0.375, -0.125, 0.125, 0.375]) and np.allclose(g[:4, 1], -0.25)
    assert np.allclose(g[4:, 1], 0.25) and np.allclose(g[:, 2], 0.0)


def test_perturbed_albedo_target():
    sc = scenes.cornell_box()
    p = scenes.perturbed_albedo(sc)
    assert p.dtype == np.float32 and p.shape == sc.albedo.shape
    ratio = p / sc.albedo
    assert (ratio >= 0.8 - 1e-6).all() and (ratio <= 1.2 + 1e-6).all() and p.max() <= 1.0
    # one factor per triangle, shared by its three channels
    assert np.allclose(ratio, ratio[:, :1], rtol=1e-6)
    assert np.array_equal(p, scenes.perturbed_albedo(sc))
