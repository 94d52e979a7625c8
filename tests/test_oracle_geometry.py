"""Pins for the oracle's ray casting: triangle test against exact rational
arithmetic, BVH traversal against brute force, and the pinhole camera against
its closed form.  Paths are sequences of mutually visible points (Sec. 3,
Eq. 1); visibility V and segment lengths (Eq. 3) come from these queries."""
from fractions import Fraction as Fr

import numpy as np
import pytest


def _exact_hit(tri, o, d):
    """Exact ray/triangle intersection in rationals: returns (t, min barycentric) or None."""
    v0, v1, v2 = ([Fr(float(x)) for x in v] for v in tri)
    O = [Fr(float(x)) for x in o]
    D = [Fr(float(x)) for x in d]

    def sub(a, b):
        return [a[i] - b[i] for i in range(3)]

    def cr(a, b):
        return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]

    def dt(a, b):
        return sum(a[i] * b[i] for i in range(3))

    n = cr(sub(v1, v0), sub(v2, v0))
    den = dt(n, D)
    if den == 0:
        return None
    t = dt(n, sub(v0, O)) / den
    P = [O[i] + t * D[i] for i in range(3)]
    a0 = dt(cr(sub(v1, P), sub(v2, P)), n)
    a1 = dt(cr(sub(v2, P), sub(v0, P)), n)
    a2 = dt(cr(sub(v0, P), sub(v1, P)), n)
    nn = dt(n, n)
    b = [a0 / nn, a1 / nn, a2 / nn]
    return t, min(b)


def test_triangle_test_matches_exact_rationals(oracle_mod, scenes_mod):
    tris = scenes_mod.random_mesh(3, 40)
    o, d = scenes_mod.random_rays(4, 60)
    checked = 0
    for k in range(len(tris)):
        sc = scenes_mod.Scene(tris[k:k + 1], np.full((1, 3), 0.5, np.float32), np.zeros(1, np.float32),
                              np.zeros(1, np.uint32), [], dict(origin=(0, 0, 5), target=(0, 0, 0), up=(0, 1, 0), fov_x_deg=40))
        osc = oracle_mod.OracleScene(sc)
        for r in range(len(o)):
            ex = _exact_hit(tris[k], o[r], d[r])
            i, t = osc.intersect(o[r].astype(np.float64), d[r].astype(np.float64), brute=True)
            if ex is None:
                assert i == -1
                continue
            te, bmin = ex
            if abs(bmin) < 1e-9 or abs(te) < 1e-9:
                continue  # on an edge or at the origin: either answer is acceptable
            expect_hit = bmin > 0 and te > 0
            assert (i == 0) == expect_hit, (k, r, float(te), float(bmin))
            if expect_hit:
                assert abs(t - float(te)) <= 1e-12 * max(1.0, abs(float(te)))
            checked += 1
    assert checked > 1000


@pytest.mark.parametrize("seed,n", [(1, 7), (2, 64), (3, 200)])
def test_bvh_matches_brute_force(oracle_mod, scenes_mod, seed, n):
    tris = scenes_mod.random_mesh(seed, n)
    sc = scenes_mod.Scene(tris, np.full((n, 3), 0.5, np.float32), np.zeros(n, np.float32), np.zeros(n, np.uint32),
                          [], dict(origin=(0, 0, 5), target=(0, 0, 0), up=(0, 1, 0), fov_x_deg=40))
    osc = oracle_mod.OracleScene(sc)
    o, d = scenes_mod.random_rays(seed + 10, 3000)
    rng = np.random.default_rng(seed)
    hits = 0
    for r in range(len(o)):
        oo, dd = o[r].astype(np.float64), d[r].astype(np.float64)
        i1, t1 = osc.intersect(oo, dd, brute=False)
        i2, t2 = osc.intersect(oo, dd, brute=True)
        assert i1 == i2 and (i1 < 0 or t1 == t2), (r, i1, i2, t1, t2)
        hits += i1 >= 0
        tm = rng.uniform(0.1, 5.0)
        assert osc.occluded(oo, dd, tm, brute=False) == osc.occluded(oo, dd, tm, brute=True)
    assert hits > 100


def test_tie_break_smaller_index(oracle_mod, scenes_mod):
    """Two coincident triangles: the closest hit reports the smaller index."""
    t = np.array([[[-1, -1, 0], [1, -1, 0], [0, 1, 0]]] * 2, np.float32)
    sc = scenes_mod.Scene(t, np.full((2, 3), 0.5, np.float32), np.zeros(2, np.float32), np.zeros(2, np.uint32),
                          [], dict(origin=(0, 0, 5), target=(0, 0, 0), up=(0, 1, 0), fov_x_deg=40))
    osc = oracle_mod.OracleScene(sc)
    for brute in (True, False):
        i, tt = osc.intersect(np.array([0.1, 0.0, 3.0]), np.array([0.0, 0.0, -1.0]), brute=brute)
        assert i == 0 and tt == 3.0


def test_camera_closed_form(oracle_mod, scenes_mod):
    sc = scenes_mod.cornell_box()
    osc = oracle_mod.OracleScene(sc)
    W, H = 64, 48
    f = np.array([0, 0, -1.0])
    o, d = osc.camera_ray(W, H, W // 2, H // 2, 0.0, 0.0)
    assert np.allclose(o, [0, 0, 3.5]) and np.allclose(d, f, atol=1e-15)
    # left image edge, vertical centre: angle to the forward axis = fov_x / 2
    o, d = osc.camera_ray(W, H, 0, H // 2, 0.0, 0.0)
    assert abs(np.degrees(np.arccos(d @ f)) - 20.0) < 1e-9 and d[0] < 0
    # top edge, horizontal centre: tan(angle) = tan(fov_x/2) * H / W
    o, d = osc.camera_ray(W, H, W // 2, 0, 0.0, 0.0)
    assert abs(np.tan(np.arccos(d @ f)) - np.tan(np.radians(20.0)) * H / W) < 1e-12 and d[1] > 0
