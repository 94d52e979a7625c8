"""Pins of the oracle's transient polarization tracking (Sec. 4.2, "Transient
polarization tracking": a Stokes vector per colour channel and time bin).

Readings (the paper defines the Stokes components but not the materials'
polarimetric models): emitters are unpolarised; Lambert is an ideal
depolariser; the GGX conductor reflects at its microfacet with the Fresnel
Mueller matrix of a complex index 1 + i kappa, kappa = 2 sqrt(F0 / (1 - F0)),
whose normal-incidence reflectance is F0; the camera's polariser axis x is the
camera's horizontal axis; S1 = I_x - I_y, S2 = I(+45) - I(-45) with y = k x x
for light travelling along k."""
import numpy as np
import pytest


def _conductor_plane(scenes_mod, f0=(0.9, 0.6, 0.3), rough=0.3):
    sc = scenes_mod.point_light_plane()
    sc.mtype[:] = 1
    sc.roughness[:] = rough
    sc.albedo[:] = np.array(f0, np.float32)
    return sc


def _fresnel_rs_rp(ci, f0):
    """Textbook Fresnel power reflectances of an interface from vacuum to n + i k."""
    kappa = 2.0 * np.sqrt(f0 / (1.0 - f0))
    N = 1.0 + 1j * kappa
    st2 = (1.0 - ci ** 2) / N ** 2
    ct = np.sqrt(1.0 - st2 + 0j)
    rs = (ci - N * ct) / (ci + N * ct)
    rp = (N * ci - ct) / (N * ci + ct)
    return np.abs(rs) ** 2, np.abs(rp) ** 2


def test_fresnel_reflectance_limits():
    for f0 in (0.3, 0.6, 0.95):
        rs, rp = _fresnel_rs_rp(1.0, f0)
        assert rs == pytest.approx(f0, rel=1e-12) and rp == pytest.approx(f0, rel=1e-12)
        rs, rp = _fresnel_rs_rp(1e-6, f0)
        assert rs > 0.999 and rp > 0.99
        ci = np.linspace(0.05, 0.95, 50)
        rs, rp = _fresnel_rs_rp(ci, f0)
        assert np.all(rs >= rp)  # s-polarised light is reflected more strongly


def test_lambertian_scene_stays_unpolarised(oracle_mod, scenes_mod):
    """An ideal depolariser everywhere: S1 = S2 = S3 = 0 exactly, S0 = the film."""
    sc = scenes_mod.cornell_box()
    assert np.all(sc.mtype == 0)
    osc = oracle_mod.OracleScene(sc)
    kw = dict(crop=(28, 36, 28, 36))
    pol = osc.render_polarized(64, 64, 64, 3.5, 0.05, 4, 17, 4, **kw)
    ref = osc.render(64, 64, 64, 3.5, 0.05, 4, 17, 4, **kw)
    assert np.all(pol["film"][:, :, :, 1:, :] == 0.0) and np.all(pol["steady"][:, :, 1:, :] == 0.0)
    assert np.allclose(pol["film"][:, :, :, 0, :], ref["film"], rtol=1e-12, atol=1e-16)
    assert np.allclose(pol["steady"][:, :, 0, :], ref["steady"], rtol=1e-12, atol=1e-16)


def test_single_conductor_reflection_closed_form(oracle_mod, scenes_mod):
    """Point light over a rough conductor, one bounce, pixel centres: the
    reflected light is partially polarised along s (perpendicular to the plane
    of incidence at the microfacet); in the camera frame
    S = k/2 (Rs + Rp, (Rs - Rp) cos 2t, -(Rs - Rp) sin 2t, 0), t the angle from s
    to the camera's x axis; relative to the unpolarised (Schlick) render
    S0 / C = ((Rs + Rp) / 2) / F_Schlick."""
    f0 = np.array([0.9, 0.6, 0.3])
    sc = _conductor_plane(scenes_mod, tuple(f0))
    osc = oracle_mod.OracleScene(sc)
    n = 8
    pol = osc.render_polarized(n, n, 4, 0.0, 100.0, 1, 3, 2, flags=oracle_mod.PIXEL_CENTER)
    ref = osc.render(n, n, 4, 0.0, 100.0, 1, 3, 2, flags=oracle_mod.PIXEL_CENTER)
    cam = sc.camera
    o = np.array(cam["origin"], np.float64)
    f = np.array(cam["target"], np.float64) - o
    f /= np.linalg.norm(f)
    r = np.cross(f, np.array(cam["up"], np.float64))
    r /= np.linalg.norm(r)
    L = np.array(sc.emitters[0]["position"], np.float64)
    checked = 0
    for py in range(n):
        for px in range(n):
            d = np.zeros(3)
            oo = np.zeros(3)
            oracle_mod.lib().mo_camera_ray(osc.h, n, n, px, py, 0.5, 0.5, oracle_mod._p(oo), oracle_mod._p(d))
            assert np.dot(d, r) * (px - (n - 1) / 2) >= -1e-12  # camera x axis points to increasing px
            S = pol["steady"][py, px]  # [4][3]
            C = ref["steady"][py, px]
            if C[0] <= 0:
                continue
            x = oo + d * (-oo[1] / d[1])
            wo = -d
            xo = x + np.array([0.0, 1.0, 0.0]) * 1e-4 * max(1.0, np.abs(x).max())  # shadow-ray origin offset
            wi = (L - xo) / np.linalg.norm(L - xo)
            h = (wo + wi) / np.linalg.norm(wo + wi)
            ci = np.dot(wi, h)
            rs, rp = _fresnel_rs_rp(ci, f0)
            schlick = f0 + (1 - f0) * (1 - ci) ** 5
            assert np.allclose(S[0] / C, 0.5 * (rs + rp) / schlick, rtol=1e-9)
            s = np.cross(wi, d)
            s /= np.linalg.norm(s)
            xc = r - np.dot(r, d) * d
            xc /= np.linalg.norm(xc)
            k = wo
            t = np.arctan2(np.dot(xc, np.cross(k, s)), np.dot(xc, s))
            dolp = (rs - rp) / (rs + rp)
            assert np.allclose(S[1] / S[0], dolp * np.cos(2 * t), atol=1e-9)
            assert np.allclose(S[2] / S[0], -dolp * np.sin(2 * t), atol=1e-9)
            assert np.all(S[3] == 0.0)
            checked += 1
    assert checked > n * n // 2


def test_degree_of_polarization_is_physical(oracle_mod, scenes_mod):
    """Cornell box with two conductor blocks (multiple specular bounces, so
    circular polarisation appears): every Stokes vector of the film has
    S0 >= |(S1, S2, S3)|, and the time-summed film equals the steady image."""
    sc = scenes_mod.cornell_box()
    sc.mtype[10:34] = 1
    sc.roughness[10:34] = 0.08
    sc.albedo[10:34] = np.clip(sc.albedo[10:34] + 0.3, 0, 0.95)
    osc = oracle_mod.OracleScene(sc)
    pol = osc.render_polarized(64, 64, 600, 0.0, 0.1, 16, 5, 6, crop=(24, 40, 24, 40))
    F, St = pol["film"], pol["steady"]
    pol_norm = np.sqrt((St[:, :, 1:, :] ** 2).sum(2))
    assert np.all(St[:, :, 0, :] >= pol_norm - 1e-12)
    assert (pol_norm > 1e-3 * St[:, :, 0, :]).mean() > 0.2   # conductors polarise a good share
    assert np.abs(St[:, :, 3, :]).max() > 0                   # and two reflections make circular light
    assert np.allclose(F.sum(2), St, rtol=1e-9, atol=1e-14)


def test_rotating_the_camera_rotates_the_linear_part(oracle_mod, scenes_mod):
    """Turning the camera by phi about its view axis turns its polariser axis
    by phi: at the centre pixel S0 and S3 stay, (S1, S2) rotates by 2 phi."""
    sc = _conductor_plane(scenes_mod, (0.8, 0.8, 0.8), 0.2)
    sc.camera = dict(origin=(0.0, 2.0, 1.5), target=(0.2, 0.0, -0.5), up=(0.0, 1.0, 0.0), fov_x_deg=30)
    n = 9
    base = None
    for phi in (0.0, 0.3, 1.1):
        f = np.array(sc.camera["target"]) - np.array(sc.camera["origin"])
        f /= np.linalg.norm(f)
        up0 = np.array([0.0, 1.0, 0.0])
        r0 = np.cross(f, up0)
        r0 /= np.linalg.norm(r0)
        u0 = np.cross(r0, f)
        up = np.cos(phi) * u0 - np.sin(phi) * r0
        sc.camera = dict(sc.camera, up=tuple(up))
        osc = oracle_mod.OracleScene(sc)
        S = osc.render_polarized(n, n, 4, 0.0, 100.0, 1, 2, 2, flags=oracle_mod.PIXEL_CENTER)["steady"][4, 4]
        z = S[1] + 1j * S[2]
        if base is None:
            base = (S, z)
            assert np.abs(z).min() > 1e-4 * S[0].min()
            continue
        S0, z0 = base
        assert np.allclose(S[0], S0[0], rtol=1e-12) and np.allclose(S[3], S0[3], atol=1e-15)
        assert np.allclose(np.abs(z), np.abs(z0), rtol=1e-10)
        ang = np.angle(z / z0)
        assert np.allclose(np.abs(np.angle(np.exp(1j * (np.abs(ang) - 2 * phi)))), 0.0, atol=1e-9), (phi, ang)


def test_reflection_on_the_continuation_path_closed_form(oracle_mod, scenes_mod):
    """Camera -> near-perfect conductor floor -> Lambertian wall lit by a point
    light: the wall depolarises, so what reaches the camera through the floor
    is one Fresnel reflection made on the continuation path (Mueller update and
    change of frame), not in a next-event estimate: S1/S0 and S2/S0 follow the
    same closed form as a single reflection at the mirror direction, S3 = 0;
    pixels that see the wall directly are unpolarised."""
    f0 = np.array([0.9, 0.6, 0.3])
    sc = scenes_mod.mirror_wall(tuple(f0))
    osc = oracle_mod.OracleScene(sc)
    n = 12
    st = osc.render_polarized(n, n, 4, 0.0, 100.0, 1, 9, 3, flags=oracle_mod.PIXEL_CENTER)["steady"]
    cam = sc.camera
    f = np.array(cam["target"], np.float64) - np.array(cam["origin"], np.float64)
    f /= np.linalg.norm(f)
    r = np.cross(f, np.array(cam["up"], np.float64))
    r /= np.linalg.norm(r)
    n_mirror = n_direct = 0
    errs = []
    for py in range(n):
        for px in range(n):
            d = np.zeros(3)
            o = np.zeros(3)
            oracle_mod.lib().mo_camera_ray(osc.h, n, n, px, py, 0.5, 0.5, oracle_mod._p(o), oracle_mod._p(d))
            S = st[py, px]
            t_floor = -o[1] / d[1] if d[1] < 0 else np.inf
            t_wall = (-3.0 - o[2]) / d[2] if d[2] < 0 else np.inf
            if S[0].min() <= 0:
                continue
            if t_wall < t_floor:
                assert np.all(S[1:] == 0.0)
                n_direct += 1
                continue
            wi = d * np.array([1.0, -1.0, 1.0])          # mirror direction off the floor
            ci = wi[1]                                    # microfacet normal ~ floor normal
            rs, rp = _fresnel_rs_rp(ci, f0)
            s = np.cross(wi, d)
            s /= np.linalg.norm(s)
            xc = r - np.dot(r, d) * d
            xc /= np.linalg.norm(xc)
            t = np.arctan2(np.dot(xc, np.cross(-d, s)), np.dot(xc, s))
            dolp = (rs - rp) / (rs + rp)
            errs.append(max(np.abs(S[1] / S[0] - dolp * np.cos(2 * t)).max(),
                            np.abs(S[2] / S[0] + dolp * np.sin(2 * t)).max()))
            assert np.abs(S[3]).max() <= 1e-6 * S[0].max()
            n_mirror += 1
    assert n_mirror > n * n // 3 and n_direct > 0
    # the floor's GGX (alpha 1e-4) scatters a few sampled directions by ~1e-3 rad (heavy tails);
    # a wrong frame or sign would be off by O(0.1 - 1)
    assert np.quantile(errs, 0.9) < 5e-4 and max(errs) < 2e-2, (np.quantile(errs, 0.9), max(errs))


def _jones_reflect(E, k_in, k_out, n, f0):
    """Reflect a complex 3-D field E (perpendicular to k_in) off a conductor of
    normal-incidence reflectance f0 (index 1 + i kappa): s = normal of the
    plane of incidence, p = k x s on each side (polarization ray tracing)."""
    s = np.cross(k_in, k_out)
    s /= np.linalg.norm(s)
    p_in, p_out = np.cross(k_in, s), np.cross(k_out, s)
    ci = -np.dot(k_in, n)
    kappa = 2.0 * np.sqrt(f0 / (1.0 - f0))
    N = 1.0 + 1j * kappa
    ct = np.sqrt(1.0 - (1.0 - ci ** 2) / N ** 2 + 0j)
    rs = (ci - N * ct) / (ci + N * ct)
    rp = (N * ci - ct) / (N * ci + ct)
    return rs * np.dot(E, s) * s + rp * np.dot(E, p_in) * p_out


def test_two_reflections_against_jones_calculus(oracle_mod, scenes_mod):
    """Camera -> conductor floor -> conductor back wall -> Lambertian ceiling
    lit by a point light: the Stokes vector the camera sees, computed with
    Mueller matrices and frame rotations in the oracle, equals the incoherent
    sum over two orthogonal polarisations leaving the ceiling of the fields
    reflected by the two conductors (3-D Jones calculus): S1/S0, S2/S0 and
    |S3|/S0 per colour."""
    f0a = np.array([0.9, 0.6, 0.3])
    f0b = np.array([0.5, 0.8, 0.95])
    sc = scenes_mod.mirror_corner(tuple(f0a), tuple(f0b))
    osc = oracle_mod.OracleScene(sc)
    n = 12
    st = osc.render_polarized(n, n, 4, 0.0, 100.0, 1, 4, 4, flags=oracle_mod.PIXEL_CENTER)["steady"]
    cam = sc.camera
    f = np.array(cam["target"], np.float64) - np.array(cam["origin"], np.float64)
    f /= np.linalg.norm(f)
    r = np.cross(f, np.array(cam["up"], np.float64))
    r /= np.linalg.norm(r)
    checked = 0
    errs = []
    for py in range(n):
        for px in range(n):
            d = np.zeros(3)
            o = np.zeros(3)
            oracle_mod.lib().mo_camera_ray(osc.h, n, n, px, py, 0.5, 0.5, oracle_mod._p(o), oracle_mod._p(d))
            if d[1] >= 0:
                continue
            x1 = o + d * (-o[1] / d[1])                   # floor
            d2 = d * np.array([1.0, -1.0, 1.0])
            if x1[2] <= -3.0 or d2[2] >= 0:
                continue
            x2 = x1 + d2 * ((-3.0 - x1[2]) / d2[2])       # back wall
            if not (0.0 < x2[1] < 6.0):
                continue
            d3 = d2 * np.array([1.0, 1.0, -1.0])
            if d3[1] <= 0:
                continue
            S = st[py, px]
            if S[0].min() <= 0:
                continue
            k1, k2, k3 = -d, -d2, -d3                     # propagation of the light, ceiling -> camera
            xc = r - np.dot(r, d) * d
            xc /= np.linalg.norm(xc)
            yc = np.cross(k1, xc)
            e1 = np.cross(k3, [0.3, 0.1, 0.9])
            e1 /= np.linalg.norm(e1)
            e2 = np.cross(k3, e1)
            for c in range(3):
                acc = np.zeros(4)
                for E in (e1.astype(complex), e2.astype(complex)):
                    Eb = _jones_reflect(E, k3, k2, np.array([0.0, 0.0, 1.0]), f0b[c])
                    Ea = _jones_reflect(Eb, k2, k1, np.array([0.0, 1.0, 0.0]), f0a[c])
                    ex, ey = np.dot(Ea, xc), np.dot(Ea, yc)
                    acc += [abs(ex) ** 2 + abs(ey) ** 2, abs(ex) ** 2 - abs(ey) ** 2,
                            2 * (ex * np.conj(ey)).real, 2 * (ex * np.conj(ey)).imag]
                got = S[:, c] / S[0, c]
                want = acc / acc[0]
                errs.append(max(np.abs(got[1:3] - want[1:3]).max(), abs(abs(got[3]) - abs(want[3]))))
            checked += 1
    assert checked > 10
    # near-specular GGX sampling (alpha 1e-4) perturbs a few paths by ~1e-3 rad; frame errors would be O(0.1 - 1)
    assert np.quantile(errs, 0.9) < 5e-4 and max(errs) < 2e-2, (np.quantile(errs, 0.9), max(errs))
