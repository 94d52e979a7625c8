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
