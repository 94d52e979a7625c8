"""Pins for the oracle's scattering functions (the rho factors of the impulse
response, Sec. 3 Eq. 8; materials Sec. 4.1): Lambertian, GGX conductor
(Smith height-correlated masking, Schlick Fresnel with F0 = albedo, visible
normal sampling) and the Henyey-Greenstein phase function."""
import numpy as np
import pytest

N = np.array([0.0, 0.0, 1.0])


def _dir(theta, phi):
    return np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])


def _hemi_quadrature(fn, n_t=200, n_p=200):
    """Midpoint rule over the upper hemisphere in (cos theta, phi)."""
    cs = (np.arange(n_t) + 0.5) / n_t
    ps = (np.arange(n_p) + 0.5) / n_p * 2 * np.pi
    acc = 0.0
    for c in cs:
        s = np.sqrt(1 - c * c)
        for p in ps:
            acc += fn(np.array([s * np.cos(p), s * np.sin(p), c]))
    return acc * (1.0 / n_t) * (2 * np.pi / n_p)


def test_lambert_closed_form(oracle_mod):
    alb = np.array([0.2, 0.5, 0.8])
    wo = _dir(0.3, 1.0)
    wi = _dir(0.9, -2.0)
    f, pdf = oracle_mod.bsdf_eval(0, alb, 0.0, N, wo, wi)
    assert np.allclose(f, alb / np.pi, rtol=1e-14)
    assert abs(pdf - wi[2] / np.pi) < 1e-14
    ok, wis, w, pdf2 = oracle_mod.bsdf_sample(0, alb, 0.0, N, wo, 0.37, 0.81)
    assert ok and np.allclose(w, alb, rtol=1e-12)
    # cosine mapping: z = sqrt(1 - u0), azimuth 2 pi u1 in the tangent frame
    assert abs(wis[2] - np.sqrt(1 - 0.37)) < 1e-12


def test_two_sided_flip(oracle_mod):
    """Geometry normal pointing away from wo: the oracle shades the other side."""
    alb = np.array([0.3, 0.3, 0.3])
    wo = _dir(0.4, 0.1)
    wi = _dir(0.7, 2.0)
    f1, p1 = oracle_mod.bsdf_eval(1, alb, 0.3, N, wo, wi)
    f2, p2 = oracle_mod.bsdf_eval(1, alb, 0.3, -N, wo, wi)
    assert np.allclose(f1, f2) and abs(p1 - p2) < 1e-15
    f3, _ = oracle_mod.bsdf_eval(0, alb, 0.0, N, wo, -wi)
    assert np.all(f3 == 0)


@pytest.mark.parametrize("alpha", [0.05, 0.2, 0.5])
def test_ggx_normal_incidence_closed_form(oracle_mod, alpha):
    """wo = wi = n: h = n, D(n) = 1/(pi a^2), G2 = 1, F = F0  =>  f = F0 / (4 pi a^2)."""
    F0 = np.array([0.5, 0.7, 1.0])
    f, pdf = oracle_mod.bsdf_eval(1, F0, alpha, N, N, N)
    assert np.allclose(f, F0 / (4 * np.pi * alpha ** 2), rtol=1e-12)
    assert abs(pdf - 1.0 / (4 * np.pi * alpha ** 2)) < 1e-9 * pdf


@pytest.mark.parametrize("alpha,theta", [(0.1, 0.5), (0.3, 1.1), (0.5, 1.3)])
def test_ggx_smith_and_schlick_closed_form(oracle_mod, alpha, theta):
    """Mirror configuration (h = n): pdf = G1(wo) D(n) / (4 cos) with the closed
    form G1 = 2 / (1 + sqrt(1 + a^2 tan^2)); Schlick scales channels by
    F0 + (1-F0)(1-cos)^5; G2 = 1 / (1 + 2 Lambda)."""
    F0 = np.array([0.2, 0.6, 1.0])
    wo = _dir(theta, 0.7)
    wi = np.array([-wo[0], -wo[1], wo[2]])
    f, pdf = oracle_mod.bsdf_eval(1, F0, alpha, N, wo, wi)
    t2 = np.tan(theta) ** 2
    G1 = 2.0 / (1.0 + np.sqrt(1.0 + alpha ** 2 * t2))
    D = 1.0 / (np.pi * alpha ** 2)
    assert abs(pdf - G1 * D / (4 * np.cos(theta))) < 1e-10 * pdf
    lam = (np.sqrt(1 + alpha ** 2 * t2) - 1) / 2
    F = F0 + (1 - F0) * (1 - np.cos(theta)) ** 5
    expect = D * F / (1 + 2 * lam) / (4 * np.cos(theta) ** 2)
    assert np.allclose(f, expect, rtol=1e-10)


@pytest.mark.parametrize("alpha", [0.08, 0.3, 0.5])
def test_ggx_reciprocity(oracle_mod, alpha):
    rng = np.random.default_rng(1)
    F0 = np.array([0.6, 0.8, 0.9])
    for _ in range(50):
        wo = _dir(rng.uniform(0, 1.5), rng.uniform(0, 6.28))
        wi = _dir(rng.uniform(0, 1.5), rng.uniform(0, 6.28))
        f1, _ = oracle_mod.bsdf_eval(1, F0, alpha, N, wo, wi)
        f2, _ = oracle_mod.bsdf_eval(1, F0, alpha, N, wi, wo)
        assert np.allclose(f1, f2, rtol=1e-12)


@pytest.mark.parametrize("alpha,theta", [(0.2, 0.3), (0.5, 1.0)])
def test_ggx_sampler_consistent_with_pdf_and_eval(oracle_mod, alpha, theta):
    """(1) the pdf integrates over the upper hemisphere to the fraction of valid
    samples; (2) white-furnace directional albedo (F0 = 1) from quadrature of
    f cos equals the mean sample weight and is <= 1 (single scattering loses energy)."""
    F0 = np.ones(3)
    wo = _dir(theta, 0.4)
    pdf_int = _hemi_quadrature(lambda w: oracle_mod.bsdf_eval(1, F0, alpha, N, wo, w)[1], 160, 160)
    alb_q = _hemi_quadrature(lambda w: oracle_mod.bsdf_eval(1, F0, alpha, N, wo, w)[0][0] * w[2], 160, 160)
    rng = np.random.default_rng(7)
    n = 20000
    valid = 0
    acc = 0.0
    for _ in range(n):
        ok, wi, w, p = oracle_mod.bsdf_sample(1, F0, alpha, N, wo, rng.random(), rng.random())
        if ok:
            valid += 1
            acc += w[0]
            fe, pe = oracle_mod.bsdf_eval(1, F0, alpha, N, wo, wi)
            assert abs(pe - p) < 1e-9 * p
    frac = valid / n
    assert abs(pdf_int - frac) < 4 * np.sqrt(frac * (1 - frac) / n) + 3e-3, (pdf_int, frac)
    assert alb_q <= 1.0 + 1e-3
    assert abs(acc / n - alb_q) < 0.01, (acc / n, alb_q)


@pytest.mark.parametrize("g", [0.0, 0.3, -0.5, 0.8])
def test_hg_normalised_and_mean_cosine(oracle_mod, g):
    """2 pi int p(c) dc = 1 and 2 pi int c p(c) dc = g (closed form for HG)."""
    n = 20000
    cc = (np.arange(n) + 0.5) / n * 2 - 1
    p = np.array([oracle_mod.hg_eval(g, x) for x in cc])
    dc = 2.0 / n
    assert abs(2 * np.pi * p.sum() * dc - 1) < 2e-3
    assert abs(2 * np.pi * (cc * p).sum() * dc - g) < 2e-3
    rng = np.random.default_rng(3)
    d = _dir(0.7, 0.2)
    cos = [oracle_mod.hg_sample(g, d, rng.random(), rng.random()) @ d for _ in range(8000)]
    sd = np.sqrt(max(np.var(cos), 1e-6) / len(cos))
    assert abs(np.mean(cos) - g) < 4 * sd
