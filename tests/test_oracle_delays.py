"""Pins of the oracle's time-resolved materials and sources (Sec. 4.1 scattering
delays; Sec. 3 emission L_e(t), Eq. 5 generalised from a delta pulse).

Readings: a surface vertex with delay mean tau re-emits the light it received
after dt ~ Exp(tau) (tau in metres of light travel, c = 1); the delay density
has unit area, so steady-state values do not change.  The source pulse p(t)
has unit area and shifts every contribution by an independent emission time.
Both are sampled (one draw per vertex / per contribution), so the film is an
unbiased estimate of the impulse response convolved with them."""
import numpy as np
import pytest
from scipy import special, stats


def _spike(oracle_mod, scenes_mod, px=8):
    """Point light over a Lambertian plane, pixel centres, one bounce: per pixel
    one deterministic contribution (c, opl) (pinned to its closed form in
    test_oracle_closed_forms)."""
    sc = scenes_mod.point_light_plane()
    osc = oracle_mod.OracleScene(sc)
    ref = osc.render(px, px, 4, 0.0, 1.0, 1, 3, 2, flags=oracle_mod.PIXEL_CENTER, dump_cap=10 * px * px)
    d = ref["dump"]
    assert len(d) == px * px and np.all(d["kind"] == 1)
    return sc, osc, d


def _check_bins(film_px, c, probs, n):
    """The estimate (1/n) sum c 1[bin] holds whole sample counts per bin; they
    must follow the multinomial of the bin probabilities p_k (chi-square
    goodness of fit, bins with fewer than 5 expected samples pooled, the mass
    outside the window as one more cell)."""
    counts = film_px * n / c
    assert np.allclose(counts, np.rint(counts), atol=1e-6)
    counts = np.rint(counts)
    exp = n * probs
    big = exp >= 5
    obs = np.concatenate([counts[big], [counts[~big].sum(), n - counts.sum()]])
    ex = np.concatenate([exp[big], [exp[~big].sum(), n * (1 - probs.sum())]])
    keep = ex > 0
    assert np.all(obs[~keep] == 0)
    obs, ex = obs[keep], ex[keep]
    p = stats.chisquare(obs, ex * obs.sum() / ex.sum()).pvalue
    assert p > 1e-4, p
    assert abs(obs.sum() - n) < 1e-9


@pytest.mark.parametrize("tau", [0.03, 0.11])
def test_exponential_delay_closed_form(oracle_mod, scenes_mod, tau):
    """One delayed vertex: the spike at t0 becomes c * Exp(tau) shifted by t0,
    so bin k holds c (F(b_k - t0) - F(a_k - t0)) with F(x) = 1 - exp(-x / tau)."""
    px, n = 8, 4000
    sc, osc, d = _spike(oracle_mod, scenes_mod, px)
    osc.set_delays(np.full(sc.n_tris, tau))
    t0min = d["opl"].min()
    start, width, T = t0min - 0.05, 0.01, 160
    crop = (2, 6, 2, 6)
    out = osc.render(px, px, T, start, width, n, 11, 2, flags=oracle_mod.PIXEL_CENTER, crop=crop)
    edges = start + width * np.arange(T + 1)
    for r in d:
        y, x = divmod(int(r["pixel"]), px)
        if not (crop[0] <= x < crop[1] and crop[2] <= y < crop[3]):
            continue
        F = np.where(edges > r["opl"], 1 - np.exp(-(edges - r["opl"]) / tau), 0.0)
        probs = np.diff(F)
        _check_bins(out["film"][y - crop[2], x - crop[0], :, 0], r["c"][0], probs, n)
        # unit-area delay density: the steady value is the undelayed spike exactly
        assert out["steady"][y - crop[2], x - crop[0], 0] == pytest.approx(r["c"][0], rel=1e-12)


@pytest.mark.parametrize("kind,a,b", [(1, 0.07, 0.0), (2, 0.05, 0.02), (3, 0.04, 0.0)])
def test_emission_pulse_closed_forms(oracle_mod, scenes_mod, kind, a, b):
    """Box [0, a), Gaussian (a, b) and exponential (mean a) pulses convolve the
    spike: bin k holds c times the pulse's probability of [a_k - t0, b_k - t0)."""
    px, n = 8, 4000
    sc, osc, d = _spike(oracle_mod, scenes_mod, px)
    osc.set_pulse(kind, a, b)
    t0min = d["opl"].min()
    start, width, T = t0min - 0.1, 0.01, 160
    crop = (3, 5, 3, 5)
    out = osc.render(px, px, T, start, width, n, 5, 2, flags=oracle_mod.PIXEL_CENTER, crop=crop)
    edges = start + width * np.arange(T + 1)
    for r in d:
        y, x = divmod(int(r["pixel"]), px)
        if not (crop[0] <= x < crop[1] and crop[2] <= y < crop[3]):
            continue
        s = edges - r["opl"]
        if kind == 1:
            F = np.clip(s / a, 0.0, 1.0)
        elif kind == 2:
            F = 0.5 * (1 + special.erf((s - a) / (b * np.sqrt(2))))
        else:
            F = np.where(s > 0, 1 - np.exp(-s / a), 0.0)
        _check_bins(out["film"][y - crop[2], x - crop[0], :, 0], r["c"][0], np.diff(F), n)


def test_delays_leave_steady_and_contributions_unchanged(oracle_mod, scenes_mod):
    """Same seed with and without delays / pulse: every contribution keeps its
    value (delays and emission times use their own random numbers), so the
    steady image is identical; a window covering all times gives T-sum = steady."""
    sc = scenes_mod.cornell_box()
    osc = oracle_mod.OracleScene(sc)
    kw = dict(crop=(28, 36, 28, 36), dump_cap=200000)
    a = osc.render(64, 64, 64, 3.5, 0.05, 8, 21, 4, **kw)
    rng = np.random.default_rng(2)
    osc.set_delays(rng.uniform(0.0, 0.2, sc.n_tris))
    osc.set_pulse(2, 0.1, 0.03)
    b = osc.render(64, 64, 64, 3.5, 0.05, 8, 21, 4, **kw)
    assert np.array_equal(a["steady"], b["steady"])
    da, db = a["dump"], b["dump"]
    assert len(da) == len(db) and np.array_equal(da["c"], db["c"]) and np.array_equal(da["depth"], db["depth"])
    assert np.all(db["opl"] > da["opl"] - 0.2)  # Gaussian emission times can be slightly negative
    c = osc.render(64, 64, 4000, 0.0, 0.01, 8, 21, 4, crop=(28, 36, 28, 36))
    assert np.allclose(c["film"].sum(2), c["steady"], rtol=1e-12, atol=1e-15)


def test_delay_accounting_per_vertex(oracle_mod, scenes_mod):
    """With one delay mean tau on every surface, a next-event contribution made
    at vertex j carries the delays of vertices 1..j (Gamma(j, tau)) and light
    found at vertex j those of 1..j-1 (Gamma(j-1, tau); none for direct view)."""
    tau = 0.05
    sc = scenes_mod.cornell_box()
    osc = oracle_mod.OracleScene(sc)
    kw = dict(crop=(16, 48, 16, 48), dump_cap=400000)
    a = osc.render(64, 64, 16, 3.5, 0.5, 8, 9, 4, **kw)["dump"]
    osc.set_delays(np.full(sc.n_tris, tau))
    b = osc.render(64, 64, 16, 3.5, 0.5, 8, 9, 4, **kw)["dump"]

    def key(r):
        return (r["pixel"].astype(np.int64) << 32) | (r["sample"].astype(np.int64) << 12) | \
               (r["depth"].astype(np.int64) << 2) | r["kind"].astype(np.int64)

    ka, kb = key(a), key(b)
    ia, ib = np.argsort(ka), np.argsort(kb)
    assert np.array_equal(ka[ia], kb[ib])
    a, b = a[ia], b[ib]
    dt = b["opl"] - a["opl"]
    nv = np.where(b["kind"] == 1, b["depth"], b["depth"] - 1)
    assert np.all(dt[nv == 0] == 0.0)
    for j in range(1, 4):
        sel = dt[nv == j]
        assert len(sel) > 300, (j, len(sel))
        p = stats.kstest(sel, stats.gamma(a=j, scale=tau).cdf).pvalue
        assert p > 1e-3, (j, p)
    # a plausible slip (the vertex's own delay missing from its next-event
    # estimate) is rejected by the same test
    wrong = dt[(nv == 2)]
    assert stats.kstest(wrong, stats.gamma(a=1, scale=tau).cdf).pvalue < 1e-6


def test_bad_delay_and_pulse_parameters(oracle_mod, scenes_mod):
    sc = scenes_mod.cornell_box()
    osc = oracle_mod.OracleScene(sc)
    with pytest.raises(ValueError):
        osc.set_delays(np.full(sc.n_tris, -1.0))
    with pytest.raises(ValueError):
        osc.set_delays(np.full(sc.n_tris - 1, 0.1))
    with pytest.raises(ValueError):
        osc.set_pulse(1, 0.0)
    with pytest.raises(ValueError):
        osc.set_pulse(2, 0.1, 0.0)
    with pytest.raises(ValueError):
        osc.set_pulse(7, 0.1, 0.1)
