"""Pins of the oracle's frequency-space rendering (Sec. 4.3, Eq. 12): each
contribution adds C * exp(-i 2 pi tof / lambda).  Reading: the phase is
2 pi * OPL / lambda with lambda in metres (the paper names Omega = 1/lambda)."""
import numpy as np
import pytest


def test_point_light_plane_phasor_closed_form(oracle_mod, scenes_mod):
    """One deterministic spike per pixel: phasor = L exp(-i 2 pi (d1 + d2) / lambda)."""
    sc = scenes_mod.point_light_plane()
    osc = oracle_mod.OracleScene(sc)
    lam = np.array([0.2, 0.133, 0.066])
    H = W = 8
    out = osc.render_phasor(H, W, lam, spp=1, seed=7, max_depth=2, flags=oracle_mod.PIXEL_CENTER)
    tr = osc.render(H, W, 2000, 0.0, 0.005, spp=1, seed=7, max_depth=2, flags=oracle_mod.PIXEL_CENTER,
                    dump_cap=1000)
    d = tr["dump"]
    assert len(d) == H * W
    for r in d:
        py, px = divmod(int(r["pixel"]), W)
        for q, l in enumerate(lam):
            z = out["phasor"][py, px, q, 0] + 1j * out["phasor"][py, px, q, 1]
            expect = r["c"] * np.exp(-2j * np.pi * r["opl"] / l)
            assert np.allclose(z, expect, rtol=1e-12, atol=1e-15)


def test_phasor_is_the_limit_of_the_binned_dft(oracle_mod, scenes_mod):
    """The DFT of a finely binned transient film approaches the phasor as the
    bin width shrinks (the naive alternative the paper describes)."""
    sc = scenes_mod.cornell_box()
    osc = oracle_mod.OracleScene(sc)
    lam = np.array([0.2, 0.066])
    kw = dict(spp=4, seed=31, max_depth=3, crop=(28, 32, 28, 32))
    out = osc.render_phasor(64, 64, lam, **kw)
    ph, st = out["phasor"], out["steady"]
    errs = []
    for w in (0.004, 0.001, 0.00025):
        T = int(np.ceil(12.0 / w))
        f = osc.render(64, 64, T, 3.0, w, **kw)["film"]
        centres = 3.0 + (np.arange(T) + 0.5) * w
        e = []
        for q, l in enumerate(lam):
            kern = np.exp(-2j * np.pi * centres / l)
            dft = np.einsum("yxtc,t->yxc", f, kern)
            z = ph[:, :, q, 0] + 1j * ph[:, :, q, 1]
            # |sum C (e^{-i phi'} - e^{-i phi})| <= (max |phi' - phi|) sum C = (pi w / lambda) * steady
            e.append((np.abs(dft - z) / st).max())
        errs.append(max(e))
    # each contribution's phase is off by at most pi * w / lambda when the DFT
    # uses bin centres, so the error is bounded by that and shrinks with w
    for w, e in zip((0.004, 0.001, 0.00025), errs):
        assert e <= np.pi * w / lam.min(), (w, e)
    assert errs[0] > errs[1] > errs[2], errs


def test_phasor_bounds_and_long_wavelength_limit(oracle_mod, scenes_mod):
    sc = scenes_mod.cornell_box()
    osc = oracle_mod.OracleScene(sc)
    out = osc.render_phasor(64, 64, np.array([0.1, 1e9]), spp=4, seed=5, max_depth=4, crop=(20, 40, 20, 40))
    ph, st = out["phasor"], out["steady"]
    mag = np.hypot(ph[..., 0, :], ph[..., 1, :])
    assert np.all(mag[:, :, 0] <= st + 1e-12)       # |sum C e^{i phi}| <= sum C
    assert np.allclose(ph[:, :, 1, 0], st, rtol=1e-12)  # lambda -> infinity: the steady image
    assert np.abs(ph[:, :, 1, 1]).max() < 1e-7 * st.max()
