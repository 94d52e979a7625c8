"""GPU parity of scattering delays (Sec. 4.1) and emission pulses (Sec. 3,
Eq. 5 with a pulse of unit area): the same Philox draws as the oracle, so
contributions match one by one, their times within FP32 rounding."""
import numpy as np
import pytest

from gpu_util import build_and_load, match_contribs, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cornell(oracle_mod, scenes_mod):
    import torch
    api = build_and_load()
    sc = scenes_mod.cornell_box()
    tau = np.random.default_rng(4).uniform(0.0, 0.15, sc.n_tris)
    tau[::5] = 0.0
    s = api.Scene(sc)
    s.set_delays(torch.from_numpy(tau.astype(np.float32)).cuda())
    s.set_pulse(api.MT_PULSE_GAUSSIAN, 0.06, 0.02)
    osc = oracle_mod.OracleScene(sc)
    osc.set_delays(tau.astype(np.float32).astype(np.float64))
    osc.set_pulse(2, np.float32(0.06), np.float32(0.02))
    return api, sc, s, osc


@pytest.mark.parametrize("form", ["megakernel", "wavefront"])
def test_delayed_contributions_match_oracle(cornell, form):
    api, sc, s, osc = cornell
    H = W = 64
    T, start, width = 256, 3.5, 0.01
    spp, seed, depth = 4, 25660, 4
    if form == "wavefront":
        s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT)
    try:
        film, steady, rec, n = api.render_dump(s, H, W, T, start, width, spp, seed, depth, cap=2_000_000)
        f2, s2 = api.render(s, H, W, T, start, width, 16, seed, depth)
        s.sync()
    finally:
        s.set_launch(api.MT_LAUNCH_RENDER)
    crop = (16, 48, 16, 48)
    ref = osc.render(H, W, T, start, width, spp, seed, depth, crop=crop, dump_cap=2_000_000)
    px, py = rec["pixel"] % W, rec["pixel"] // W
    sel = (px >= crop[0]) & (px < crop[1]) & (py >= crop[2]) & (py < crop[3])
    nm, div, worst, bad, bin_bad, dopl = match_contribs(rec[sel], ref["dump"], start=start, width=width)
    assert nm > 3000 and div <= 1e-4 * nm and bad <= 1e-3 * nm and bin_bad == 0, (nm, div, bad, bin_bad)
    assert np.quantile(dopl, 0.999) < 2e-5
    ref16 = osc.render(H, W, T, start, width, 16, seed, depth, crop=(24, 40, 24, 40))
    g = f2.cpu().numpy()[24:40, 24:40]
    assert rel_l2(g, ref16["film"]) < 0.01
    assert rel_l2(s2.cpu().numpy()[24:40, 24:40], ref16["steady"]) < 0.01


def test_delays_shift_time_not_steady(cornell):
    """Same seed with and without delays and pulse: the steady image agrees to
    FP32 summation order, the mean arrival time moves later."""
    api, sc, s, osc = cornell
    H = W = 64
    T, start, width = 512, 3.0, 0.01
    f1, s1 = api.render(s, H, W, T, start, width, 8, 3, 4)
    s.set_delays(None)
    s.set_pulse(api.MT_PULSE_DELTA)
    try:
        f0, s0 = api.render(s, H, W, T, start, width, 8, 3, 4)
        s.sync()
    finally:
        import torch
        tau = np.random.default_rng(4).uniform(0.0, 0.15, sc.n_tris)
        tau[::5] = 0.0
        s.set_delays(torch.from_numpy(tau.astype(np.float32)).cuda())
        s.set_pulse(api.MT_PULSE_GAUSSIAN, 0.06, 0.02)
    assert rel_l2(s1.cpu().numpy(), s0.cpu().numpy()) < 1e-5
    t = start + width * (np.arange(T) + 0.5)
    m1 = (f1.sum((0, 1, 3)).cpu().numpy() * t).sum() / f1.sum().item()
    m0 = (f0.sum((0, 1, 3)).cpu().numpy() * t).sum() / f0.sum().item()
    assert m1 > m0 + 0.06


def test_delayed_backward_matches_oracle(cornell):
    import torch
    api, sc, s, osc = cornell
    H = W = 32
    T, start, width = 128, 3.5, 0.02
    spp, seed, depth = 4, 8, 4
    g = np.random.default_rng(5).uniform(-1, 1, (H, W, T, 3))
    ga, gr, gm = api.render_backward(s, T, start, width, spp, seed, depth, torch.from_numpy(g.astype(np.float32)).cuda())
    ref = osc.render_backward(H, W, T, start, width, spp, seed, depth, g)
    assert np.linalg.norm(ga.cpu().numpy() - ref["albedo"]) < 0.02 * np.linalg.norm(ref["albedo"])
    assert np.linalg.norm(gr.cpu().numpy() - ref["radiance"]) < 0.02 * np.linalg.norm(ref["radiance"])


def test_delayed_phasor_matches_oracle(cornell):
    api, sc, s, osc = cornell
    lam = np.array([0.2, 0.05])
    ph, st = api.render_phasor(s, 64, 64, lam, 8, 2, 4)
    ref = osc.render_phasor(64, 64, lam, spp=8, seed=2, max_depth=4, crop=(24, 40, 24, 40))
    g = ph.cpu().numpy().reshape(64, 64, 2, 2, 3)[24:40, 24:40]
    assert rel_l2(g, ref["phasor"]) < 0.01


def test_bad_delay_and_pulse_arguments(cornell):
    import torch
    api, sc, s, osc = cornell
    with pytest.raises(api.MtError) as e:
        s.set_delays(torch.full((sc.n_tris,), -1.0, device="cuda"))
    assert e.value.status == api.MT_ERR_INVALID_ARGUMENT
    with pytest.raises(api.MtError):
        s.set_pulse(api.MT_PULSE_BOX, 0.0)
    with pytest.raises(api.MtError):
        s.set_pulse(9, 0.1, 0.1)
