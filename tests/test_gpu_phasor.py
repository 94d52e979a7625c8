"""GPU frequency-space rendering (Sec. 4.3, Eq. 12) against the oracle on the
same Philox stream, and the single-spike closed form."""
import numpy as np
import pytest

from gpu_util import build_and_load, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["megakernel", "wavefront"])
def test_phasor_matches_oracle(oracle_mod, scenes_mod, form):
    api = build_and_load()
    sc = scenes_mod.cornell_box()
    s = api.Scene(sc)
    if form == "wavefront":
        s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT)
    lam = np.array([0.2, 0.133, 0.066])
    ph, st = api.render_phasor(s, 64, 64, lam, spp=8, seed=3, max_depth=4)
    s.sync()
    crop = (24, 40, 24, 40)
    ref = oracle_mod.OracleScene(sc).render_phasor(64, 64, lam, spp=8, seed=3, max_depth=4, crop=crop)
    g = ph.cpu().numpy()[crop[2]:crop[3], crop[0]:crop[1]]
    assert rel_l2(g, ref["phasor"]) < 1e-3
    assert rel_l2(st.cpu().numpy()[crop[2]:crop[3], crop[0]:crop[1]], ref["steady"]) < 1e-4


def test_phasor_point_light_closed_form(oracle_mod, scenes_mod):
    api = build_and_load()
    sc = scenes_mod.point_light_plane()
    s = api.Scene(sc)
    lam = np.array([0.2, 0.066])
    ph, st = api.render_phasor(s, 16, 16, lam, spp=1, seed=7, max_depth=2, flags=api.MT_PIXEL_CENTER)
    s.sync()
    ref = oracle_mod.OracleScene(sc).render_phasor(16, 16, lam, spp=1, seed=7, max_depth=2,
                                                   flags=oracle_mod.PIXEL_CENTER)
    g = ph.cpu().numpy()
    z = g[..., 0, :] + 1j * g[..., 1, :]
    zr = ref["phasor"][..., 0, :] + 1j * ref["phasor"][..., 1, :]
    assert np.abs(z - zr).max() < 2e-4 * np.abs(zr).max()
