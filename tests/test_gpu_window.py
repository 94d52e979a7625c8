"""Film windows: a frame rendered band by band (each band a window of the
frame: same camera rays and per-pixel random numbers) equals the frame
rendered at once, in every form."""
import numpy as np
import pytest

from gpu_util import build_and_load, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["megakernel", "wavefront"])
def test_banded_render_equals_full(scenes_mod, form):
    import torch
    api = build_and_load()
    sc = scenes_mod.cornell_box()
    s = api.Scene(sc)
    if form == "wavefront":
        s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT)
    H = W = 64
    T, start, width = 256, 3.5, 0.01
    full, fs = api.render(s, H, W, T, start, width, 8, 3, 4)
    film, steady = api.new_film(H, W, T)
    for r0, r1 in ((0, 16), (16, 40), (40, 41), (41, 64)):
        api.render(s, r1 - r0, W, T, start, width, 8, 3, 4, out=(film[r0:r1], steady[r0:r1]), window=(H, r0))
    s.sync()
    assert rel_l2(film.cpu().numpy(), full.cpu().numpy()) < 1e-6
    assert rel_l2(steady.cpu().numpy(), fs.cpu().numpy()) < 1e-6


def test_banded_dump_records_carry_frame_pixels(scenes_mod):
    api = build_and_load()
    sc = scenes_mod.cornell_box()
    s = api.Scene(sc)
    H = W = 32
    _, _, full, _ = api.render_dump(s, H, W, 64, 3.5, 0.04, 2, 5, 4, cap=200000)
    _, _, band, _ = api.render_dump(s, 8, W, 64, 3.5, 0.04, 2, 5, 4, cap=200000, window=(H, 12))
    sel = (full["pixel"] // W >= 12) & (full["pixel"] // W < 20)
    key = lambda r: np.sort((r["pixel"].astype(np.int64) << 32) | (r["sample"].astype(np.int64) << 12) |
                            (r["depth"].astype(np.int64) << 2) | r["kind"])
    assert np.array_equal(key(full[sel]), key(band))


def test_banded_polarized_equals_full(scenes_mod):
    import torch
    api = build_and_load()
    sc = scenes_mod.mirror_corner()
    s = api.Scene(sc)
    H = W = 32
    pf, ps = api.render_polarized(s, H, W, 8, 0.0, 5.0, 2, 1, 4)
    bf = torch.empty_like(pf)
    bs = torch.empty_like(ps)
    for r0 in range(0, H, 8):
        api.render_polarized(s, 8, W, 8, 0.0, 5.0, 2, 1, 4, out=(bf[r0:r0 + 8], bs[r0:r0 + 8]), window=(H, r0))
    s.sync()
    assert rel_l2(bs.cpu().numpy(), ps.cpu().numpy()) < 1e-6


def test_window_must_fit(scenes_mod):
    api = build_and_load()
    s = api.Scene(scenes_mod.cornell_box())
    with pytest.raises(api.MtError):
        api.render(s, 16, 16, 8, 3.5, 0.1, 1, 1, 2, window=(20, 8))
