"""mt_render_to_host: the render with its film and steady image copied to host
memory band by band as the bands finish (the wavefront form in queue order
flags a band once all its paths and their shadow rays are done).  The host
arrays equal the device film of the same render, for band heights that divide
the frame or not, one band, one row per band, a windowed film, the persistent
form (copies after the render) and the refilled small pool; argument errors."""
import numpy as np
import pytest

from gpu_util import build_and_load, rel_l2

pytestmark = pytest.mark.gpu

T, START, WIDTH = 256, 3.5, 0.01


@pytest.fixture(scope="module")
def cornell(scenes_mod):
    api = build_and_load()
    sc = scenes_mod.cornell_box()
    s = api.Scene(sc)
    s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT)
    return api, sc, s


def _host(H, W):
    import torch
    return (torch.zeros((H, W, T, 3), dtype=torch.float32, pin_memory=True),
            torch.zeros((H, W, 3), dtype=torch.float32, pin_memory=True))


@pytest.mark.parametrize("band_rows", [8, 5, 1, 64, 100])
def test_bands_equal_the_device_film(cornell, band_rows):
    import torch
    api, sc, s = cornell
    H = W = 64
    spp, seed, depth = 16, 25660, 4
    cp = torch.cuda.Stream()
    hf, hs = _host(H, W)
    film, steady = api.render_to_host(s, H, W, T, START, WIDTH, spp, seed, depth, hf, hs, band_rows, cp)
    cp.synchronize()
    torch.cuda.synchronize()
    assert np.abs(hf.numpy()).max() > 0
    # the host copy is the device film of this render ...
    assert np.array_equal(hf.numpy(), film.cpu().numpy())
    assert np.array_equal(hs.numpy(), steady.cpu().numpy())
    # ... which is mt_render's film up to the order of the atomic additions
    f2, s2 = api.render(s, H, W, T, START, WIDTH, spp, seed, depth)
    assert rel_l2(hf.numpy(), f2.cpu().numpy()) < 1e-6
    assert rel_l2(hs.numpy(), s2.cpu().numpy()) < 1e-6


def test_small_pool_window_and_persistent_form(cornell):
    import torch
    api, sc, s = cornell
    H, W = 40, 48
    spp, seed, depth = 8, 3, 4
    cp = torch.cuda.Stream()
    # a window of a taller frame, through a pool refilled many times
    s.set_wavefront_pool(512)
    try:
        hf, hs = _host(H, W)
        film, steady = api.render_to_host(s, H, W, T, START, WIDTH, spp, seed, depth, hf, hs, 7, cp,
                                          window=(100, 30))
        cp.synchronize()
        torch.cuda.synchronize()
        ref, ref_s = api.render(s, H, W, T, START, WIDTH, spp, seed, depth, window=(100, 30))
        torch.cuda.synchronize()
    finally:
        s.set_wavefront_pool(0)
    assert np.array_equal(hf.numpy(), film.cpu().numpy())
    assert rel_l2(hf.numpy(), ref.cpu().numpy()) < 1e-6 and rel_l2(hs.numpy(), ref_s.cpu().numpy()) < 1e-6
    # the persistent form: every band after the render
    s.set_launch(api.MT_LAUNCH_RENDER)
    try:
        hf2, hs2 = _host(H, W)
        film2, steady2 = api.render_to_host(s, H, W, T, START, WIDTH, spp, seed, depth, hf2, hs2, 16, cp)
        cp.synchronize()
        torch.cuda.synchronize()
    finally:
        s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, api.MT_OPT_WAVEFRONT)
    assert np.array_equal(hf2.numpy(), film2.cpu().numpy())
    assert np.array_equal(hs2.numpy(), steady2.cpu().numpy())


def test_back_to_back_calls_reuse_the_film(cornell):
    """A second call on the same device film, ordered after the first call's
    copies, and the bands of a frame rendered as windows of one film."""
    import torch
    api, sc, s = cornell
    H = W = 64
    cp = torch.cuda.Stream()
    out = api.new_film(H, W, T)
    hosts = [_host(H, W), _host(H, W)]
    for k, (hf, hs) in enumerate(hosts):
        torch.cuda.current_stream().wait_stream(cp)  # the film is cleared after the last call's copies
        api.render_to_host(s, H, W, T, START, WIDTH, 8, 100 + k, 4, hf, hs, 16, cp, out=out)
    cp.synchronize()
    torch.cuda.synchronize()
    for k, (hf, hs) in enumerate(hosts):
        ref, ref_s = api.render(s, H, W, T, START, WIDTH, 8, 100 + k, 4)
        assert rel_l2(hf.numpy(), ref.cpu().numpy()) < 1e-6
        assert rel_l2(hs.numpy(), ref_s.cpu().numpy()) < 1e-6
    # a frame as three windows (40, 16, 8 rows) of one film, each streamed: the windows' renders
    # follow one another on the render stream while earlier windows' copies run
    hf, hs = _host(H, W)
    r0 = 0
    for rows in (40, 16, 8):
        api.render_to_host(s, rows, W, T, START, WIDTH, 8, 7, 4, hf[r0:r0 + rows], hs[r0:r0 + rows], 8, cp,
                           out=(out[0][r0:r0 + rows], out[1][r0:r0 + rows]), window=(H, r0))
        r0 += rows
    cp.synchronize()
    torch.cuda.synchronize()
    ref, ref_s = api.render(s, H, W, T, START, WIDTH, 8, 7, 4)
    assert rel_l2(hf.numpy(), ref.cpu().numpy()) < 1e-6
    assert rel_l2(hs.numpy(), ref_s.cpu().numpy()) < 1e-6


def test_argument_errors(cornell):
    import torch
    api, sc, s = cornell
    H = W = 16
    film, steady = api.new_film(H, W, T)
    f = api.Film(film, steady, START, WIDTH)
    hf, hs = _host(H, W)
    cp = torch.cuda.Stream()
    st = api._stream(None)
    for args in ((0, hf, hs, cp), (4, None, hs, cp), (4, hf, None, cp), (1, hf, hs, cp)):
        rows, a, b, c = args
        stream_c = api._stream(c)
        with pytest.raises(api.MtError) as e:
            if rows == 1:  # copy stream equal to the render stream
                api.mt_render_to_host(s.h, f.h, 4, 1, 4, 0, 4, api._hptr(a), api._hptr(b), st, st)
            else:
                api.mt_render_to_host(s.h, f.h, 4, 1, 4, 0, rows, api._hptr(a), api._hptr(b), st, stream_c)
        assert e.value.status == api.MT_ERR_INVALID_ARGUMENT
