"""Argument checks of the Python binding that run before any pointer reaches
the C ABI (no GPU): a film whose dtype, size or device does not match what the
kernels write is refused with ValueError, also under `python -O`."""
import pytest
import torch

from paper_2510_25660_gb300 import api


def test_film_dtype_and_size_are_checked_before_the_library():
    H, W, T = 2, 3, 4
    with pytest.raises(ValueError, match="float32"):
        api.Film(torch.zeros((H, W, T, 3), dtype=torch.float16), None, 0.0, 1.0)
    with pytest.raises(ValueError, match="steady image holds"):
        api.Film(torch.zeros((H, W, T, 3)), torch.zeros((H, W, 1)), 0.0, 1.0)
    with pytest.raises(ValueError, match="steady image must be float32"):
        api.Film(torch.zeros((H, W, T, 3)), torch.zeros((H, W, 3), dtype=torch.float64), 0.0, 1.0)
    with pytest.raises(ValueError, match=r"\[H, W, T, C\]"):
        api.Film(torch.zeros((H, W, T)), None, 0.0, 1.0)
    # Stokes films: 12 values per bin in trailing dimensions
    with pytest.raises(ValueError, match="film holds"):
        api.Film(torch.zeros((H, W, T, 4, 2)), None, 0.0, 1.0, C_=12)
    # right dtype and sizes, but host memory
    with pytest.raises(ValueError, match="CUDA"):
        api.Film(torch.zeros((H, W, T, 3)), torch.zeros((H, W, 3)), 0.0, 1.0)
    with pytest.raises(ValueError, match="CUDA"):
        api.Film(torch.zeros((H, W, T, 4, 3)), torch.zeros((H, W, 4, 3)), 0.0, 1.0, C_=12)


def test_pointer_helpers_refuse_the_wrong_memory():
    with pytest.raises(ValueError, match="CUDA"):
        api._ptr(torch.zeros(4))
    assert api._ptr(None) is None
    with pytest.raises(ValueError, match="host float32"):
        api._hptr(torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError, match="host float32"):
        api._hptr(torch.zeros((4, 4)).t())
    assert api._hptr(torch.zeros(4)).value != 0


def test_parameter_buffers_are_checked_before_the_library():
    import types
    scene = types.SimpleNamespace(n_tris=5, n_em=2, h=None)
    with pytest.raises(ValueError, match="albedo must be float32"):
        api.Scene.set_params(scene, albedo=torch.zeros((5, 3), dtype=torch.float64))
    with pytest.raises(ValueError, match="albedo holds 12 values where 15"):
        api.Scene.set_params(scene, albedo=torch.zeros((4, 3)))
    with pytest.raises(ValueError, match="radiance holds 3 values where 6"):
        api.Scene.set_params(scene, radiance=torch.zeros((1, 3)))
    with pytest.raises(ValueError, match="medium albedo holds"):
        api.Scene.set_params(scene, medium_albedo=torch.zeros(2))
    with pytest.raises(ValueError, match="CUDA"):
        api.Scene.set_params(scene, albedo=torch.zeros((5, 3)), radiance=torch.zeros((2, 3)))
    # larger gradient accumulators are accepted, smaller ones are not
    with pytest.raises(ValueError, match="gradient holds 2 values where 3"):
        api._check_f32([(torch.zeros(2), 3, "gradient")], at_least=True)
    with pytest.raises(ValueError, match="CUDA"):
        api._check_f32([(torch.zeros(6), 3, "gradient"), (None, 9, "skipped")], at_least=True)


def test_scan_points_are_checked_before_the_library():
    wall = dict(normal=(0.0, 0.0, 1.0), albedo=0.8)
    with pytest.raises(ValueError, match=r"laser points must be \[n, 3\]"):
        api.make_scan(torch.zeros((4, 2)), None, api.MT_CONFOCAL, wall["normal"], wall["albedo"], (0, 1))
    with pytest.raises(ValueError, match="sensor points must be float32"):
        api.make_scan(torch.zeros((4, 3)), torch.zeros((2, 3), dtype=torch.float64), api.MT_EXHAUSTIVE,
                      wall["normal"], wall["albedo"], (0, 1))
    with pytest.raises(ValueError, match="CUDA"):
        api.make_scan(torch.zeros((4, 3)), None, api.MT_CONFOCAL, wall["normal"], wall["albedo"], (0, 1))


def test_streamed_output_host_buffers_must_match_the_film():
    H, W, T = 2, 3, 4
    out = (torch.zeros((H, W, T, 3)), torch.zeros((H, W, 3)))
    with pytest.raises(ValueError, match="host film holds 60 values where the film copies 72"):
        api.render_to_host(None, H, W, T, 0.0, 1.0, 1, 1, 1, torch.zeros((H - 1, W + 2, T, 3)),
                           torch.zeros((H, W, 3)), 1, None, out=out)
    with pytest.raises(ValueError, match="host steady image holds"):
        api.render_to_host(None, H, W, T, 0.0, 1.0, 1, 1, 1, torch.zeros((H, W, T, 3)), torch.zeros((H, W, 1)),
                           1, None, out=out)


def test_autograd_function_is_one_class():
    assert api.TransientRender is api.TransientRender
    assert issubclass(api.TransientRender, torch.autograd.Function)
    with pytest.raises(AttributeError):
        api.NoSuchName
