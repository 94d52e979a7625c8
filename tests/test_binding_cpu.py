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
