"""mt_render_nlos_noalloc: the NLOS capture for callers that cannot allocate
device memory when they render (device memory reserved up front by their own
allocator or a fixed budget).
It must give the same impulse responses as mt_render_nlos, through the C ABI,
on two calls in a row, without changing the device's free memory.

This file is collected last so that a failure here leaves every other test run.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_util import build_and_load, rel_l2

pytestmark = pytest.mark.gpu


def _film(api, rows, T):
    import torch
    film = torch.empty((rows, T), dtype=torch.float32, device="cuda")
    steady = torch.empty((rows,), dtype=torch.float32, device="cuda")
    h = C.c_void_p()
    api.mt_film_create(rows, 1, T, 1, 0.0, 0.003, api._ptr(film), api._ptr(steady), 0, C.byref(h))
    return film, steady, h


@pytest.mark.parametrize("launch", ["default", "global_aggregated"])
@pytest.mark.parametrize("mode", ["exhaustive", "confocal"])
def test_noalloc_matches_allocating_entry_point(mode, launch):
    """Also under a launch configuration that keeps no time bin in shared
    memory and combines equal-bin atomics across a warp: both entry points
    take the same configuration and the same kernel path."""
    import torch
    api = build_and_load()
    from paper_2510_25660_gb300 import scenes
    sc = scenes.nlos_scene()
    s = api.Scene(sc)
    if launch == "global_aggregated":
        s.set_launch(api.MT_LAUNCH_NLOS, 256, 0, 0, 0, api.MT_OPT_AGGREGATE)
    T, spp, seed = 4096, 256, 25660
    lasers = torch.from_numpy(scenes.wall_grid(4, 4)).cuda()
    if mode == "exhaustive":
        sensors = torch.from_numpy(scenes.wall_grid(8, 8)).cuda()
        m, rows = api.MT_EXHAUSTIVE, 16 * 64
    else:
        sensors, m, rows = None, api.MT_CONFOCAL, 16
    scan = api.make_scan(lasers, sensors, m, sc.wall["normal"], sc.wall["albedo"], sc.hidden)
    stream = api._stream()
    # the allocating entry point
    f_ref, s_ref, h_ref = _film(api, rows, T)
    api.mt_render_nlos(s.h, h_ref, C.byref(scan), spp, seed, 0, stream)
    s.sync()
    # the allocation-free entry point, twice in a row
    outs = []
    free = []
    for _ in range(2):
        f, st, h = _film(api, rows, T)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        api.mt_render_nlos_noalloc(s.h, h, C.byref(scan), spp, seed, 0, stream)
        s.sync()
        free.append(torch.cuda.mem_get_info()[0])
        outs.append((f, st))
        api.mt_film_destroy(h)
    api.mt_film_destroy(h_ref)
    for f, st in outs:
        # same samples, same kernels: equal up to the order of float additions
        assert rel_l2(f.cpu().numpy(), f_ref.cpu().numpy()) < 1e-4
        assert rel_l2(st.cpu().numpy(), s_ref.cpu().numpy()) < 1e-4
        assert float(s_ref.sum()) > 0
    # no allocation by the second call (the first may map the library's static array)
    assert free[2] == free[3]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    api = build_and_load()
    from paper_2510_25660_gb300 import scenes
    sc = scenes.nlos_scene()
    s = api.Scene(sc)
    lasers = torch.from_numpy(scenes.wall_grid(16, 16)).cuda()
    sensors = torch.from_numpy(scenes.wall_grid(2, 2)).cuda()
    scan = api.make_scan(lasers, sensors, api.MT_EXHAUSTIVE, sc.wall["normal"], sc.wall["albedo"], sc.hidden)
    f, st, h = _film(api, 256 * 4, 64)
    with pytest.raises(api.MtError) as e:
        api.mt_render_nlos_noalloc(s.h, h, C.byref(scan), 1024, 1, 0, api._stream())  # 256 * 1024 > 131072
    assert e.value.status == api.MT_ERR_INVALID_ARGUMENT
    assert "static scratch limit" in str(e.value)
    api.mt_film_destroy(h)
