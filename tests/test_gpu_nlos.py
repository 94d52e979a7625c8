"""GPU parity of the batched relay-wall NLOS estimator (Sec. 4.5) against the
oracle: per-connection contributions and films, confocal and exhaustive grids;
graph replay and the per-scan-point launch loop give the same films."""
import numpy as np
import pytest

from gpu_util import build_and_load, match_contribs, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nlos(oracle_mod, scenes_mod):
    api = build_and_load()
    sc = scenes_mod.nlos_scene()
    return api, sc, api.Scene(sc), oracle_mod.OracleScene(sc)


def _pts(scenes_mod, n):
    return scenes_mod.wall_grid(n, n)


@pytest.mark.parametrize("mode", ["confocal", "exhaustive"])
def test_nlos_contributions_and_film(nlos, scenes_mod, mode):
    import torch
    api, sc, s, osc = nlos
    T, start, width = 4096, 0.0, 0.003
    spp, seed = 128, 25660
    if mode == "confocal":
        lasers = _pts(scenes_mod, 8)
        sensors = None
        m = api.MT_CONFOCAL
    else:
        lasers = scenes_mod.wall_grid(2, 2)
        sensors = _pts(scenes_mod, 6)
        m = api.MT_EXHAUSTIVE
    L = torch.from_numpy(lasers).cuda()
    S = torch.from_numpy(sensors).cuda() if sensors is not None else None
    film, steady, rec, n = api.render_dump(s, 0, 0, T, start, width, spp, seed, 2, cap=4_000_000,
                                           scan_args=(L, S, m))
    ref = osc.render_nlos(lasers, sensors, m == api.MT_EXHAUSTIVE, T, start, width, spp, seed, dump_cap=4_000_000)
    nm, div, worst, bad, bin_bad, _ = match_contribs(rec, ref["dump"], start=start, width=width)
    assert nm > 1000
    assert div <= 1e-4 * nm, (div, nm)  # measured: none
    assert bad <= 1e-3 * nm, (bad, worst)
    assert bin_bad == 0
    f = film.cpu().numpy().reshape(ref["film"].shape)
    assert rel_l2(f, ref["film"]) < 0.01
    assert rel_l2(steady.cpu().numpy().reshape(-1), ref["steady"]) < 0.01


def test_graph_replay_and_per_point_loop_agree(nlos, scenes_mod):
    """The cached-graph replay reproduces the first launch; the plain
    per-scan-point launch loop (one launch per point, laser index 0 each time)
    matches the oracle run with the same indexing."""
    import torch
    api, sc, s, osc = nlos
    T, start, width = 4096, 0.0, 0.003
    pts = _pts(scenes_mod, 8)
    lasers = torch.from_numpy(pts).cuda()
    f1, s1 = api.render_nlos(s, lasers, None, api.MT_CONFOCAL, T, start, width, 64, 5)
    f2, s2 = api.render_nlos(s, lasers, None, api.MT_CONFOCAL, T, start, width, 64, 5)  # cached graph
    s.sync()
    assert torch.allclose(f1, f2, rtol=1e-5, atol=1e-9)
    for i in (0, 9, 27, 63):
        fi, si = api.render_nlos(s, lasers[i:i + 1].contiguous(), None, api.MT_CONFOCAL, T, start, width, 256, 5)
        ref = osc.render_nlos(pts[i:i + 1], None, False, T, start, width, 256, 5)
        assert rel_l2(si.cpu().numpy(), ref["steady"]) < 0.01
        assert rel_l2(fi.cpu().numpy(), ref["film"]) < 0.01


@pytest.mark.parametrize("cfg", [(256, 2, 0, -1, 0), (256, 6, 0, -1, 1), (128, 64, 0, 0, 0), (256, 5, 0, 1000, 0)])
def test_exhaustive_launch_configurations_agree(nlos, scenes_mod, cfg):
    """Exhaustive grids launch with their own configuration kind (default: 32
    sensors per tile, every splat in global memory, lanes sensor-fastest):
    tiles that do or do not divide the sensors, shared-memory histograms of
    every bin or of part of them, and warp aggregation give the default's film;
    the scan-point kind's configuration does not apply to them."""
    import torch
    api, sc, s, osc = nlos
    T, start, width = 4096, 0.0, 0.003
    L = torch.from_numpy(scenes_mod.wall_grid(3, 3)).cuda()
    S = torch.from_numpy(scenes_mod.wall_grid(7, 7)).cuda()
    ref, ref_s = [x.clone() for x in api.render_nlos(s, L, S, api.MT_EXHAUSTIVE, T, start, width, 256, 3)]
    threads, tile, cps, priv, agg = cfg
    s.set_launch(api.MT_LAUNCH_NLOS, 32, 1, 0, 0, 0)  # scan-point kind only: no effect here
    s.set_launch(api.MT_LAUNCH_NLOS_EXHAUSTIVE, threads, tile, cps, priv, api.MT_OPT_AGGREGATE if agg else 0)
    try:
        f, st = api.render_nlos(s, L, S, api.MT_EXHAUSTIVE, T, start, width, 256, 3)
        s.sync()
    finally:
        s.set_launch(api.MT_LAUNCH_NLOS)
        s.set_launch(api.MT_LAUNCH_NLOS_EXHAUSTIVE, 256, 32, 0, 0, 0)
    assert ref.abs().max() > 0
    assert rel_l2(f.cpu().numpy(), ref.cpu().numpy()) < 1e-5
    assert rel_l2(st.cpu().numpy(), ref_s.cpu().numpy()) < 1e-5
    with pytest.raises(api.MtError) as e:  # no launch kind beyond the exhaustive one
        s.set_launch(api.MT_LAUNCH_NLOS_EXHAUSTIVE + 1)
    assert e.value.status == api.MT_ERR_INVALID_ARGUMENT
