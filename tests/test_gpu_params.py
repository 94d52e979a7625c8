"""Scene parameter updates (mt_scene_set_params): a render after updating
albedos and emitter radiances equals a render of a scene built with those
values, in both forms of the tracer (the wavefront form reads its own copy of
the materials, in the per-triangle shading records)."""
import dataclasses

import numpy as np
import pytest

from gpu_util import build_and_load, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form", ["megakernel", "wavefront"])
def test_set_params_equals_fresh_scene(scenes_mod, form):
    import torch
    api = build_and_load()
    sc = scenes_mod.cornell_box()
    sc.mtype[10:22] = 1
    sc.roughness[10:22] = 0.25
    rng = np.random.default_rng(11)
    alb = np.clip(sc.albedo * rng.uniform(0.6, 1.3, (sc.n_tris, 1)), 0.0, 0.95).astype(np.float32)
    rad = np.array([[14.0, 9.0, 6.0]], np.float32)
    opts = api.MT_OPT_WAVEFRONT if form == "wavefront" else 0
    s = api.Scene(sc)
    s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, opts)
    s.set_params(albedo=torch.from_numpy(alb).cuda(), radiance=torch.from_numpy(rad).cuda())
    a, sa = api.render(s, 48, 48, 128, 3.5, 0.02, 8, 5, 5)
    a, sa = a.clone(), sa.clone()
    emitters = [dict(e, radiance=tuple(float(v) for v in rad[0])) for e in sc.emitters]
    sc2 = dataclasses.replace(sc, albedo=alb, emitters=emitters)
    s2 = api.Scene(sc2)
    s2.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, opts)
    b, sb = api.render(s2, 48, 48, 128, 3.5, 0.02, 8, 5, 5)
    s2.sync()
    assert a.abs().max().item() > 0
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-5
    assert rel_l2(sa.cpu().numpy(), sb.cpu().numpy()) < 1e-5
