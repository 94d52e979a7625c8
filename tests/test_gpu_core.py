"""GPU parity of the forward path against the FP64 oracle, through the C ABI.

Philox bit-exact; time-bin indices bit-exact away from bin edges; closest-hit
triangle ids bit-exact on margin-filtered ray sets; the single-bounce closed
form; per-path contributions within 1e-4 relative on the same Philox stream;
films within 1% relative L2 over bins with >= 100 samples; the T-sum
invariant; resumable rendering.
"""
import numpy as np
import pytest

from gpu_util import build_and_load, match_contribs, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return build_and_load()


def test_philox_bit_exact(api, oracle_mod):
    import torch
    rng = np.random.default_rng(0)
    n = 1 << 20
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:1000, 1:] = 0  # small counters too
    for seed in (25660, 0xDEADBEEF12345678):
        out = api.probe_philox(seed, torch.from_numpy(ctr.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
        ref = oracle_mod.philox_batch(ctr, seed)
        assert np.array_equal(out, ref)


def test_bins_bit_exact(api):
    import torch
    rng = np.random.default_rng(1)
    for start, width, T in ((3.5, 0.01, 256), (12.0, 0.005, 2048), (0.0, 0.003, 4096)):
        opl = rng.uniform(start - 1.0, start + width * T + 1.0, 200000).astype(np.float32)
        opl[:100] = start + width * np.arange(100, dtype=np.float32)  # near edges
        got = api.probe_bins(torch.from_numpy(opl).cuda(), start, width, T).cpu().numpy()
        x = (opl.astype(np.float64) - start) / width
        ref = np.floor(x).astype(np.int64)
        ref[(ref < 0) | (ref >= T)] = -1
        edge = np.abs(x - np.round(x)) * width < 1e-5
        assert np.array_equal(got[~edge], ref[~edge])
        assert np.all((got[edge] == ref[edge]) | (np.abs(got[edge] - ref[edge]) == 1) | (got[edge] == -1) | (ref[edge] == -1))


def _exact_hits(tris, o, d):
    """All hits of each ray (float64 Moller-Trumbore): t [R, M] (inf if miss) and the margin
    min barycentric [R, M]."""
    v0 = tris[:, 0].astype(np.float64)
    e1 = tris[:, 1].astype(np.float64) - v0
    e2 = tris[:, 2].astype(np.float64) - v0
    O = o.astype(np.float64)[:, None, :]
    D = d.astype(np.float64)[:, None, :]
    p = np.cross(D, e2[None])
    det = np.einsum("rmk,mk->rm", p, e1)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / det
        s = O - v0[None]
        u = np.einsum("rmk,rmk->rm", s, p) * inv
        q = np.cross(s, e1[None])
        v = np.einsum("rmk,rmk->rm", np.broadcast_to(D, q.shape), q) * inv
        t = np.einsum("mk,rmk->rm", e2, q) * inv
    bmin = np.minimum(np.minimum(u, v), 1 - u - v)
    hit = (bmin >= 0) & (t > 0) & np.isfinite(t)
    return np.where(hit, t, np.inf), bmin, t


@pytest.mark.parametrize("wide", [False, True], ids=["binary", "wide"])
@pytest.mark.parametrize("seed,n_tris", [(1, 7), (2, 64), (3, 200), (4, 1500)])
def test_closest_hit_ids_bit_exact(api, scenes_mod, seed, n_tris, wide):
    import torch
    tris = scenes_mod.random_mesh(seed, n_tris)
    sc = scenes_mod.Scene(tris, np.full((n_tris, 3), 0.5, np.float32), np.zeros(n_tris, np.float32),
                          np.zeros(n_tris, np.uint32), [], dict(origin=(0, 0, 5), target=(0, 0, 0), up=(0, 1, 0), fov_x_deg=40))
    s = api.Scene(sc)
    o, d = scenes_mod.random_rays(seed + 100, 4000)
    rays = torch.from_numpy(np.concatenate([o, d], 1)).cuda()
    tri, t = api.probe_trace(s, rays, wide=wide)
    occ, _ = api.probe_trace(s, rays, tmax=1.5, any_hit=True, wide=wide)
    tri, t, occ = tri.cpu().numpy(), t.cpu().numpy(), occ.cpu().numpy()
    T, bmin, traw = _exact_hits(tris, o, d)
    best = T.argmin(1)
    tb = T[np.arange(len(o)), best]
    T2 = T.copy()
    T2[np.arange(len(o)), best] = np.inf
    second = T2.min(1)
    # margin filter: clear hit (barycentrics > 1e-4, next hit > 1.0001 t) or clear miss
    near_edge = np.any((np.abs(bmin) < 1e-4) & (traw > 0), axis=1)
    clear_hit = np.isfinite(tb) & (second > tb * 1.0001) & ~near_edge
    clear_miss = ~np.isfinite(tb) & ~near_edge
    assert clear_hit.sum() > 200 or n_tris < 64
    assert np.array_equal(tri[clear_hit], best[clear_hit])
    assert np.all(tri[clear_miss] == -1)
    # watertight t = T/det carries an absolute error ~ eps * |coordinates|
    assert np.allclose(t[clear_hit], tb[clear_hit], rtol=1e-5, atol=2e-6)
    # any hit within t < 1.5
    clear_occ = (~near_edge) & (np.abs(T - 1.5) > 1e-4).all(1)
    ref_occ = (T < 1.5).any(1)
    assert np.array_equal(occ[clear_occ].astype(bool), ref_occ[clear_occ])


@pytest.mark.parametrize("which", ["cornell_box", "diff_scene", "large_scene"])
def test_wide_bvh_hits_equal_binary(api, scenes_mod, which):
    """Both trees cull conservatively and share the triangle test and the tie
    rule, so closest hits (index and t) and occlusion agree bit for bit."""
    import torch
    sc = getattr(scenes_mod, which)()
    s = api.Scene(sc)
    rng = np.random.default_rng(17)
    n = 200_000
    lo, hi = sc.tris.reshape(-1, 3).min(0), sc.tris.reshape(-1, 3).max(0)
    # origins inside the scene box and on scene triangles (bounce-like rays)
    o1 = rng.uniform(lo, hi, (n // 2, 3))
    k = rng.integers(0, sc.n_tris, n - n // 2)
    b = rng.dirichlet([1, 1, 1], n - n // 2)
    o2 = np.einsum("nk,nkc->nc", b, sc.tris[k].astype(np.float64))
    o = np.concatenate([o1, o2]).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    o = o + 1e-4 * d * (np.abs(o).max(1, keepdims=True) + 1)
    rays = torch.from_numpy(np.concatenate([o, d], 1).astype(np.float32)).cuda()
    ta, da = api.probe_trace(s, rays)
    tb, db = api.probe_trace(s, rays, wide=True)
    oa, _ = api.probe_trace(s, rays, tmax=0.7, any_hit=True)
    ob, _ = api.probe_trace(s, rays, tmax=0.7, any_hit=True, wide=True)
    s.sync()
    assert (ta >= 0).float().mean().item() > 0.3
    assert torch.equal(ta, tb)
    assert torch.equal(da, db)
    assert torch.equal(oa, ob)


def test_closest_hit_large_scene_vs_oracle(api, oracle_mod, scenes_mod):
    """97k-triangle scene: GPU SAH BVH vs oracle median-split BVH on 20k rays;
    id mismatches only on near ties."""
    import torch
    sc = scenes_mod.diff_scene()
    s = api.Scene(sc)
    st = s.stats()
    assert st["n_tris"] == sc.n_tris and st["bvh_depth"] < 64
    osc = oracle_mod.OracleScene(sc)
    rng = np.random.default_rng(9)
    n = 20000
    o = np.stack([rng.uniform(-9, 9, n), rng.uniform(3, 7, n), rng.uniform(-9, 9, n)], 1).astype(np.float32)
    tgt = np.stack([rng.uniform(-10, 10, n), rng.uniform(0, 2, n), rng.uniform(-10, 10, n)], 1)
    d = (tgt - o)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    tri, t = api.probe_trace(s, torch.from_numpy(np.concatenate([o, d], 1)).cuda())
    tri, t = tri.cpu().numpy(), t.cpu().numpy()
    mism = 0
    for i in range(n):
        oi, ot = osc.intersect(o[i].astype(np.float64), d[i].astype(np.float64))
        if oi != tri[i]:
            mism += 1
            assert oi >= 0 and tri[i] >= 0 and abs(ot - t[i]) < 1e-5 * max(1, ot), (i, oi, tri[i], ot, t[i])
        elif oi >= 0:
            assert abs(ot - t[i]) < 2e-6 * max(1.0, ot)
    assert mism < 1e-3 * n


def test_point_light_plane_closed_form(api, oracle_mod, scenes_mod):
    sc = scenes_mod.point_light_plane()
    s = api.Scene(sc)
    H = W = 32
    T, start, width = 600, 0.0, 0.01
    film, steady = api.render(s, H, W, T, start, width, spp=1, seed=7, max_depth=2, flags=api.MT_PIXEL_CENTER)
    s.sync()
    film = film.cpu().numpy()
    osc = oracle_mod.OracleScene(sc)
    ref = osc.render(H, W, T, start, width, spp=1, seed=7, max_depth=2, flags=oracle_mod.PIXEL_CENTER)
    # same single spike per pixel, same bin except at edges, value within FP32 rounding
    fr = ref["film"][..., 0]
    fg = film[..., 0]
    kb = np.argmax(fr, axis=2)
    kg = np.argmax(fg, axis=2)
    assert np.all((fg > 0).sum(2) == 1)
    vr = fr.max(2)
    vg = fg.max(2)
    assert np.allclose(vg, vr, rtol=2e-5)
    assert np.mean(kb == kg) > 0.99 and np.all(np.abs(kb - kg) <= 1)
    assert np.allclose(steady.cpu().numpy(), ref["steady"], rtol=2e-5)


@pytest.fixture(scope="module")
def cornell(api, oracle_mod, scenes_mod):
    sc = scenes_mod.cornell_box()
    return sc, api.Scene(sc), oracle_mod.OracleScene(sc)


def test_cornell_per_path_contributions(api, cornell):
    sc, s, osc = cornell
    H = W = 64
    T, start, width = 256, 3.5, 0.01
    spp, seed, depth = 4, 25660, 4
    film, steady, rec, n = api.render_dump(s, H, W, T, start, width, spp, seed, depth, cap=2_000_000)
    assert n <= 2_000_000
    crop = (16, 48, 16, 48)
    ref = osc.render(H, W, T, start, width, spp, seed, depth, crop=crop, dump_cap=2_000_000)
    px = rec["pixel"] % W
    py = rec["pixel"] // W
    sel = (px >= crop[0]) & (px < crop[1]) & (py >= crop[2]) & (py < crop[3])
    nm, div, worst, bad, bin_bad, _ = match_contribs(rec[sel], ref["dump"], start=start, width=width)
    assert nm > 3000
    assert div <= 1e-4 * nm, (div, nm)  # measured: none
    assert bad <= 1e-3 * nm, (bad, worst)
    assert bin_bad == 0


def test_cornell_film_parity_and_tsum(api, cornell):
    sc, s, osc = cornell
    H = W = 64
    T, start, width = 256, 3.5, 0.01
    spp, seed, depth = 16, 25660, 4
    film, steady = api.render(s, H, W, T, start, width, spp, seed, depth)
    s.sync()
    film, steady = film.cpu().numpy(), steady.cpu().numpy()
    crop = (20, 44, 20, 44)
    ref = osc.render(H, W, T, start, width, spp, seed, depth, crop=crop, dump_cap=3_000_000)
    g = film[crop[2]:crop[3], crop[0]:crop[1]]
    d = ref["dump"]
    cnt = np.zeros(ref["film"].shape[:3])
    inb = (d["bin"] >= 0) & (d["bin"] < T)
    np.add.at(cnt, ((d["pixel"][inb] // W) - crop[2], (d["pixel"][inb] % W) - crop[0], d["bin"][inb]), 1)
    mask = np.broadcast_to((cnt >= 100)[..., None], g.shape)
    assert rel_l2(g, ref["film"]) < 0.01
    if mask.any():
        assert rel_l2(g, ref["film"], mask) < 0.01
    assert rel_l2(steady[crop[2]:crop[3], crop[0]:crop[1]], ref["steady"]) < 0.01
    # T-sum: with a window covering all OPLs the time-summed film equals the steady image
    film2, steady2 = api.render(s, H, W, 1024, 0.0, 0.05, spp, seed, depth)
    s.sync()
    f2, s2 = film2.cpu().numpy(), steady2.cpu().numpy()
    assert np.allclose(f2.sum(2), s2, rtol=1e-4, atol=1e-6)


def test_resume_and_accumulate(api, cornell):
    sc, s, osc = cornell
    import torch
    H = W = 64
    T, start, width = 256, 3.5, 0.01
    film, steady = api.new_film(H, W, T)
    film.zero_()
    steady.zero_()
    api.render(s, H, W, T, start, width, 3, 11, 4, sample_offset=0, flags=api.MT_ACCUMULATE, out=(film, steady))
    api.render(s, H, W, T, start, width, 5, 11, 4, sample_offset=3, flags=api.MT_ACCUMULATE, out=(film, steady))
    full, fs = api.render(s, H, W, T, start, width, 8, 11, 4)
    s.sync()
    assert torch.allclose(film / 8, full, rtol=1e-4, atol=1e-6)
    assert torch.allclose(steady / 8, fs, rtol=1e-4, atol=1e-6)


def test_unwarp_moves_spike_to_d1(api, oracle_mod, scenes_mod):
    sc = scenes_mod.point_light_plane()
    s = api.Scene(sc)
    H = W = 16
    film, _ = api.render(s, H, W, 600, 0.0, 0.01, 1, 7, 2, flags=api.MT_PIXEL_CENTER | api.MT_UNWARP)
    s.sync()
    ref = oracle_mod.OracleScene(sc).render(H, W, 600, 0.0, 0.01, 1, 7, 2,
                                             flags=oracle_mod.PIXEL_CENTER | oracle_mod.UNWARP)
    kg = film.cpu().numpy()[..., 0].argmax(2)
    kb = ref["film"][..., 0].argmax(2)
    assert np.mean(kg == kb) > 0.98


def test_counters_and_stats(api, cornell):
    sc, s, osc = cornell
    s.read_counters(reset=True)
    api.render(s, 64, 64, 256, 3.5, 0.01, 2, 1, 4, flags=api.MT_COUNTERS)
    c = s.read_counters(reset=True)
    assert c["paths"] == 64 * 64 * 2
    assert c["vertices"] > c["paths"] and c["node_bytes"] > 0 and c["tri_tests"] > 0
    ref = osc.render(64, 64, 256, 3.5, 0.01, 2, 1, 4)
    assert abs(c["vertices"] - ref["counters"]["vertices"]) <= 1e-3 * ref["counters"]["vertices"]
    st = s.stats()
    assert st["n_tris"] == 36 and st["light_units"] == 2


def test_invalid_arguments_give_status(api, cornell):
    sc, s, osc = cornell
    with pytest.raises(api.MtError) as e:
        api.render(s, 64, 64, 256, 3.5, 0.01, 0, 1, 4)
    assert e.value.status == api.MT_ERR_INVALID_ARGUMENT
    with pytest.raises(api.MtError) as e:
        api.render(s, 64, 64, 256, 3.5, 0.01, 1, 1, 65)
    assert e.value.status == api.MT_ERR_INVALID_ARGUMENT


def _form_options(api, opts):
    return {"wavefront": api.MT_OPT_WAVEFRONT,
            "wavefront_wide_bvh": api.MT_OPT_WAVEFRONT | api.MT_OPT_WIDE_BVH,
            "wavefront_sorted": api.MT_OPT_WAVEFRONT | api.MT_OPT_SORT_RAYS,
            "wavefront_sorted_shadow": api.MT_OPT_WAVEFRONT | api.MT_OPT_SORT_SHADOW,
            "wavefront_dynamic_fetch": api.MT_OPT_WAVEFRONT | api.MT_OPT_DYNAMIC_FETCH,
            "megakernel_refill16": api.MT_OPT_REFILL(16)}[opts]


@pytest.mark.parametrize("opts", ["wavefront", "wavefront_wide_bvh", "wavefront_sorted", "wavefront_sorted_shadow",
                                  "wavefront_dynamic_fetch", "megakernel_refill16"])
def test_forward_forms_per_path_parity(api, cornell, opts):
    """The wavefront form (with or without dynamic ray fetch in its traversal
    kernels) and the megakernel with deferred refill compute the same
    contributions as the oracle on the same Philox stream."""
    sc, s, osc = cornell
    H = W = 64
    T, start, width = 256, 3.5, 0.01
    spp, seed, depth = 4, 77, 4
    opt = _form_options(api, opts)
    s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, opt)
    try:
        film, steady, rec, n = api.render_dump(s, H, W, T, start, width, spp, seed, depth, cap=2_000_000)
        f2, s2 = api.render(s, H, W, T, start, width, spp, seed, depth)
    finally:
        s.set_launch(api.MT_LAUNCH_RENDER)
    crop = (16, 48, 16, 48)
    ref = osc.render(H, W, T, start, width, spp, seed, depth, crop=crop, dump_cap=2_000_000)
    px, py = rec["pixel"] % W, rec["pixel"] // W
    sel = (px >= crop[0]) & (px < crop[1]) & (py >= crop[2]) & (py < crop[3])
    nm, div, worst, bad, bin_bad, _ = match_contribs(rec[sel], ref["dump"], start=start, width=width)
    assert nm > 3000 and div <= 1e-4 * nm and bad <= 1e-3 * nm and bin_bad == 0, (nm, div, bad, bin_bad)
    g = f2.cpu().numpy()[crop[2]:crop[3], crop[0]:crop[1]]
    assert rel_l2(g, ref["film"]) < 0.01
    assert rel_l2(s2.cpu().numpy()[crop[2]:crop[3], crop[0]:crop[1]], ref["steady"]) < 0.01
    # the default form on the same samples gives the same film
    f3, s3 = api.render(s, H, W, T, start, width, spp, seed, depth)
    assert rel_l2(f2.cpu().numpy(), f3.cpu().numpy()) < 1e-4


@pytest.mark.parametrize("opts", ["wavefront", "wavefront_wide_bvh", "wavefront_sorted", "wavefront_sorted_shadow",
                                  "wavefront_dynamic_fetch"])
def test_wavefront_large_scene_matches_megakernel(api, scenes_mod, opts):
    sc = scenes_mod.diff_scene()
    s = api.Scene(sc)
    f = scenes_mod.DIFF_FILM
    a, sa = api.render(s, 64, 64, f.T, f.start_opl, f.bin_width, 16, 3, 8)
    s.set_launch(api.MT_LAUNCH_RENDER, 256, 0, 0, -1, _form_options(api, opts))
    b, sb = api.render(s, 64, 64, f.T, f.start_opl, f.bin_width, 16, 3, 8)
    s.sync()
    assert rel_l2(b.cpu().numpy(), a.cpu().numpy()) < 1e-4
    assert rel_l2(sb.cpu().numpy(), sa.cpu().numpy()) < 1e-4
