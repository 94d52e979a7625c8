"""Host logic of the launch autotuner (no GPU): the search space, the limits
every candidate must respect, the path-pool sizing, the cache and the shipped
launch table.

The tuner searches tile size, paths per thread and privatisation depth for the
batched launches (Sec. 4.5 grids of impulse responses, the renders of Sec. 3);
timing itself needs a GPU and is covered by the `-m gpu` tests.
"""
import json
import types

import pytest

from paper_2510_25660_gb300 import autotune

# launch limits checked by mt_set_launch / mt_set_wavefront_pool (include/mt_api.h)
KNOWN_OPTIONS = 1 | 2 | 4 | 8 | 16 | 32 | 64 | 128 | 0xFF00
POOL_MAX = 1 << 22


@pytest.fixture
def fake_gpu(monkeypatch):
    """torch.cuda queries answered as on a 152-SM GB300."""
    import torch
    props = types.SimpleNamespace(multi_processor_count=152)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a, **k: "NVIDIA GB300")
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda *a, **k: props)
    return props


class FakeScene:
    def __init__(self):
        self.calls = []

    def set_launch(self, *a):
        self.calls.append(("set_launch",) + a)

    def set_wavefront_pool(self, n):
        self.calls.append(("set_wavefront_pool", n))


def _large():
    sc = types.SimpleNamespace(n_tris=1164296, medium=None)
    film = types.SimpleNamespace(T=2048, W=512)
    return sc, film


def test_render_search_space_covers_tile_paths_per_thread_and_depth():
    T = 2048
    c = autotune.candidates("render", T)
    wf = [x for x in c if x[4] & 4]
    mk = [x for x in c if not x[4] & 4]
    # the wavefront form comes first, at 1, 2, 4, 8 paths per thread and the default pool
    assert c[:len(wf)] == wf
    assert sorted(x[5] for x in wf) == [0, 1, 2, 4, 8]
    assert {x[1] for x in mk} == {1, 2, 4, 8, 16}
    assert {x[3] for x in mk} == {-1, 0, T // 4, T // 2}
    assert {x[2] for x in mk} == {0, 4}
    assert {x[0] for x in mk} == {128, 256}
    assert len(set(c)) == len(c)
    assert autotune.candidates("render", T, wavefront_only=True) == wf


def test_nlos_search_space():
    c = autotune.candidates("nlos", 4096)
    assert {x[1] for x in c} == {1, 2, 4, 8, 16}
    assert {x[2] for x in c} == {0, 4}
    assert {x[3] for x in c} == {-1, 0}
    assert {x[4] for x in c} == {0, 1}
    assert all(len(x) == 5 for x in c)


@pytest.mark.parametrize("kind", ["render", "backward", "nlos"])
def test_candidates_respect_the_launch_limits(kind, fake_gpu):
    for x in autotune.candidates(kind, 512):
        threads, tile, cps, priv, opts = x[:5]
        assert 32 <= threads <= 256 and threads % 32 == 0
        assert 0 <= tile <= 4096 and 0 <= cps <= 32 and priv >= -1
        assert opts & ~KNOWN_OPTIONS == 0
        if len(x) > 5:
            n = autotune.pool_paths(x[5])
            assert n == 0 or 32 <= n <= POOL_MAX


def test_pool_paths(fake_gpu):
    assert autotune.pool_paths(0) == 0
    assert autotune.pool_paths(1) == 152 * 8 * 256
    assert autotune.pool_paths(8) == 8 * 152 * 8 * 256
    assert autotune.pool_paths(16) == POOL_MAX  # capped at the library's maximum
    fake_gpu.multi_processor_count = 1
    assert autotune.pool_paths(1) == 2048


def test_apply_takes_the_user_cache_then_the_shipped_table(fake_gpu, tmp_path, monkeypatch):
    monkeypatch.setenv("MT_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    sc, film = _large()
    s = FakeScene()
    cfg = autotune.apply(s, "render", sc, film, 256, 8)
    table = json.load(open(autotune.TABLE))
    assert cfg == table[autotune._key("render", sc, film, 256, 8)]
    assert s.calls == [("set_launch", 0, cfg["threads"], cfg["tile"], cfg["ctas_per_sm"], cfg["priv"],
                        cfg["options"]),
                       ("set_wavefront_pool", autotune.pool_paths(cfg.get("paths_per_thread", 0)))]
    # a user cache entry for the same workload wins over the table
    mine = {"threads": 128, "tile": 4, "ctas_per_sm": 4, "priv": 0, "options": 0, "paths_per_thread": 0}
    autotune._store({autotune._key("render", sc, film, 256, 8): mine})
    s = FakeScene()
    assert autotune.apply(s, "render", sc, film, 256, 8) == mine
    assert s.calls[0] == ("set_launch", 0, 128, 4, 4, 0, 0)
    # an unknown workload leaves the scene's configuration alone
    s = FakeScene()
    assert autotune.apply(s, "render", sc, film, 3, 8) is None
    assert s.calls == []
    # NLOS configurations do not touch the path pool
    s = FakeScene()
    nlos_sc = types.SimpleNamespace(n_tris=49410, medium=None)
    cfg = autotune.apply(s, "nlos", nlos_sc, None, 1024, 0)
    assert cfg is not None and [c[0] for c in s.calls] == ["set_launch"] and s.calls[0][1] == 2


def test_cache_round_trip_and_unreadable_cache(tmp_path, monkeypatch):
    p = tmp_path / "sub" / "cache.json"
    monkeypatch.setenv("MT_AUTOTUNE_CACHE", str(p))
    assert autotune._load() == {}
    autotune._store({"k": {"threads": 256}})
    assert autotune._load() == {"k": {"threads": 256}}
    assert [x.name for x in p.parent.iterdir()] == ["cache.json"]  # no temporary left behind
    p.write_text("{not json")
    assert autotune._load() == {}


def test_shipped_table_is_valid_and_picks_the_wavefront_form_for_large_renders():
    table = json.load(open(autotune.TABLE))
    assert table
    for key, cfg in table.items():
        dev, kind, n, shape, spp, depth, med = key.split("|")
        assert kind in autotune.KINDS and n.startswith("n") and spp.startswith("spp")
        threads, tile, cps, priv = cfg["threads"], cfg["tile"], cfg["ctas_per_sm"], cfg["priv"]
        assert 32 <= threads <= 256 and threads % 32 == 0
        assert 0 <= tile <= 4096 and 0 <= cps <= 32 and priv >= -1
        assert cfg.get("options", 0) & ~KNOWN_OPTIONS == 0
        if kind != "nlos" and int(n[1:]) > 10000:
            assert cfg["options"] & 4, key  # the wavefront form (MT_OPT_WAVEFRONT)
