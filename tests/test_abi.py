"""C-ABI checks that need no GPU: libmt.so builds for sm_103a, loads, exports
every function declared in include/mt_api.h, and rejects invalid arguments
with status codes before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_25660_gb300 import build as b
    b.build()
    from paper_2510_25660_gb300 import api
    return api, api.load()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mt_[a-z0-9_]+)\s*\(", txt))
    return names


def test_exports_every_declared_function(lib):
    api, L = lib
    names = _declared()
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    assert set(api.SIGNATURES) == names, "binding and header disagree"


def test_struct_layouts_match_header(lib, tmp_path):
    """ctypes structs of the binding have the C compiler's size and field offsets."""
    api, _ = lib
    structs = {"mt_material": api.mt_material, "mt_emitter": api.mt_emitter, "mt_camera": api.mt_camera,
               "mt_medium": api.mt_medium, "mt_scan": api.mt_scan, "mt_contrib": api.mt_contrib}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{ROOT}/include/mt_api.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", str(src), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == C.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(out[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)


def test_invalid_arguments_without_gpu(lib):
    api, L = lib
    h = C.c_void_p()
    # film: bad sizes, bad window, NULL pointer, unknown flags
    buf = C.c_void_p(0x1000)
    assert L.mt_film_create(0, 4, 4, 3, 0.0, 0.1, buf, None, 0, C.byref(h)) == api.MT_ERR_INVALID_ARGUMENT
    assert L.mt_film_create(4, 4, 4, 2, 0.0, 0.1, buf, None, 0, C.byref(h)) == api.MT_ERR_INVALID_ARGUMENT
    assert L.mt_film_create(4, 4, 4, 3, 0.0, 0.0, buf, None, 0, C.byref(h)) == api.MT_ERR_INVALID_ARGUMENT
    assert L.mt_film_create(4, 4, 4, 3, 0.0, 0.1, None, None, 0, C.byref(h)) == api.MT_ERR_INVALID_ARGUMENT
    assert L.mt_film_create(4, 4, 4, 3, 0.0, 0.1, buf, None, 1 << 9, C.byref(h)) == api.MT_ERR_INVALID_ARGUMENT
    assert b"flags" in L.mt_last_error()
    assert L.mt_film_create(4, 4, 4, 3, 0.0, 0.1, buf, None, 0, C.byref(h)) == api.MT_OK
    L.mt_film_destroy(h)
    # scene: NaN vertex, NULL arrays, bad emitter ranges, bad materials
    tris = np.zeros((2, 3, 3), np.float32)
    tris[1, 2, 1] = np.nan
    mats = (api.mt_material * 2)()
    cam = api.mt_camera((C.c_float * 3)(0, 0, 3), (C.c_float * 3)(0, 0, 0), (C.c_float * 3)(0, 1, 0), 40.0)
    tp = tris.ctypes.data_as(C.c_void_p)
    assert L.mt_scene_create(tp, 2, mats, None, 0, C.byref(cam), None, None, C.byref(h)) == api.MT_ERR_INVALID_ARGUMENT
    assert b"non-finite" in L.mt_last_error()
    tris[1, 2, 1] = 0.0
    assert L.mt_scene_create(None, 2, mats, None, 0, C.byref(cam), None, None, C.byref(h)) == api.MT_ERR_INVALID_ARGUMENT
    assert L.mt_scene_create(tp, 0, mats, None, 0, C.byref(cam), None, None, C.byref(h)) == api.MT_ERR_INVALID_ARGUMENT
    ems = (api.mt_emitter * 1)(api.mt_emitter(0, 1, 5, (C.c_float * 3)(1, 1, 1), (C.c_float * 3)(0, 0, 0)))
    assert L.mt_scene_create(tp, 2, mats, ems, 1, C.byref(cam), None, None, C.byref(h)) == api.MT_ERR_INVALID_ARGUMENT
    mats[0].type = 7
    assert L.mt_scene_create(tp, 2, mats, None, 0, C.byref(cam), None, None, C.byref(h)) == api.MT_ERR_INVALID_ARGUMENT
    mats[0].type = api.MT_GGX_CONDUCTOR
    mats[0].roughness = 0.0
    assert L.mt_scene_create(tp, 2, mats, None, 0, C.byref(cam), None, None, C.byref(h)) == api.MT_ERR_INVALID_ARGUMENT
    # NULL handles
    assert L.mt_render(None, None, 1, 0, 1, 0, None) == api.MT_ERR_INVALID_ARGUMENT
    assert L.mt_render_backward(None, None, None, None, 1, 0, 1, 0, None, None, None, None) == api.MT_ERR_INVALID_ARGUMENT
    assert L.mt_render_nlos(None, None, None, 1, 0, 0, None) == api.MT_ERR_INVALID_ARGUMENT
    assert L.mt_sync(None, None) == api.MT_ERR_INVALID_ARGUMENT
    assert L.mt_set_launch(None, 0, 0, 0, 0, -1, 0) == api.MT_ERR_INVALID_ARGUMENT
    assert L.mt_set_wavefront_pool(None, 0) == api.MT_ERR_INVALID_ARGUMENT
    assert L.mt_render_nlos_noalloc(None, None, None, 1, 0, 0, None) == api.MT_ERR_INVALID_ARGUMENT
    assert L.mt_probe_bins(None, 4, 0.0, 1.0, 4, None, None) == api.MT_ERR_INVALID_ARGUMENT


def test_product_path_fails_loudly_without_library(tmp_path):
    from paper_2510_25660_gb300 import api
    old = api._lib
    try:
        api._lib = None
        with pytest.raises(RuntimeError):
            api.load(str(tmp_path / "missing.so"))
    finally:
        api._lib = old


def test_oracle_builds_and_is_isolated():
    """The oracle shares no code with the CUDA path: neither includes the other."""
    from oracle import oracle as O
    O.build()
    csrc = os.path.join(ROOT, "paper_2510_25660_gb300", "csrc")
    for f in os.listdir(csrc):
        txt = open(os.path.join(csrc, f)).read()
        assert "oracle" not in txt.lower(), f
    for f in ("mt_oracle.c", "mt_oracle.h"):
        txt = open(os.path.join(ROOT, "oracle", f)).read()
        assert "mt_api.h" not in txt and "csrc" not in txt
    for f in os.listdir(os.path.join(ROOT, "paper_2510_25660_gb300")):
        if f.endswith(".py") and f != "scenes.py":
            txt = open(os.path.join(ROOT, "paper_2510_25660_gb300", f)).read()
            assert "import oracle" not in txt and "from oracle" not in txt, f
