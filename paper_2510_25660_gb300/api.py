"""ctypes binding of libmt.so (the C ABI in include/mt_api.h).

Argument marshalling only: torch tensors supply device memory and the current
CUDA stream; every step of the rendering path runs in libmt's kernels.  The
functions ``mt_*`` mirror the C entry points one to one; ``Scene``,
``render``, ``render_nlos``, ``render_backward`` and ``TransientRender`` are
thin conveniences over them.  There is no fallback: if libmt.so is missing
or no CUDA device is present, the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import scenes as _scenes

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmt.so")

MT_OK, MT_ERR_INVALID_ARGUMENT, MT_ERR_OUT_OF_MEMORY, MT_ERR_CUDA, MT_ERR_TIMEOUT, MT_ERR_UNSUPPORTED, \
    MT_ERR_INTERNAL = range(7)
MT_LAMBERT, MT_GGX_CONDUCTOR = 0, 1
MT_EMITTER_AREA, MT_EMITTER_POINT = 0, 1
MT_UNWARP, MT_ACCUMULATE, MT_PIXEL_CENTER, MT_COUNTERS = 1, 2, 4, 8
MT_CONFOCAL, MT_EXHAUSTIVE = 0, 1
MT_LAUNCH_RENDER, MT_LAUNCH_BACKWARD, MT_LAUNCH_NLOS, MT_LAUNCH_NLOS_EXHAUSTIVE = 0, 1, 2, 3
MT_OPT_AGGREGATE, MT_OPT_NO_GRAPH, MT_OPT_WAVEFRONT, MT_OPT_DYNAMIC_FETCH, MT_OPT_WIDE_BVH = 1, 2, 4, 8, 16
MT_OPT_SORT_RAYS, MT_OPT_STAGE_TIMING, MT_OPT_SORT_SHADOW = 32, 64, 128
MT_PULSE_DELTA, MT_PULSE_BOX, MT_PULSE_GAUSSIAN, MT_PULSE_EXPONENTIAL = 0, 1, 2, 3


def MT_OPT_REFILL(k):
    return int(k) << 8
STATUS_NAMES = ["MT_OK", "MT_ERR_INVALID_ARGUMENT", "MT_ERR_OUT_OF_MEMORY", "MT_ERR_CUDA", "MT_ERR_TIMEOUT",
                "MT_ERR_UNSUPPORTED", "MT_ERR_INTERNAL"]


class mt_material(C.Structure):
    _fields_ = [("albedo", C.c_float * 3), ("roughness", C.c_float), ("type", C.c_uint32)]


class mt_emitter(C.Structure):
    _fields_ = [("type", C.c_uint32), ("first_tri", C.c_uint32), ("n_tris", C.c_uint32),
                ("radiance", C.c_float * 3), ("position", C.c_float * 3)]


class mt_camera(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3), ("fov_x_deg", C.c_float)]


class mt_medium(C.Structure):
    _fields_ = [("lo", C.c_float * 3), ("hi", C.c_float * 3), ("res", C.c_int32 * 3), ("density", C.c_void_p),
                ("albedo", C.c_float), ("g", C.c_float)]


class mt_scan(C.Structure):
    _fields_ = [("lasers", C.c_void_p), ("n_lasers", C.c_int32), ("sensors", C.c_void_p), ("n_sensors", C.c_int32),
                ("mode", C.c_uint32), ("wall_normal", C.c_float * 3), ("wall_albedo", C.c_float),
                ("hidden_first", C.c_uint32), ("hidden_count", C.c_uint32)]


class mt_contrib(C.Structure):
    _fields_ = [("pixel", C.c_int32), ("sample", C.c_int32), ("depth", C.c_int32), ("kind", C.c_int32),
                ("tri", C.c_int32), ("bin", C.c_int32), ("opl", C.c_float), ("c", C.c_float * 3)]


CONTRIB_DTYPE = np.dtype([("pixel", np.int32), ("sample", np.int32), ("depth", np.int32), ("kind", np.int32),
                          ("tri", np.int32), ("bin", np.int32), ("opl", np.float32), ("c", np.float32, (3,))])

# name -> (restype, argtypes)
_P, _I32, _I64, _U32, _U64, _F = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_float
SIGNATURES = {
    "mt_last_error": (C.c_char_p, []),
    "mt_scene_create": (C.c_int, [_P, _I64, _P, _P, _I32, _P, _P, _P, _P]),
    "mt_scene_set_params": (C.c_int, [_P, _P, _P, _P, _P]),
    "mt_film_create": (C.c_int, [_I32, _I32, _I32, _I32, _F, _F, _P, _P, _U32, _P]),
    "mt_render": (C.c_int, [_P, _P, _I32, _U64, _I32, _U64, _P]),
    "mt_render_to_host": (C.c_int, [_P, _P, _I32, _U64, _I32, _U64, _I32, _P, _P, _P, _P]),
    "mt_render_nlos": (C.c_int, [_P, _P, _P, _I32, _U64, _U64, _P]),
    "mt_render_backward": (C.c_int, [_P, _P, _P, _P, _I32, _U64, _I32, _U64, _P, _P, _P, _P]),
    "mt_sync": (C.c_int, [_P, _P]),
    "mt_read_counters": (C.c_int, [_P, _P, _I32, _P]),
    "mt_stage_times": (C.c_int, [_P, _P, _I32]),
    "mt_film_set_window": (C.c_int, [_P, _I32, _I32]),
    "mt_render_tangent": (C.c_int, [_P, _P, _P, _P, C.c_float, _I32, _U64, _I32, _U64, _P]),
    "mt_render_polarized": (C.c_int, [_P, _P, _I32, _U64, _I32, _U64, _P]),
    "mt_scene_set_delays": (C.c_int, [_P, _P, _P]),
    "mt_scene_set_pulse": (C.c_int, [_P, _U32, C.c_float, C.c_float]),
    "mt_scene_stats": (C.c_int, [_P, _P]),
    "mt_set_launch": (C.c_int, [_P, _I32, _I32, _I32, _I32, _I32, _U32]),
    "mt_set_wavefront_pool": (C.c_int, [_P, _I64]),
    "mt_scene_destroy": (None, [_P]),
    "mt_film_destroy": (None, [_P]),
    "mt_probe_philox": (C.c_int, [_U64, _P, _I64, _P, _P]),
    "mt_probe_trace": (C.c_int, [_P, _P, _I64, _F, _I32, _P, _P, _P]),
    "mt_probe_bins": (C.c_int, [_P, _I64, _F, _F, _I32, _P, _P]),
    "mt_render_dump": (C.c_int, [_P, _P, _P, _I32, _U64, _I32, _U64, _P, _I64, _P, _P]),
    "mt_render_nlos_noalloc": (C.c_int, [_P, _P, _P, _I32, _U64, _U64, _P]),
    "mt_microbench": (C.c_int, [_I32, _P, _I64, _I32, _P, _P]),
    "mt_render_phasor": (C.c_int, [_P, _P, _P, _I32, _I32, _U64, _I32, _U64, _P]),
}

_lib = None


class MtError(RuntimeError):
    def __init__(self, status, name, msg):
        super().__init__(f"{name}: {STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libmt.so (no build, no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libmt.so not built at {path}; run paper_2510_25660_gb300.build.build()")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _call(name, *args):
    rc = getattr(load(), name)(*args)
    if rc != MT_OK:
        raise MtError(rc, name, load().mt_last_error().decode())
    return rc


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _hptr(t):
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous() or t.dtype != torch_float32():
        raise ValueError("expected a contiguous host float32 tensor")
    return C.c_void_p(t.data_ptr())


def _check_f32(tensors, at_least=False):
    """The library reads or writes `numel` float32 values through each
    (tensor, numel, name)'s pointer (None tensors are skipped): dtypes and
    sizes first, then memory.  at_least: larger tensors are accepted."""
    tensors = [x for x in tensors if x[0] is not None]
    for t, numel, what in tensors:
        if t.dtype != torch_float32():
            raise ValueError(f"{what} must be float32, not {t.dtype}")
        if t.numel() < numel if at_least else t.numel() != numel:
            raise ValueError(f"{what} holds {t.numel()} values where {numel} are needed")
    for t, _, what in tensors:
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError(f"{what} must be a contiguous CUDA tensor")


def torch_float32():
    import torch
    return torch.float32


# --- mirrors of the C entry points ---------------------------------------------
def mt_last_error() -> str:
    return load().mt_last_error().decode()


def mt_scene_create(tris, n_tris, materials, emitters, n_emitters, camera, medium, stream, out):
    return _call("mt_scene_create", tris, n_tris, materials, emitters, n_emitters, camera, medium, stream, out)


def mt_scene_set_params(scene, d_albedo, d_radiance, d_medium_albedo, stream):
    return _call("mt_scene_set_params", scene, d_albedo, d_radiance, d_medium_albedo, stream)


def mt_film_create(H, W, T, Cc, start, width, d_film, d_steady, flags, out):
    return _call("mt_film_create", H, W, T, Cc, start, width, d_film, d_steady, flags, out)


def mt_render(scene, film, spp, seed, max_depth, sample_offset, stream):
    return _call("mt_render", scene, film, spp, seed, max_depth, sample_offset, stream)


def mt_render_to_host(scene, film, spp, seed, max_depth, sample_offset, band_rows, host_film, host_steady, stream,
                      copy_stream):
    return _call("mt_render_to_host", scene, film, spp, seed, max_depth, sample_offset, band_rows, host_film,
                 host_steady, stream, copy_stream)


def mt_render_nlos(scene, film, scan, spp, seed, sample_offset, stream):
    return _call("mt_render_nlos", scene, film, scan, spp, seed, sample_offset, stream)


def mt_render_backward(scene, film, d_grad_film, d_grad_steady, spp, seed, max_depth, sample_offset, d_grad_albedo,
                       d_grad_radiance, d_grad_medium_albedo, stream):
    return _call("mt_render_backward", scene, film, d_grad_film, d_grad_steady, spp, seed, max_depth, sample_offset,
                 d_grad_albedo, d_grad_radiance, d_grad_medium_albedo, stream)


def mt_sync(scene, stream):
    return _call("mt_sync", scene, stream)


def mt_read_counters(scene, out, reset, stream):
    return _call("mt_read_counters", scene, out, reset, stream)


def mt_scene_set_delays(scene, d_tau, stream):
    return _call("mt_scene_set_delays", scene, d_tau, stream)


def mt_scene_set_pulse(scene, shape, a, b):
    return _call("mt_scene_set_pulse", scene, shape, a, b)


def mt_render_tangent(scene, film, d_dalbedo, d_dradiance, dmedium, spp, seed, max_depth, sample_offset, stream):
    return _call("mt_render_tangent", scene, film, d_dalbedo, d_dradiance, dmedium, spp, seed, max_depth,
                 sample_offset, stream)


def mt_render_polarized(scene, film, spp, seed, max_depth, sample_offset, stream):
    return _call("mt_render_polarized", scene, film, spp, seed, max_depth, sample_offset, stream)


def mt_film_set_window(film, frame_H, row0):
    return _call("mt_film_set_window", film, frame_H, row0)


def mt_stage_times(scene, out, reset):
    return _call("mt_stage_times", scene, out, reset)


def mt_scene_stats(scene, out):
    return _call("mt_scene_stats", scene, out)


def mt_set_launch(scene, kind, threads, tile, ctas_per_sm, priv_bins, options):
    return _call("mt_set_launch", scene, kind, threads, tile, ctas_per_sm, priv_bins, options)


def mt_set_wavefront_pool(scene, max_paths):
    return _call("mt_set_wavefront_pool", scene, max_paths)


def mt_scene_destroy(scene):
    load().mt_scene_destroy(scene)


def mt_film_destroy(film):
    load().mt_film_destroy(film)


def mt_probe_philox(seed, d_counters, n, d_out, stream):
    return _call("mt_probe_philox", seed, d_counters, n, d_out, stream)


def mt_probe_trace(scene, d_rays, n, tmax, any_hit, d_tri, d_t, stream):
    return _call("mt_probe_trace", scene, d_rays, n, tmax, any_hit, d_tri, d_t, stream)


def mt_probe_bins(d_opl, n, start, width, T, d_bin, stream):
    return _call("mt_probe_bins", d_opl, n, start, width, T, d_bin, stream)


def mt_render_nlos_noalloc(scene, film, scan, spp, seed, sample_offset, stream):
    return _call("mt_render_nlos_noalloc", scene, film, scan, spp, seed, sample_offset, stream)


def mt_render_dump(scene, film, scan, spp, seed, max_depth, sample_offset, d_dump, cap, d_count, stream):
    return _call("mt_render_dump", scene, film, scan, spp, seed, max_depth, sample_offset, d_dump, cap, d_count, stream)


# --- conveniences ---------------------------------------------------------------
def _f3(v):
    return (C.c_float * 3)(*[float(x) for x in v])


class Scene:
    """A scene on the device (libmt handle) built from a scenes.Scene."""

    def __init__(self, sc: "_scenes.Scene", stream=None):
        self.sc = sc
        n = sc.n_tris
        tris = np.ascontiguousarray(sc.tris, np.float32)
        # mt_material rows (albedo[3], roughness, type bits) packed by torch's threaded cat into page-locked
        # memory from torch's host cache, so that the upload runs at copy-engine speed
        import torch
        alb = torch.from_numpy(np.ascontiguousarray(sc.albedo, np.float32))
        rough = torch.from_numpy(np.ascontiguousarray(sc.roughness, np.float32))
        mt = torch.from_numpy(np.ascontiguousarray(sc.mtype, np.uint32).view(np.float32))
        mats_t = torch.empty((n, 5), dtype=torch.float32, pin_memory=torch.cuda.is_available())
        torch.cat((alb, rough[:, None], mt[:, None]), dim=1, out=mats_t)
        mats = C.c_void_p(mats_t.data_ptr())  # read before mt_scene_create returns
        ne = len(sc.emitters)
        ems = (mt_emitter * max(ne, 1))()
        for i, e in enumerate(sc.emitters):
            ems[i] = mt_emitter(int(e["type"]), int(e["first_tri"]), int(e["n_tris"]), _f3(e["radiance"]),
                                _f3(e.get("position", (0, 0, 0))))
        cam = mt_camera(_f3(sc.camera["origin"]), _f3(sc.camera["target"]), _f3(sc.camera["up"]),
                        float(sc.camera["fov_x_deg"]))
        med = None
        self._dens = None
        if sc.medium is not None:
            m = sc.medium
            self._dens = np.ascontiguousarray(m["density"], np.float32)
            rz, ry, rx = self._dens.shape
            med = mt_medium(_f3(m["lo"]), _f3(m["hi"]), (C.c_int32 * 3)(rx, ry, rz),
                            self._dens.ctypes.data_as(C.c_void_p), float(m["albedo"]), float(m["g"]))
        h = C.c_void_p()
        mt_scene_create(tris.ctypes.data_as(C.c_void_p), n, mats, ems, ne, C.byref(cam),
                        C.byref(med) if med is not None else None, _stream(stream), C.byref(h))
        self.h = h
        self.n_tris = n
        self.n_em = ne

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                mt_scene_destroy(h)
            except Exception:
                pass
            self.h = None

    def set_params(self, albedo=None, radiance=None, medium_albedo=None, stream=None):
        """Albedos [n_tris, 3], radiances [n_em, 3], medium albedo [1]: float32 CUDA tensors or None."""
        _check_f32([(albedo, 3 * self.n_tris, "albedo"), (radiance, 3 * self.n_em, "radiance"),
                    (medium_albedo, 1, "medium albedo")])
        mt_scene_set_params(self.h, _ptr(albedo), _ptr(radiance), _ptr(medium_albedo), _stream(stream))

    def stats(self) -> dict:
        out = (C.c_int64 * 8)()
        mt_scene_stats(self.h, out)
        keys = ["n_tris", "bvh_nodes", "bvh_depth", "sah_x1000", "light_units", "device_bytes", "build_us",
                "launches"]
        return {k: int(out[i]) for i, k in enumerate(keys)}

    def set_delays(self, tau=None, stream=None):
        """Per-triangle exponential scattering-delay means (metres), a device
        float32 tensor [n_tris] (copied); None removes them."""
        if tau is not None:
            if not (tau.is_cuda and tau.dtype.is_floating_point and tau.numel() == self.n_tris):
                raise ValueError(f"delays must be a floating-point CUDA tensor of {self.n_tris} values")
            tau = tau.float().contiguous()
        mt_scene_set_delays(self.h, _ptr(tau) if tau is not None else None, _stream(stream))

    def set_pulse(self, shape=0, a=0.0, b=0.0):
        """Emission pulse of all emitters: MT_PULSE_DELTA / BOX (width a) /
        GAUSSIAN (mean a, deviation b) / EXPONENTIAL (mean a)."""
        mt_scene_set_pulse(self.h, int(shape), float(a), float(b))

    def stage_times(self, reset=True) -> dict:
        """Milliseconds per wavefront stage of renders run with MT_OPT_STAGE_TIMING:
        generate (with the extension-ray sort, if on), extend (the traversal pass:
        extension rays and, in the fused forward form, the shadow rays of the
        previous shading pass), shade (with the shadow-ray sort, if on), shadow
        (a shadow pass of its own: replay, polarization, dynamic fetch)."""
        out = (C.c_double * 5)()
        mt_stage_times(self.h, out, int(reset))
        keys = ["generate_ms", "extend_ms", "shade_ms", "shadow_ms", "iterations"]
        return {k: float(out[i]) for i, k in enumerate(keys)}

    def read_counters(self, reset=True, stream=None) -> dict:
        out = (C.c_uint64 * 8)()
        mt_read_counters(self.h, out, int(reset), _stream(stream))
        keys = ["vertices", "paths", "contributions", "rays", "node_bytes", "tri_tests", "smem_splats", "gmem_splats"]
        return {k: int(out[i]) for i, k in enumerate(keys)}

    def sync(self, stream=None):
        mt_sync(self.h, _stream(stream))

    def set_launch(self, kind, threads=0, tile=0, ctas_per_sm=0, priv_bins=-1, options=0):
        mt_set_launch(self.h, kind, threads, tile, ctas_per_sm, priv_bins, options)

    def set_wavefront_pool(self, max_paths=0):
        """Paths in flight of the wavefront form (0 = the default 4,194,304)."""
        mt_set_wavefront_pool(self.h, int(max_paths))


class Film:
    """A film handle over caller-owned torch tensors."""

    def __init__(self, film, steady, start, width, flags=0, C_=None, window=None):
        if film.dim() < (4 if C_ is None else 3):
            raise ValueError(f"film must be [H, W, T, C], not {tuple(film.shape)}")
        H, W, T = film.shape[:3]
        Cc = film.shape[3] if C_ is None else C_
        _check_f32([(film, H * W * T * Cc, "film")] + ([] if steady is None else [(steady, H * W * Cc, "steady image")]))
        self.film, self.steady = film, steady
        h = C.c_void_p()
        mt_film_create(H, W, T, Cc, float(start), float(width), _ptr(film), _ptr(steady), int(flags), C.byref(h))
        self.h = h
        if window is not None:  # (frame_H, row0): these rows of a taller frame
            mt_film_set_window(h, int(window[0]), int(window[1]))

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                mt_film_destroy(h)
            except Exception:
                pass


def new_film(H, W, T, Cc=3, device="cuda"):
    import torch
    return (torch.empty((H, W, T, Cc), dtype=torch.float32, device=device),
            torch.empty((H, W, Cc), dtype=torch.float32, device=device))


def render(scene: Scene, H, W, T, start, width, spp, seed, max_depth, sample_offset=0, flags=0, out=None,
           stream=None, window=None):
    """Transient render; returns (film [H,W,T,3], steady [H,W,3]) torch tensors.
    window=(frame_H, row0): the H rows are rows row0.. of a frame_H-row image."""
    film, steady = out if out is not None else new_film(H, W, T, 3)
    f = Film(film, steady, start, width, flags, window=window)
    mt_render(scene.h, f.h, spp, seed, max_depth, sample_offset, _stream(stream))
    return film, steady


def render_to_host(scene: Scene, H, W, T, start, width, spp, seed, max_depth, host_film, host_steady, band_rows,
                   copy_stream, sample_offset=0, flags=0, out=None, stream=None, window=None):
    """render() into the device film `out` (or a new one), with the film and
    steady image copied band by band (band_rows rows) into the page-locked host
    tensors host_film [H,W,T,3] / host_steady [H,W,3] on copy_stream as the
    bands finish; synchronise copy_stream before reading them."""
    film, steady = out if out is not None else new_film(H, W, T, 3)
    # the library copies the whole film and steady image into these host buffers
    for h, d, what in ((host_film, film, "host film"), (host_steady, steady, "host steady image")):
        if h is not None and d is not None and h.numel() != d.numel():
            raise ValueError(f"{what} holds {h.numel()} values where the film copies {d.numel()}")
    f = Film(film, steady, start, width, flags, window=window)
    mt_render_to_host(scene.h, f.h, spp, seed, max_depth, sample_offset, band_rows, _hptr(host_film),
                      _hptr(host_steady), _stream(stream), _stream(copy_stream))
    return film, steady


def mt_render_phasor(scene, film, d_lambdas, K, spp, seed, max_depth, sample_offset, stream):
    return _call("mt_render_phasor", scene, film, d_lambdas, K, spp, seed, max_depth, sample_offset, stream)


def render_phasor(scene: Scene, H, W, lambdas, spp, seed, max_depth, sample_offset=0, flags=0, stream=None):
    """Frequency-space film [H, W, K, 2 (re, im), 3] and the steady image [H, W, 3]."""
    import torch
    lam = torch.as_tensor(lambdas, dtype=torch.float32, device="cuda").contiguous()
    K = lam.shape[0]
    film = torch.empty((H, W, 2 * K, 3), dtype=torch.float32, device="cuda")
    steady = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    f = Film(film, steady, 0.0, 1.0, flags)
    mt_render_phasor(scene.h, f.h, _ptr(lam), K, spp, seed, max_depth, sample_offset, _stream(stream))
    return film.view(H, W, K, 2, 3), steady


def render_tangent(scene: Scene, H, W, T, start, width, spp, seed, max_depth, dalbedo=None, dradiance=None,
                   dmedium=0.0, sample_offset=0, flags=0, out=None, stream=None):
    """Forward-mode derivative film dI/dtheta . dtheta [H, W, T, 3] and its
    steady image for the tangent (dalbedo [n_tris, 3], dradiance [n_em, 3],
    dmedium) on the same paths as render()."""
    film, steady = out if out is not None else new_film(H, W, T, 3)
    f = Film(film, steady, start, width, flags)
    da = None if dalbedo is None else dalbedo.float().contiguous()
    dr = None if dradiance is None else dradiance.float().contiguous()
    _check_f32([(da, 3 * scene.n_tris, "albedo tangent"), (dr, 3 * scene.n_em, "radiance tangent")])
    mt_render_tangent(scene.h, f.h, _ptr(da), _ptr(dr), float(dmedium), spp, seed, max_depth, sample_offset,
                      _stream(stream))
    return film, steady


def render_polarized(scene: Scene, H, W, T, start, width, spp, seed, max_depth, sample_offset=0, flags=0, out=None,
                     stream=None, window=None):
    """Transient polarization: Stokes film [H, W, T, 4, 3] and steady Stokes image [H, W, 4, 3]."""
    import torch
    if out is None:
        film = torch.empty((H, W, T, 4, 3), dtype=torch.float32, device="cuda")
        steady = torch.empty((H, W, 4, 3), dtype=torch.float32, device="cuda")
    else:
        film, steady = out
    f = Film(film, steady, start, width, flags, C_=12, window=window)
    mt_render_polarized(scene.h, f.h, spp, seed, max_depth, sample_offset, _stream(stream))
    return film, steady


def render_backward(scene: Scene, T, start, width, spp, seed, max_depth, grad_film, grad_steady=None,
                    sample_offset=0, flags=0, out=None, stream=None):
    """Path-replay gradients (accumulated into `out` if given)."""
    import torch
    H, W = grad_film.shape[:2]
    if out is None:
        out = (torch.zeros((scene.n_tris, 3), dtype=torch.float32, device="cuda"),
               torch.zeros((max(scene.n_em, 1), 3), dtype=torch.float32, device="cuda"),
               torch.zeros(1, dtype=torch.float32, device="cuda"))
    galb, grad, gmed = out
    f = Film(grad_film, None, start, width, flags)
    _check_f32([(grad_steady, H * W * 3, "steady-image gradient")])
    _check_f32([(galb, 3 * scene.n_tris, "albedo gradient"), (grad, 3 * scene.n_em, "radiance gradient"),
                (gmed, 1, "medium-albedo gradient")], at_least=True)
    mt_render_backward(scene.h, f.h, _ptr(grad_film), _ptr(grad_steady), spp, seed, max_depth, sample_offset,
                       _ptr(galb), _ptr(grad), _ptr(gmed), _stream(stream))
    del H, W
    return galb, grad, gmed


def make_scan(lasers, sensors, mode, wall_normal, wall_albedo, hidden):
    """Scan grid of laser (and, for EXHAUSTIVE grids, sensor) points on the relay
    wall: float32 CUDA tensors [n, 3]."""
    for t, what in ((lasers, "laser points"), (sensors, "sensor points")):
        if t is not None and (t.dim() != 2 or t.shape[1] != 3):
            raise ValueError(f"{what} must be [n, 3], not {tuple(t.shape)}")
    _check_f32([(lasers, 3 * lasers.shape[0], "laser points"),
                (sensors, 3 * sensors.shape[0] if sensors is not None else 0, "sensor points")])
    return mt_scan(_ptr(lasers), int(lasers.shape[0]), _ptr(sensors) if sensors is not None else None,
                   int(sensors.shape[0]) if sensors is not None else 0, int(mode), _f3(wall_normal),
                   float(wall_albedo), int(hidden[0]), int(hidden[1]))


def render_nlos(scene: Scene, lasers, sensors, mode, T, start, width, spp, seed, sample_offset=0, flags=0,
                out=None, stream=None):
    """Relay-wall impulse responses; returns (film [rows, T], steady [rows])."""
    import torch
    rows = lasers.shape[0] * (sensors.shape[0] if mode == MT_EXHAUSTIVE else 1)
    if out is None:
        out = (torch.empty((rows, T), dtype=torch.float32, device="cuda"),
               torch.empty((rows,), dtype=torch.float32, device="cuda"))
    film, steady = out
    sc = scene.sc
    scan = make_scan(lasers, sensors if mode == MT_EXHAUSTIVE else None, mode, sc.wall["normal"], sc.wall["albedo"],
                     sc.hidden)
    f = Film(film.view(rows, 1, T, 1), steady, start, width, flags)
    mt_render_nlos(scene.h, f.h, C.byref(scan), spp, seed, sample_offset, _stream(stream))
    return film, steady


def render_dump(scene: Scene, H, W, T, start, width, spp, seed, max_depth, cap, sample_offset=0, flags=0,
                scan_args=None, stream=None, window=None):
    """Forward render (or NLOS when scan_args is given) that also returns every
    contribution record as a numpy structured array (CONTRIB_DTYPE)."""
    import torch
    dump = torch.empty((max(cap, 1), 10), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    if scan_args is None:
        film, steady = new_film(H, W, T, 3)
        f = Film(film, steady, start, width, flags, window=window)
        mt_render_dump(scene.h, f.h, None, spp, seed, max_depth, sample_offset, _ptr(dump), cap, _ptr(cnt),
                       _stream(stream))
    else:
        lasers, sensors, mode = scan_args
        rows = lasers.shape[0] * (sensors.shape[0] if mode == MT_EXHAUSTIVE else 1)
        film = torch.empty((rows, 1, T, 1), dtype=torch.float32, device="cuda")
        steady = torch.empty((rows, 1, 1), dtype=torch.float32, device="cuda")
        sc = scene.sc
        scan = make_scan(lasers, sensors if mode == MT_EXHAUSTIVE else None, mode, sc.wall["normal"],
                         sc.wall["albedo"], sc.hidden)
        f = Film(film, steady, start, width, flags)
        mt_render_dump(scene.h, f.h, C.byref(scan), spp, seed, max_depth, sample_offset, _ptr(dump), cap,
                       _ptr(cnt), _stream(stream))
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    n = int(cnt.item())
    rec = dump[:min(n, cap)].cpu().numpy().view(CONTRIB_DTYPE).reshape(-1)
    return film, steady, rec, n


MT_MICRO_GATHER32, MT_MICRO_RED_GLOBAL, MT_MICRO_RED_SHARED = 0, 1, 2


def mt_microbench(kind, d_buf, nbytes, iters, out_rate, stream):
    return _call("mt_microbench", kind, d_buf, nbytes, iters, out_rate, stream)


def microbench(kind, nbytes=64 << 20, iters=256):
    """Measured rate of one access pattern (GB/s for gathers, Gop/s for atomics)."""
    import torch
    buf = torch.zeros(max(nbytes, 4096) // 4, dtype=torch.float32, device="cuda")
    rate = C.c_double(0.0)
    mt_microbench(kind, _ptr(buf), buf.numel() * 4, iters, C.byref(rate), _stream())
    return rate.value


def probe_philox(seed, counters):
    import torch
    out = torch.empty_like(counters)
    mt_probe_philox(int(seed), _ptr(counters), counters.shape[0], _ptr(out), _stream())
    return out


def probe_trace(scene: Scene, rays, tmax=float("inf"), any_hit=False, wide=False):
    """Closest (or any) hits of rays [n][6]; wide=True traverses the 8-wide BVH."""
    import torch
    n = rays.shape[0]
    tri = torch.empty(n, dtype=torch.int32, device="cuda")
    t = torch.empty(n, dtype=torch.float32, device="cuda")
    mode = (1 if any_hit else 0) | (2 if wide else 0)
    mt_probe_trace(scene.h, _ptr(rays), n, float(tmax), mode, _ptr(tri), _ptr(t), _stream())
    return tri, t


def probe_bins(opl, start, width, T):
    import torch
    out = torch.empty(opl.shape[0], dtype=torch.int32, device="cuda")
    mt_probe_bins(_ptr(opl), opl.shape[0], float(start), float(width), int(T), _ptr(out), _stream())
    return out


def _autograd():
    import torch

    class TransientRender(torch.autograd.Function):
        """(albedo [n,3], radiance [e,3]) -> (film [H,W,T,3], steady [H,W,3]).

        Forward is mt_render with the given parameters; backward is
        mt_render_backward (path replay, Sec. 4.4) with the same seed."""

        @staticmethod
        def forward(ctx, albedo, radiance, scene, H, W, T, start, width, spp, seed, max_depth):
            scene.set_params(albedo=albedo.detach().contiguous(), radiance=radiance.detach().contiguous())
            film, steady = render(scene, H, W, T, start, width, spp, seed, max_depth)
            ctx.args = (scene, T, start, width, spp, seed, max_depth)
            ctx.hw = (H, W)
            ctx.save_for_backward(albedo, radiance)
            return film, steady

        @staticmethod
        def backward(ctx, g_film, g_steady):
            scene, T, start, width, spp, seed, max_depth = ctx.args
            albedo, radiance = ctx.saved_tensors
            scene.set_params(albedo=albedo.detach().contiguous(), radiance=radiance.detach().contiguous())
            g_film = g_film.contiguous() if g_film is not None else None
            g_steady = g_steady.contiguous() if g_steady is not None else None
            if g_film is None:
                H, W = ctx.hw
                g_film = torch.zeros((H, W, T, 3), device="cuda")
            ga, gr, _ = render_backward(scene, T, start, width, spp, seed, max_depth, g_film, g_steady)
            return ga, gr[:radiance.shape[0]], None, None, None, None, None, None, None, None, None

    return TransientRender


_transient_render = None


def __getattr__(name):
    # built on first use, so that importing the binding does not import torch
    global _transient_render
    if name == "TransientRender":
        if _transient_render is None:
            _transient_render = _autograd()
        return _transient_render
    raise AttributeError(name)
