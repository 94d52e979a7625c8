"""ctypes binding of the FP64 C oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The oracle is a plain single-threaded
double-precision path tracer written from arXiv 2510.25660 (Sec. 3 Eqs. 1-9,
path reuse and camera unwarping; Sec. 4.1 media; Sec. 4.4 backward mode;
Sec. 4.5 NLOS).  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mt_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libmt_oracle.so")

UNWARP = 1
ACCUMULATE = 2
PIXEL_CENTER = 4
PULSE_DELTA, PULSE_BOX, PULSE_GAUSSIAN, PULSE_EXPONENTIAL = 0, 1, 2, 3
STRAT_MIS, STRAT_NEE_ONLY, STRAT_BSDF_ONLY = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 (FP64, no fast-math)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    hdr = os.path.join(_HERE, "mt_oracle.h")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class Contrib(C.Structure):
    _fields_ = [("pixel", C.c_int32), ("sample", C.c_int32), ("depth", C.c_int32), ("kind", C.c_int32),
                ("tri", C.c_int32), ("bin", C.c_int32), ("opl", C.c_double), ("c", C.c_double * 3)]


CONTRIB_DTYPE = np.dtype([("pixel", np.int32), ("sample", np.int32), ("depth", np.int32), ("kind", np.int32),
                          ("tri", np.int32), ("bin", np.int32), ("opl", np.float64), ("c", np.float64, (3,))])


class Args(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("T", C.c_int32), ("start", C.c_double),
                ("width", C.c_double), ("flags", C.c_uint32), ("spp", C.c_int32), ("seed", C.c_uint64),
                ("max_depth", C.c_int32), ("sample_offset", C.c_uint64), ("x0", C.c_int32),
                ("x1", C.c_int32), ("y0", C.c_int32), ("y1", C.c_int32), ("strategy", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.mo_scene_create.restype = P
        _lib.mo_scene_create.argtypes = [P, C.c_int64, P, P, P, C.c_int32, P, P, P, P, P, P, P, P, P]
        _lib.mo_scene_destroy.argtypes = [P]
        _lib.mo_scene_set_params.argtypes = [P, P, P, C.c_double]
        _lib.mo_scene_set_delays.restype = C.c_int
        _lib.mo_scene_set_delays.argtypes = [P, P]
        _lib.mo_scene_set_pulse.restype = C.c_int
        _lib.mo_scene_set_pulse.argtypes = [P, C.c_int, C.c_double, C.c_double]
        _lib.mo_philox4x32_10.argtypes = [P, P, P]
        _lib.mo_philox_batch.argtypes = [P, C.c_int64, C.c_uint64, P]
        _lib.mo_intersect.restype = C.c_int64
        _lib.mo_intersect.argtypes = [P, P, P, C.c_double, C.c_int, P]
        _lib.mo_occluded.restype = C.c_int
        _lib.mo_occluded.argtypes = [P, P, P, C.c_double, C.c_int]
        _lib.mo_camera_ray.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, P, P]
        _lib.mo_bsdf_eval.restype = C.c_double
        _lib.mo_bsdf_eval.argtypes = [C.c_uint32, P, C.c_double, P, P, P, P, P]
        _lib.mo_bsdf_sample.restype = C.c_int
        _lib.mo_bsdf_sample.argtypes = [C.c_uint32, P, C.c_double, P, P, C.c_double, C.c_double, P, P, P]
        _lib.mo_hg_eval.restype = C.c_double
        _lib.mo_hg_eval.argtypes = [C.c_double, C.c_double]
        _lib.mo_hg_sample.argtypes = [C.c_double, P, C.c_double, C.c_double, P]
        _lib.mo_density.restype = C.c_double
        _lib.mo_density.argtypes = [P, P]
        _lib.mo_majorant.restype = C.c_double
        _lib.mo_majorant.argtypes = [P]
        _lib.mo_track.restype = C.c_double
        _lib.mo_track.argtypes = [P, P, P, C.c_double, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int]
        _lib.mo_render.restype = C.c_int
        _lib.mo_render.argtypes = [P, P, P, P, P, P, C.c_int64, P, P]
        _lib.mo_render_phasor.restype = C.c_int
        _lib.mo_render_phasor.argtypes = [P, P, P, C.c_int32, P, P]
        _lib.mo_render_polarized.restype = C.c_int
        _lib.mo_render_polarized.argtypes = [P, P, P, P]
        _lib.mo_conductor_kappa.restype = C.c_double
        _lib.mo_conductor_kappa.argtypes = [C.c_double]
        _lib.mo_render_tangent.restype = C.c_int
        _lib.mo_render_tangent.argtypes = [P, P, P, P, C.c_double, P, P]
        _lib.mo_render_backward.restype = C.c_int
        _lib.mo_render_backward.argtypes = [P, P, P, P, P, P, P]
        _lib.mo_render_nlos.restype = C.c_int
        _lib.mo_render_nlos.argtypes = [P, C.c_int32, C.c_int32, P, C.c_double, P, C.c_int32, P, C.c_int32,
                                        C.c_int32, C.c_int64, C.c_int64, C.c_int32, C.c_double, C.c_double,
                                        C.c_int32, C.c_uint64, C.c_uint64, C.c_uint32, P, P, P, C.c_int64, P, P]
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def conductor_kappa(F0: float) -> float:
    """Extinction coefficient of the polarized conductor model (index 1 + i kappa) for reflectance F0."""
    return float(lib().mo_conductor_kappa(float(F0)))


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one counter (4 x u32) under key (2 x u32)."""
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib().mo_philox4x32_10(_p(c), _p(k), _p(o))
    return o


def philox_batch(ctr, seed) -> np.ndarray:
    """Philox4x32-10 of n counters [n, 4] under key (seed_lo, seed_hi)."""
    c = np.ascontiguousarray(ctr, np.uint32)
    o = np.zeros_like(c)
    lib().mo_philox_batch(_p(c), c.shape[0], int(seed), _p(o))
    return o


class OracleScene:
    """Host FP64 copy of a scene (scenes.Scene) with its own median-split BVH."""

    def __init__(self, sc):
        L = lib()
        self.sc = sc
        self._keep = []
        tris = np.ascontiguousarray(sc.tris, np.float32)
        alb = np.ascontiguousarray(sc.albedo, np.float32)
        rough = np.ascontiguousarray(sc.roughness, np.float32)
        mt = np.ascontiguousarray(sc.mtype, np.uint32)
        ne = len(sc.emitters)
        et = np.array([e["type"] for e in sc.emitters] or [0], np.int32)
        ef = np.array([e["first_tri"] for e in sc.emitters] or [0], np.int32)
        en = np.array([e["n_tris"] for e in sc.emitters] or [0], np.int32)
        er = np.array([e["radiance"] for e in sc.emitters] or [(0, 0, 0)], np.float64).reshape(-1)
        ep = np.array([e.get("position", (0, 0, 0)) for e in sc.emitters] or [(0, 0, 0)], np.float64).reshape(-1)
        cam = sc.camera
        camv = np.array(list(cam["origin"]) + list(cam["target"]) + list(cam["up"]) + [cam["fov_x_deg"]], np.float64)
        dens = res = med = None
        if sc.medium is not None:
            m = sc.medium
            dens = np.ascontiguousarray(m["density"], np.float32)
            rz, ry, rx = dens.shape
            res = np.array([rx, ry, rz], np.int32)
            med = np.array(list(m["lo"]) + list(m["hi"]) + [m["albedo"], m["g"]], np.float64)
        self._keep = [tris, alb, rough, mt, et, ef, en, er, ep, camv, dens, res, med]
        self.h = L.mo_scene_create(_p(tris), tris.shape[0], _p(alb), _p(rough), _p(mt), ne, _p(et), _p(ef),
                                   _p(en), _p(er), _p(ep), _p(camv), _p(dens), _p(res), _p(med))
        self.n_tris = tris.shape[0]
        self.n_em = ne

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().mo_scene_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def set_params(self, albedo=None, radiance=None, medium_albedo=None):
        a = None if albedo is None else np.ascontiguousarray(albedo, np.float64).reshape(-1)
        r = None if radiance is None else np.ascontiguousarray(radiance, np.float64).reshape(-1)
        lib().mo_scene_set_params(self.h, _p(a), _p(r), float("nan") if medium_albedo is None else float(medium_albedo))

    def set_delays(self, tau=None):
        """Per-triangle exponential scattering-delay means (metres of light travel); None clears."""
        t = None if tau is None else np.ascontiguousarray(tau, np.float64).reshape(-1)
        if t is not None and t.shape[0] != self.n_tris:
            raise ValueError("one delay per triangle")
        if lib().mo_scene_set_delays(self.h, _p(t)) != 0:
            raise ValueError("bad delay")

    def set_pulse(self, kind=0, a=0.0, b=0.0):
        """Emission pulse: 0 delta, 1 box [0, a), 2 Gaussian (mean a, deviation b), 3 exponential (mean a)."""
        if lib().mo_scene_set_pulse(self.h, int(kind), float(a), float(b)) != 0:
            raise ValueError("bad pulse")

    # -- geometry queries -------------------------------------------------
    def intersect(self, o, d, tmax=np.inf, brute=False):
        t = C.c_double(0.0)
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        i = lib().mo_intersect(self.h, _p(o), _p(d), float(tmax), int(brute), C.byref(t))
        return int(i), t.value

    def occluded(self, o, d, tmax, brute=False):
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        return bool(lib().mo_occluded(self.h, _p(o), _p(d), float(tmax), int(brute)))

    def camera_ray(self, W, H, px, py, jx=0.5, jy=0.5):
        o = np.zeros(3)
        d = np.zeros(3)
        lib().mo_camera_ray(self.h, W, H, px, py, jx, jy, _p(o), _p(d))
        return o, d

    def density(self, p):
        p = np.ascontiguousarray(p, np.float64)
        return lib().mo_density(self.h, _p(p))

    def majorant(self):
        return lib().mo_majorant(self.h)

    def track(self, o, d, dist, seed, a, b, method):
        """One transmittance estimate: method 0 ratio tracking, 1 delta tracking."""
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        return lib().mo_track(self.h, _p(o), _p(d), float(dist), int(seed), int(a), int(b), int(method))

    # -- estimators ---------------------------------------------------------
    def render(self, H, W, T, start, width, spp, seed, max_depth, flags=0, sample_offset=0, crop=None,
               strategy=STRAT_MIS, dump_cap=0, want_dropped=False):
        x0, x1, y0, y1 = crop if crop is not None else (0, W, 0, H)
        npx = (x1 - x0) * (y1 - y0)
        film = np.zeros((y1 - y0, x1 - x0, T, 3), np.float64)
        steady = np.zeros((y1 - y0, x1 - x0, 3), np.float64)
        dropped = np.zeros((y1 - y0, x1 - x0, 3), np.float64) if want_dropped else None
        a = Args(H, W, T, start, width, flags, spp, seed, max_depth, sample_offset, x0, x1, y0, y1, strategy)
        dump = np.zeros(max(dump_cap, 0), CONTRIB_DTYPE) if dump_cap else None
        nd = C.c_int64(0)
        cnt = np.zeros(4, np.uint64)
        rc = lib().mo_render(self.h, C.byref(a), _p(film), _p(steady), _p(dropped), _p(dump), int(dump_cap),
                             C.byref(nd), _p(cnt))
        if rc:
            raise ValueError("oracle render: invalid arguments")
        out = dict(film=film, steady=steady, counters=dict(vertices=int(cnt[0]), rays=int(cnt[1]),
                                                           contributions=int(cnt[2]), paths=int(cnt[3])))
        if dropped is not None:
            out["dropped"] = dropped
        if dump is not None:
            out["dump"] = dump[:min(nd.value, dump_cap)]
            out["n_dump"] = nd.value
        del npx
        return out

    def render_tangent(self, H, W, T, start, width, spp, seed, max_depth, dalb=None, drad=None, dmed=0.0, flags=0,
                       sample_offset=0, crop=None):
        """Forward-mode derivative film dI/dtheta . dtheta (crop-sized) and its steady image."""
        x0, x1, y0, y1 = crop if crop is not None else (0, W, 0, H)
        film = np.zeros((y1 - y0, x1 - x0, T, 3), np.float64)
        steady = np.zeros((y1 - y0, x1 - x0, 3), np.float64)
        a = Args(H, W, T, start, width, flags, spp, seed, max_depth, sample_offset, x0, x1, y0, y1, STRAT_MIS)
        da = None if dalb is None else np.ascontiguousarray(dalb, np.float64).reshape(-1)
        dr = None if drad is None else np.ascontiguousarray(drad, np.float64).reshape(-1)
        if lib().mo_render_tangent(self.h, C.byref(a), _p(da), _p(dr), float(dmed), _p(film), _p(steady)):
            raise ValueError("oracle tangent render: invalid arguments")
        return dict(film=film, steady=steady)

    def render_polarized(self, H, W, T, start, width, spp, seed, max_depth, flags=0, sample_offset=0, crop=None):
        """Stokes film [h, w, T, 4, 3] and steady Stokes image [h, w, 4, 3] (crop-sized)."""
        x0, x1, y0, y1 = crop if crop is not None else (0, W, 0, H)
        film = np.zeros((y1 - y0, x1 - x0, T, 4, 3), np.float64)
        steady = np.zeros((y1 - y0, x1 - x0, 4, 3), np.float64)
        a = Args(H, W, T, start, width, flags, spp, seed, max_depth, sample_offset, x0, x1, y0, y1, STRAT_MIS)
        if lib().mo_render_polarized(self.h, C.byref(a), _p(film), _p(steady)):
            raise ValueError("oracle polarized render: invalid arguments")
        return dict(film=film, steady=steady)

    def render_phasor(self, H, W, lambdas, spp, seed, max_depth, flags=0, sample_offset=0, crop=None):
        """Frequency-space film [h, w, K, 2 (re, im), 3] (Sec. 4.3) and the steady image."""
        x0, x1, y0, y1 = crop if crop is not None else (0, W, 0, H)
        lam = np.ascontiguousarray(lambdas, np.float64)
        K = lam.shape[0]
        ph = np.zeros((y1 - y0, x1 - x0, K, 2, 3), np.float64)
        steady = np.zeros((y1 - y0, x1 - x0, 3), np.float64)
        a = Args(H, W, 0, 0.0, 1.0, flags, spp, seed, max_depth, sample_offset, x0, x1, y0, y1, STRAT_MIS)
        rc = lib().mo_render_phasor(self.h, C.byref(a), _p(lam), K, _p(ph), _p(steady))
        if rc:
            raise ValueError("oracle phasor: invalid arguments")
        return dict(phasor=ph, steady=steady)

    def render_backward(self, H, W, T, start, width, spp, seed, max_depth, grad_film, grad_steady=None,
                        flags=0, sample_offset=0, crop=None):
        x0, x1, y0, y1 = crop if crop is not None else (0, W, 0, H)
        gf = np.ascontiguousarray(grad_film, np.float64)
        assert gf.shape == (y1 - y0, x1 - x0, T, 3), gf.shape
        gs = None if grad_steady is None else np.ascontiguousarray(grad_steady, np.float64)
        ga = np.zeros((self.n_tris, 3))
        gr = np.zeros((max(self.n_em, 1), 3))
        gm = C.c_double(0.0)
        a = Args(H, W, T, start, width, flags, spp, seed, max_depth, sample_offset, x0, x1, y0, y1, STRAT_MIS)
        rc = lib().mo_render_backward(self.h, C.byref(a), _p(gf), _p(gs), _p(ga), _p(gr), C.byref(gm))
        if rc:
            raise ValueError("oracle backward: invalid arguments")
        return dict(albedo=ga, radiance=gr[:self.n_em], medium_albedo=gm.value)

    def render_nlos(self, lasers, sensors, exhaustive, T, start, width, spp, seed, pair_range=None,
                    flags=0, sample_offset=0, dump_cap=0):
        sc = self.sc
        hf, hn = sc.hidden
        wall = sc.wall
        nw = np.array(wall["normal"], np.float64)
        las = np.ascontiguousarray(lasers, np.float32)
        sen = np.ascontiguousarray(sensors if sensors is not None else lasers, np.float32)
        nl, ns = las.shape[0], sen.shape[0]
        npairs = nl * ns if exhaustive else nl
        p0, p1 = pair_range if pair_range is not None else (0, npairs)
        film = np.zeros((p1 - p0, T), np.float64)
        steady = np.zeros(p1 - p0, np.float64)
        dump = np.zeros(max(dump_cap, 0), CONTRIB_DTYPE) if dump_cap else None
        nd = C.c_int64(0)
        cnt = np.zeros(4, np.uint64)
        rc = lib().mo_render_nlos(self.h, hf, hn, _p(nw), float(wall["albedo"]), _p(las), nl, _p(sen), ns,
                                  int(bool(exhaustive)), p0, p1, T, start, width, spp, seed, sample_offset,
                                  flags, _p(film), _p(steady), _p(dump), int(dump_cap), C.byref(nd), _p(cnt))
        if rc:
            raise ValueError("oracle nlos: invalid arguments")
        out = dict(film=film, steady=steady, counters=dict(connections=int(cnt[3]), rays=int(cnt[1]),
                                                           contributions=int(cnt[2])))
        if dump is not None:
            out["dump"] = dump[:min(nd.value, dump_cap)]
            out["n_dump"] = nd.value
        return out


def bsdf_eval(mtype, albedo, rough, ng, wo, wi):
    f = np.zeros(3)
    pdf = C.c_double(0)
    al = np.ascontiguousarray(albedo, np.float64)
    lib().mo_bsdf_eval(int(mtype), _p(al), float(rough), _p(np.ascontiguousarray(ng, np.float64)),
                       _p(np.ascontiguousarray(wo, np.float64)), _p(np.ascontiguousarray(wi, np.float64)),
                       _p(f), C.byref(pdf))
    return f, pdf.value


def bsdf_sample(mtype, albedo, rough, ng, wo, u0, u1):
    wi = np.zeros(3)
    w = np.zeros(3)
    pdf = C.c_double(0)
    al = np.ascontiguousarray(albedo, np.float64)
    ok = lib().mo_bsdf_sample(int(mtype), _p(al), float(rough), _p(np.ascontiguousarray(ng, np.float64)),
                              _p(np.ascontiguousarray(wo, np.float64)), float(u0), float(u1), _p(wi), _p(w),
                              C.byref(pdf))
    return bool(ok), wi, w, pdf.value


def hg_eval(g, cos_theta):
    return lib().mo_hg_eval(float(g), float(cos_theta))


def hg_sample(g, d, u0, u1):
    wi = np.zeros(3)
    lib().mo_hg_sample(float(g), _p(np.ascontiguousarray(d, np.float64)), float(u0), float(u1), _p(wi))
    return wi
