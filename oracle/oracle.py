"""ctypes front end of the FP64 C oracle (test infrastructure only).

The C file ``oracle.c`` restates the method step by step in double precision;
this module compiles it with gcc, marshals numpy arrays into its structs and
returns complex128 fields.  Nothing here is used by the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, IEEE double, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class OrScene(C.Structure):
    _fields_ = [("nv", C.c_int32), ("nt", C.c_int32), ("nm", C.c_int32), ("ntex", C.c_int32),
                ("nl", C.c_int32), ("npts", C.c_int32),
                ("verts", C.c_void_p), ("normals", C.c_void_p), ("uvs", C.c_void_p),
                ("tris", C.c_void_p), ("tri_mat", C.c_void_p),
                ("mat_type", C.c_void_p), ("mat_albedo", C.c_void_p), ("mat_rough", C.c_void_p),
                ("mat_ior", C.c_void_p), ("mat_Le", C.c_void_p), ("mat_tex", C.c_void_p),
                ("mat_emit_tex", C.c_void_p), ("mat_light", C.c_void_p),
                ("tex_data", C.c_void_p), ("tex_info", C.c_void_p), ("lights", C.c_void_p),
                ("points", C.c_void_p), ("cache_res", C.c_int32),
                ("cache_bmin", C.c_void_p), ("cache_bmax", C.c_void_p), ("cache_E", C.c_void_p)]


class OrRender(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("pitch", C.c_double), ("n_lambda", C.c_int32),
                ("lam", C.c_double * 3), ("channel", C.c_int32 * 3), ("spp", C.c_int32),
                ("max_depth", C.c_int32), ("K", C.c_int32), ("hologram_offset", C.c_int32),
                ("seed", C.c_uint64), ("phase_seed", C.c_uint64), ("phase_mode", C.c_int32),
                ("facet_size", C.c_double), ("T", C.c_double * 16), ("use_cache", C.c_int32),
                ("grf_nx", C.c_int32), ("grf_ny", C.c_int32), ("grf_phi", C.c_void_p), ("omit_obliquity", C.c_int32)]


class OrBake(C.Structure):
    _fields_ = [("res", C.c_int32), ("bmin", C.c_double * 3), ("bmax", C.c_double * 3), ("spp", C.c_int32),
                ("max_depth", C.c_int32), ("seed", C.c_uint64)]


REC_FIELDS = ["L", "beta", "opl", "r", "cos", "cosP", "vP", "Px", "Py", "Pz", "tri", "flags",
              "re", "im", "nrays", "u0", "Qx", "Qy"]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.or_build.restype = C.c_void_p
            lib.or_build.argtypes = [C.POINTER(OrScene)]
            lib.or_free.argtypes = [C.c_void_p]
            lib.or_trace.restype = C.c_int
            lib.or_trace.argtypes = [C.c_void_p, C.POINTER(OrRender), C.c_void_p, C.c_int64,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
            lib.or_sample.restype = C.c_int
            lib.or_sample.argtypes = [C.c_void_p, C.POINTER(OrRender), C.c_int, C.c_int64, C.c_int, C.c_void_p]
            lib.or_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            lib.or_bake.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int]
            lib.or_bake.restype = C.c_int
            lib.or_bake_sens.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int]
            lib.or_bake_sens.restype = C.c_int
            lib.or_grf_phases.argtypes = [C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]
            lib.or_grf_phases.restype = None
            lib.or_cone_dir.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p,
                                        C.POINTER(C.c_double)]
            lib.or_closest_hit.restype = C.c_int
            lib.or_closest_hit.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                           C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int32)]
            lib.or_fresnel_dielectric.restype = C.c_double
            lib.or_fresnel_dielectric.argtypes = [C.c_double, C.c_double, C.c_double]
            lib.or_ggx_eval.argtypes = [C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double)]
            lib.or_ggx_sample.restype = C.c_int
            lib.or_ggx_sample.argtypes = [C.c_double, C.c_double, C.c_void_p, C.c_double, C.c_double,
                                          C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            lib.or_frame.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            lib.or_tex_lookup.restype = C.c_double
            lib.or_tex_lookup.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_int32]
            lib.or_cache_lookup.restype = C.c_double
            lib.or_cache_lookup.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
            lib.or_half_to_double.restype = C.c_double
            lib.or_half_to_double.argtypes = [C.c_uint16]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data if a is not None else None


def _render_struct(r, grf=None) -> OrRender:
    """grf: phase maps [K][ny][nx] (radians, float64) for phase_mode 2, kept alive by the caller."""
    s = OrRender()
    s.W, s.H, s.pitch = int(r.W), int(r.H), float(r.pitch)
    s.n_lambda = len(r.lambdas)
    for i, (l, c) in enumerate(zip(r.lambdas, r.channels)):
        s.lam[i] = float(l)
        s.channel[i] = int(c)
    s.spp, s.max_depth, s.K, s.hologram_offset = int(r.spp), int(r.max_depth), int(r.K), int(r.hologram_offset)
    s.seed, s.phase_seed, s.phase_mode = int(r.seed), int(r.phase_seed), int(r.phase_mode)
    s.facet_size = float(r.facet_size)
    T = np.asarray(r.T, np.float64).reshape(16)
    for i in range(16):
        s.T[i] = float(T[i])
    s.use_cache = int(r.use_cache)
    s.omit_obliquity = int(getattr(r, "omit_obliquity", 0))
    if grf is not None:
        assert grf.dtype == np.float64 and grf.flags.c_contiguous and grf.ndim == 3 and grf.shape[0] >= r.K
        s.grf_ny, s.grf_nx = int(grf.shape[1]), int(grf.shape[2])
        s.grf_phi = grf.ctypes.data
    return s


class Oracle:
    """FP64 oracle bound to one scene (arrays are kept alive by this object)."""

    def __init__(self, scene):
        lib = _load()
        self._keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a

        s = OrScene()
        s.nv, s.nt, s.nm = len(scene.verts), len(scene.tris), len(scene.mat_type)
        s.ntex, s.nl, s.npts = len(scene.tex_info), len(scene.lights), len(scene.points)
        s.verts = _ptr(arr(scene.verts, np.float32))
        s.normals = _ptr(arr(scene.normals, np.float32))
        s.uvs = _ptr(arr(scene.uvs, np.float32))
        s.tris = _ptr(arr(scene.tris, np.uint32))
        s.tri_mat = _ptr(arr(scene.tri_mat, np.uint32))
        s.mat_type = _ptr(arr(scene.mat_type, np.int32))
        s.mat_albedo = _ptr(arr(scene.mat_albedo, np.float32))
        s.mat_rough = _ptr(arr(scene.mat_rough, np.float32))
        s.mat_ior = _ptr(arr(scene.mat_ior, np.float32))
        s.mat_Le = _ptr(arr(scene.mat_Le, np.float32))
        s.mat_tex = _ptr(arr(scene.mat_tex, np.int32))
        s.mat_emit_tex = _ptr(arr(scene.mat_emit_tex, np.int32))
        s.mat_light = _ptr(arr(scene.mat_light, np.int32))
        s.tex_data = _ptr(arr(scene.tex_data, np.float32))
        s.tex_info = _ptr(arr(scene.tex_info, np.int32))
        s.lights = _ptr(arr(scene.lights, np.float32)) if len(scene.lights) else None
        s.points = _ptr(arr(scene.points, np.float64)) if len(scene.points) else None
        s.cache_res = int(scene.cache_res)
        if scene.cache_res:
            s.cache_bmin = _ptr(arr(scene.cache_bmin, np.float32))
            s.cache_bmax = _ptr(arr(scene.cache_bmax, np.float32))
            s.cache_E = _ptr(arr(scene.cache_E.view(np.uint16), np.uint16))
        self._s = s
        self._h = lib.or_build(C.byref(s))
        self._lib = lib

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                self._lib.or_free(self._h)
                self._h = None
        except Exception:
            pass

    def trace(self, render, pixels=None, n_threads=None, with_flags=False, grf=None):
        """U[lambda][m][pixel] (complex128) for the listed pixel linear indices (all by default).
        with_flags: also the per-pixel flag counts and delta-chain sensitivity bound
        [lambda][pixel] (see or_trace), returned as (U, flags, sens).  grf: the phase maps of
        phase_mode 2 (``waveoptics.grf_maps``)."""
        if pixels is None:
            pixels = np.arange(render.W * render.H, dtype=np.int64)
        pixels = np.ascontiguousarray(pixels, np.int64)
        n = len(pixels)
        nl = len(render.lambdas)
        out = np.zeros((nl, render.K, n, 2), np.float64)
        flags = np.zeros((nl, n), np.int64)
        sens = np.zeros((nl, n), np.float64)
        grf = None if grf is None else np.ascontiguousarray(grf, np.float64)
        rs = _render_struct(render, grf)
        nt = n_threads or os.cpu_count() or 1
        rc = self._lib.or_trace(self._h, C.byref(rs), pixels.ctypes.data, n, out.ctypes.data,
                                flags.ctypes.data if with_flags else None,
                                sens.ctypes.data if with_flags else None, int(nt))
        if rc != 0:
            raise ValueError(f"or_trace failed: {rc}")
        U = out[..., 0] + 1j * out[..., 1]
        return (U, flags, sens) if with_flags else U

    def bake(self, res, bmin, bmax, spp, max_depth, seed=1, cells=None, n_threads=None, with_sens=False):
        """Ambient cache E [n_cells][3] (float64) at the listed cell indices (all by default);
        with_sens: (E, sens), sens [n_cells][3] the float32-sensitivity bound of or_bake_sens."""
        if cells is None:
            cells = np.arange(res ** 3, dtype=np.int64)
        cells = np.ascontiguousarray(cells, np.int64)
        d = OrBake()
        d.res, d.spp, d.max_depth, d.seed = int(res), int(spp), int(max_depth), int(seed)
        for k in range(3):
            d.bmin[k], d.bmax[k] = float(bmin[k]), float(bmax[k])
        E = np.zeros((len(cells), 3), np.float64)
        sens = np.zeros((len(cells), 3), np.float64) if with_sens else None
        rc = self._lib.or_bake_sens(self._h, C.byref(d), cells.ctypes.data, len(cells), E.ctypes.data,
                                    sens.ctypes.data if with_sens else None, int(n_threads or os.cpu_count() or 1))
        if rc != 0:
            raise ValueError(f"or_bake failed: {rc}")
        return (E, sens) if with_sens else E

    def trace_full(self, render, n_threads=None, grf=None):
        U = self.trace(render, None, n_threads, grf=grf)
        return U.reshape(len(render.lambdas), render.K, render.H, render.W)

    def sample(self, render, lam, pixel, s, grf=None):
        rec = np.zeros(len(REC_FIELDS), np.float64)
        grf = None if grf is None else np.ascontiguousarray(grf, np.float64)
        rs = _render_struct(render, grf)
        ok = self._lib.or_sample(self._h, C.byref(rs), int(lam), int(pixel), int(s), rec.ctypes.data)
        d = dict(zip(REC_FIELDS, rec.tolist()))
        d["ok"] = bool(ok)
        return d

    def tex_lookup(self, tex, u, v, ch):
        """The scene's bilinear texture lookup at (u, v), channel ch."""
        return self._lib.or_tex_lookup(self._h, int(tex), float(u), float(v), int(ch))

    def cache_lookup(self, p, ch):
        """The scene's trilinear ambient-cache lookup at world point p, channel ch."""
        p = np.ascontiguousarray(p, np.float64)
        return self._lib.or_cache_lookup(self._h, p.ctypes.data, int(ch))

    def closest_hit(self, o, d, tmin=0.0, tmax=np.inf, brute=False):
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        t = C.c_double()
        tri = C.c_int32()
        self._lib.or_closest_hit(self._h, o.ctypes.data, d.ctypes.data, float(tmin), float(tmax),
                                 int(brute), C.byref(t), C.byref(tri))
        return t.value, tri.value


def philox4x32_10(ctr, key):
    lib = _load()
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    o = np.zeros(4, np.uint32)
    lib.or_philox4x32_10(c.ctypes.data, k.ctypes.data, o.ctypes.data)
    return o


def cone_dir(lam, pitch, u0, u1):
    lib = _load()
    d = np.zeros(3, np.float64)
    pdf = C.c_double()
    lib.or_cone_dir(float(lam), float(pitch), float(u0), float(u1), d.ctypes.data, C.byref(pdf))
    return d, pdf.value


def fresnel_dielectric(cos_i, n_i, n_t):
    return _load().or_fresnel_dielectric(float(cos_i), float(n_i), float(n_t))


def ggx_eval(alpha, F0, wo, wi):
    lib = _load()
    wo = np.ascontiguousarray(wo, np.float64)
    wi = np.ascontiguousarray(wi, np.float64)
    f, pdf = C.c_double(), C.c_double()
    lib.or_ggx_eval(float(alpha), float(F0), wo.ctypes.data, wi.ctypes.data, C.byref(f), C.byref(pdf))
    return f.value, pdf.value


def ggx_sample(alpha, F0, wo, u0, u1):
    lib = _load()
    wo = np.ascontiguousarray(wo, np.float64)
    wi = np.zeros(3, np.float64)
    w, pdf = C.c_double(), C.c_double()
    ok = lib.or_ggx_sample(float(alpha), float(F0), wo.ctypes.data, float(u0), float(u1), wi.ctypes.data,
                           C.byref(w), C.byref(pdf))
    return bool(ok), wi, w.value, pdf.value


def frame(n):
    lib = _load()
    n = np.ascontiguousarray(n, np.float64)
    t = np.zeros(3)
    b = np.zeros(3)
    lib.or_frame(n.ctypes.data, t.ctypes.data, b.ctypes.data)
    return t, b


def half_to_double(h):
    return _load().or_half_to_double(int(h))


def grf_phases(seed, m, nx, ny):
    """Random spectral phases xi_m of GRF map m, [ny][nx] in FFT order (Eq. 4)."""
    xi = np.zeros((ny, nx), np.float64)
    _load().or_grf_phases(int(seed), int(m), int(nx), int(ny), xi.ctypes.data)
    return xi
