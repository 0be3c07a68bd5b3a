"""Python binding of the C-ABI in include/hpt.h (argument marshalling only).

Every step of the wave path tracer runs in the CUDA library ``_lib/libhpt.so``;
this module only packs numpy arrays and torch device buffers into the C structs.
It raises if the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# HPT_LIB selects another build of the library (the checked build in its tests)
LIB_PATH = os.environ.get("HPT_LIB") or os.path.join(_PKG, "_lib", "libhpt.so")

HPT_OK = 0
STATUS_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "TIMEOUT", -5: "BUSY",
                -6: "NOT_FOUND", -7: "UNSUPPORTED", -8: "DEVICE", -9: "CANCELLED"}
CTX_NO_GRAPHS, CTX_FAIL_SERVING_WAVES = 1, 2
PREC_FP64, PREC_DF32 = 0, 1
NCOUNTERS = 8
COUNTER_NAMES = ["samples", "rays", "box_tests", "tri_tests", "refines", "fp64_fallbacks", "shadow_rays", "bounces"]

# exported symbols, as declared in include/hpt.h
SYMBOLS = ["hpt_create", "hpt_destroy", "hpt_last_error", "hpt_scene_upload", "hpt_scene_release", "hpt_scene_info",
           "hpt_trace", "hpt_trace_host", "hpt_sync", "hpt_trace_counters", "hpt_submit", "hpt_poll", "hpt_wait",
           "hpt_request_times", "hpt_trace_fixed_scratch", "hpt_autotune", "hpt_trace_timed", "hpt_grf_build",
           "hpt_asm_propagate", "hpt_cache_bake", "hpt_scene_set_cache", "hpt_phase_encode",
           "hpt_probe_peaks", "hpt_cache_upload", "hpt_cancel", "hpt_request_output", "hpt_request_release"]


# kernel kinds of hpt_trace_timed, in the order of HPT_K_GEN .. HPT_K_ACCUM
KERNEL_NAMES = ["k_gen", "k_trace", "k_shade", "k_accum"]


class HptError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class CtxDesc(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_uint64), ("max_inflight", C.c_int32), ("flags", C.c_int32),
                ("max_queue", C.c_int32), ("reserved", C.c_int32)]


class Material(C.Structure):
    _fields_ = [("kind", C.c_int32), ("albedo", C.c_float * 3), ("roughness", C.c_float), ("ior", C.c_float),
                ("Le", C.c_float * 3), ("tex", C.c_int32), ("emit_tex", C.c_int32), ("light", C.c_int32)]


class SceneDesc(C.Structure):
    _fields_ = [("nv", C.c_int32), ("nt", C.c_int32), ("nm", C.c_int32), ("ntex", C.c_int32), ("nl", C.c_int32),
                ("np", C.c_int32), ("verts", C.c_void_p), ("normals", C.c_void_p), ("uvs", C.c_void_p),
                ("tris", C.c_void_p), ("tri_mat", C.c_void_p), ("materials", C.c_void_p), ("tex_data", C.c_void_p),
                ("tex_floats", C.c_int64), ("tex_info", C.c_void_p), ("lights", C.c_void_p), ("points", C.c_void_p),
                ("cache_res", C.c_int32), ("cache_bmin", C.c_float * 3), ("cache_bmax", C.c_float * 3),
                ("cache_E", C.c_void_p)]


class RenderDesc(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("pitch", C.c_double), ("n_lambda", C.c_int32),
                ("lam", C.c_double * 3), ("channel", C.c_int32 * 3), ("spp", C.c_int32), ("max_depth", C.c_int32),
                ("K", C.c_int32), ("hologram_offset", C.c_int32), ("seed", C.c_uint64), ("phase_seed", C.c_uint64),
                ("phase_mode", C.c_int32), ("facet_size", C.c_double), ("T", C.c_double * 16),
                ("precision", C.c_int32), ("use_cache", C.c_int32), ("grf_phi", C.c_void_p),
                ("grf_nx", C.c_int32), ("grf_ny", C.c_int32), ("omit_obliquity", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("paths_per_wave", C.c_int32), ("lanes", C.c_int32), ("trace_blocks_per_sm", C.c_int32),
                ("shade_blocks_per_sm", C.c_int32), ("scene_class", C.c_int32), ("candidates", C.c_int32),
                ("band_ms", C.c_double), ("band_ms_start", C.c_double), ("band_path_samples", C.c_int64)]


class BakeDesc(C.Structure):
    _fields_ = [("res", C.c_int32), ("bmin", C.c_float * 3), ("bmax", C.c_float * 3), ("spp", C.c_int32),
                ("max_depth", C.c_int32), ("seed", C.c_uint64)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libhpt.so (no fallback: a missing library is an error)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = C.CDLL(path)
    vp, st = C.c_void_p, C.c_int
    lib.hpt_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(CtxDesc)]
    lib.hpt_destroy.argtypes = [vp]
    lib.hpt_destroy.restype = None
    lib.hpt_last_error.restype = C.c_char_p
    lib.hpt_scene_upload.argtypes = [vp, C.POINTER(SceneDesc), C.POINTER(C.c_uint64)]
    lib.hpt_scene_release.argtypes = [vp, C.c_uint64]
    lib.hpt_scene_info.argtypes = [vp, C.c_uint64, C.POINTER(C.c_uint64), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.hpt_trace.argtypes = [vp, C.c_uint64, C.POINTER(RenderDesc), vp, C.c_size_t, vp]
    lib.hpt_trace_host.argtypes = [vp, C.c_uint64, C.POINTER(RenderDesc), vp, C.c_size_t, vp]
    lib.hpt_sync.argtypes = [vp]
    lib.hpt_trace_counters.argtypes = [vp, C.c_uint64, C.POINTER(RenderDesc), vp, C.c_size_t, C.POINTER(C.c_uint64)]
    lib.hpt_probe_peaks.argtypes = [vp, C.POINTER(C.c_double)]
    lib.hpt_cache_upload.argtypes = [vp, C.c_uint64, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_float), vp]
    lib.hpt_phase_encode.argtypes = [vp, vp, vp, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_int32,
                                     C.c_float, C.POINTER(C.c_double), vp]
    lib.hpt_cache_bake.argtypes = [vp, C.c_uint64, C.POINTER(BakeDesc), vp, C.c_size_t, vp]
    lib.hpt_scene_set_cache.argtypes = [vp, C.c_uint64, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_float), vp]
    lib.hpt_grf_build.argtypes = [vp, C.c_uint64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_double, vp, vp]
    lib.hpt_asm_propagate.argtypes = [vp, vp, vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                      C.c_double, C.c_double, vp]
    lib.hpt_trace_timed.argtypes = [vp, C.c_uint64, C.POINTER(RenderDesc), vp, C.c_size_t, C.POINTER(C.c_float),
                                    C.POINTER(C.c_uint32)]
    lib.hpt_submit.argtypes = [vp, C.c_uint64, C.POINTER(RenderDesc), vp, C.c_size_t, C.POINTER(C.c_uint64)]
    lib.hpt_poll.argtypes = [vp, C.c_uint64, C.POINTER(C.c_int)]
    lib.hpt_wait.argtypes = [vp, C.c_uint64, C.c_uint32]
    lib.hpt_request_times.argtypes = [vp, C.c_uint64, C.POINTER(C.c_double)]
    lib.hpt_cancel.argtypes = [vp, C.c_uint64]
    lib.hpt_request_output.argtypes = [vp, C.c_uint64, vp, C.c_size_t]
    lib.hpt_request_release.argtypes = [vp, C.c_uint64]
    lib.hpt_trace_fixed_scratch.argtypes = [vp, C.c_uint64, C.POINTER(RenderDesc), vp, C.c_size_t, vp]
    lib.hpt_autotune.argtypes = [vp, C.c_uint64, C.POINTER(RenderDesc), C.POINTER(Tuning)]
    for name in SYMBOLS:
        f = getattr(lib, name)
        if name not in ("hpt_destroy", "hpt_last_error"):
            f.restype = st
    _lib = lib
    return lib


def _check(status):
    if status != HPT_OK:
        raise HptError(status, load_library().hpt_last_error().decode())


def render_desc(r, precision=PREC_DF32) -> RenderDesc:
    d = RenderDesc()
    d.W, d.H, d.pitch = int(r.W), int(r.H), float(r.pitch)
    d.n_lambda = len(r.lambdas)
    for i, (l, c) in enumerate(zip(r.lambdas, r.channels)):
        d.lam[i] = float(l)
        d.channel[i] = int(c)
    d.spp, d.max_depth, d.K, d.hologram_offset = int(r.spp), int(r.max_depth), int(r.K), int(r.hologram_offset)
    d.seed, d.phase_seed, d.phase_mode = int(r.seed), int(r.phase_seed), int(r.phase_mode)
    d.facet_size = float(r.facet_size)
    T = np.asarray(r.T, np.float64).reshape(16)
    for i in range(16):
        d.T[i] = float(T[i])
    d.precision = int(precision)
    d.use_cache = int(r.use_cache)
    d.omit_obliquity = int(getattr(r, "omit_obliquity", 0))
    g = getattr(r, "grf", None)
    if g is not None:
        if not (g.is_cuda and g.dtype.is_floating_point and g.element_size() == 4 and g.is_contiguous()
                and g.dim() == 3 and g.shape[0] >= r.K):
            raise ValueError("grf must be a contiguous float32 CUDA tensor [>= K][ny][nx]")
        d.grf_phi = g.data_ptr()
        d.grf_ny, d.grf_nx = int(g.shape[1]), int(g.shape[2])
    return d


def out_bytes(r) -> int:
    return 8 * len(r.lambdas) * int(r.K) * int(r.W) * int(r.H)


class Context:
    """One library context on one CUDA device (owns scenes and launch slots)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_inflight: int = 0, graphs: bool = True,
                 max_queue: int = 0, flags: int = 0):
        self.lib = load_library()
        self.h = C.c_void_p()
        desc = CtxDesc(hbm_budget_bytes, max_inflight, (0 if graphs else CTX_NO_GRAPHS) | int(flags), max_queue, 0)
        _check(self.lib.hpt_create(C.byref(self.h), int(device), C.byref(desc)))
        self.device = device

    def close(self):
        if self.h:
            self.lib.hpt_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- scenes
    def upload_scene(self, s) -> int:
        keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            keep.append(a)
            return a.ctypes.data

        nm = len(s.mat_type)
        mats = (Material * nm)()
        for i in range(nm):
            m = mats[i]
            m.kind = int(s.mat_type[i])
            for c in range(3):
                m.albedo[c] = float(s.mat_albedo[i, c])
                m.Le[c] = float(s.mat_Le[i, c])
            m.roughness = float(s.mat_rough[i])
            m.ior = float(s.mat_ior[i])
            m.tex = int(s.mat_tex[i])
            m.emit_tex = int(s.mat_emit_tex[i])
            m.light = int(s.mat_light[i])
        d = SceneDesc()
        d.nv, d.nt, d.nm = len(s.verts), len(s.tris), nm
        d.ntex, d.nl, d.np = len(s.tex_info), len(s.lights), len(s.points)
        d.verts = arr(s.verts, np.float32)
        d.normals = arr(s.normals, np.float32)
        d.uvs = arr(s.uvs, np.float32)
        d.tris = arr(s.tris, np.uint32)
        d.tri_mat = arr(s.tri_mat, np.uint32)
        d.materials = C.cast(mats, C.c_void_p)
        d.tex_data = arr(s.tex_data, np.float32)
        d.tex_floats = int(np.asarray(s.tex_data).size)
        d.tex_info = arr(s.tex_info, np.int32)
        d.lights = arr(s.lights, np.float32) if len(s.lights) else None
        d.points = arr(s.points, np.float64) if len(s.points) else None
        d.cache_res = int(s.cache_res)
        if s.cache_res:
            for c in range(3):
                d.cache_bmin[c] = float(s.cache_bmin[c])
                d.cache_bmax[c] = float(s.cache_bmax[c])
            d.cache_E = arr(np.asarray(s.cache_E).view(np.uint16), np.uint16)
        sid = C.c_uint64()
        _check(self.lib.hpt_scene_upload(self.h, C.byref(d), C.byref(sid)))
        return sid.value

    def release_scene(self, sid: int):
        _check(self.lib.hpt_scene_release(self.h, C.c_uint64(sid)))

    def scene_info(self, sid: int):
        b, n, dep = C.c_uint64(), C.c_int32(), C.c_int32()
        _check(self.lib.hpt_scene_info(self.h, C.c_uint64(sid), C.byref(b), C.byref(n), C.byref(dep)))
        return {"device_bytes": b.value, "nodes": n.value, "depth": dep.value}

    # ----------------------------------------------------------------- traces
    def trace(self, sid: int, r, out, precision=PREC_DF32, stream=None):
        """Asynchronous trace into a caller-owned device buffer (a torch complex64 CUDA tensor
        of shape (n_lambda, K, H, W), or a raw device pointer with out_nbytes given by out_bytes(r))."""
        ptr, nbytes = _dev_buffer(out, r)
        d = render_desc(r, precision)
        _check(self.lib.hpt_trace(self.h, C.c_uint64(sid), C.byref(d), C.c_void_p(ptr), nbytes, _stream_ptr(stream)))

    def trace_host(self, sid: int, r, out_host: np.ndarray, precision=PREC_DF32, stream=None):
        """End-to-end trace into host memory (numpy complex64 array, pinned or pageable)."""
        assert out_host.dtype == np.complex64 and out_host.flags.c_contiguous
        d = render_desc(r, precision)
        _check(self.lib.hpt_trace_host(self.h, C.c_uint64(sid), C.byref(d), C.c_void_p(out_host.ctypes.data),
                                       out_host.nbytes, _stream_ptr(stream)))

    def trace_fixed_scratch(self, sid: int, r, out, precision=PREC_DF32, stream=None):
        """hpt_trace_fixed_scratch: the same trace, with all scratch in the library's fixed
        64 MiB device array; the call allocates no device memory."""
        ptr, nbytes = _dev_buffer(out, r)
        d = render_desc(r, precision)
        _check(self.lib.hpt_trace_fixed_scratch(self.h, C.c_uint64(sid), C.byref(d), C.c_void_p(ptr), nbytes,
                                                _stream_ptr(stream)))

    def trace_counters(self, sid: int, r, out, precision=PREC_DF32):
        ptr, nbytes = _dev_buffer(out, r)
        d = render_desc(r, precision)
        c = (C.c_uint64 * NCOUNTERS)()
        _check(self.lib.hpt_trace_counters(self.h, C.c_uint64(sid), C.byref(d), C.c_void_p(ptr), nbytes, c))
        return dict(zip(COUNTER_NAMES, [int(x) for x in c]))

    def trace_timed(self, sid: int, r, out, precision=PREC_DF32):
        """One frame with CUDA events around every launch: {kernel: (device ms, launches)}."""
        ptr, nbytes = _dev_buffer(out, r)
        d = render_desc(r, precision)
        ms = (C.c_float * len(KERNEL_NAMES))()
        n = (C.c_uint32 * len(KERNEL_NAMES))()
        _check(self.lib.hpt_trace_timed(self.h, C.c_uint64(sid), C.byref(d), C.c_void_p(ptr), nbytes, ms, n))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_NAMES)}

    def probe_peaks(self):
        """Measured FP32 / FP64 FMA TFLOP/s, L2 read GB/s and the SM count of this device."""
        p = (C.c_double * 4)()
        _check(self.lib.hpt_probe_peaks(self.h, p))
        return {"fp32_tflops": p[0], "fp64_tflops": p[1], "l2_read_gbs": p[2], "sms": int(p[3])}

    def phase_encode(self, target, phi, lam: float, pitch: float, z: float, iters: int, lr: float, stream=None):
        """Gradient steps on phi (float32 CUDA tensor [H][W], updated in place) towards the complex
        target (complex64 CUDA tensor [H][W]); returns the loss before each step."""
        if not (target.is_cuda and target.dtype.is_complex and target.element_size() == 8 and target.is_contiguous()
                and target.dim() == 2):
            raise ValueError("target must be a contiguous complex64 CUDA tensor [H][W]")
        if not (phi.is_cuda and phi.dtype.is_floating_point and phi.element_size() == 4 and phi.is_contiguous()
                and tuple(phi.shape) == tuple(target.shape)):
            raise ValueError("phi must be a contiguous float32 CUDA tensor of the target's shape")
        H, W = (int(x) for x in target.shape)
        losses = (C.c_double * max(int(iters), 1))()
        _check(self.lib.hpt_phase_encode(self.h, C.c_void_p(target.data_ptr()), C.c_void_p(phi.data_ptr()), W, H,
                                         float(lam), float(pitch), float(z), int(iters), float(lr), losses,
                                         _stream_ptr(stream)))
        return np.array(losses[:int(iters)])

    def cache_bake(self, sid: int, res: int, bmin, bmax, spp: int, max_depth: int, seed: int = 1, stream=None):
        """Ambient cache E [res][res][res][3] (float32 CUDA tensor, [z][y][x][c]) of the scene."""
        import torch
        E = torch.empty((res, res, res, 3), dtype=torch.float32, device=f"cuda:{self.device}")
        d = BakeDesc()
        d.res, d.spp, d.max_depth, d.seed = int(res), int(spp), int(max_depth), int(seed)
        for k in range(3):
            d.bmin[k], d.bmax[k] = float(bmin[k]), float(bmax[k])
        _check(self.lib.hpt_cache_bake(self.h, C.c_uint64(sid), C.byref(d), C.c_void_p(E.data_ptr()),
                                       E.numel() * 4, _stream_ptr(stream)))
        return E

    def cache_upload(self, sid: int, E_half, bmin, bmax):
        """Upload a host binary16 cache [res][res][res][3] (numpy float16) to the scene."""
        E_half = np.ascontiguousarray(E_half, np.float16)
        if not (E_half.ndim == 4 and E_half.shape[0] == E_half.shape[1] == E_half.shape[2] and E_half.shape[3] == 3):
            raise ValueError("E_half must be [res][res][res][3]")
        lo = (C.c_float * 3)(*[float(x) for x in bmin])
        hi = (C.c_float * 3)(*[float(x) for x in bmax])
        _check(self.lib.hpt_cache_upload(self.h, C.c_uint64(sid), int(E_half.shape[0]), lo, hi,
                                         C.c_void_p(E_half.ctypes.data)))

    def set_cache(self, sid: int, E, bmin, bmax):
        """Replace the scene's ambient cache by the float32 CUDA tensor E [res][res][res][3] (None: remove)."""
        lo = (C.c_float * 3)(*[float(x) for x in bmin])
        hi = (C.c_float * 3)(*[float(x) for x in bmax])
        if E is None:
            _check(self.lib.hpt_scene_set_cache(self.h, C.c_uint64(sid), 0, lo, hi, None))
            return
        if not (E.is_cuda and E.dtype.is_floating_point and E.element_size() == 4 and E.is_contiguous()
                and E.dim() == 4 and E.shape[0] == E.shape[1] == E.shape[2] and E.shape[3] == 3):
            raise ValueError("E must be a contiguous float32 CUDA tensor [res][res][res][3]")
        _check(self.lib.hpt_scene_set_cache(self.h, C.c_uint64(sid), int(E.shape[0]), lo, hi, C.c_void_p(E.data_ptr())))

    def grf_build(self, phase_seed: int, K: int, nx: int, ny: int, pitch: float, hologram_offset: int = 0,
                  stream=None):
        """Eq. 4 phase maps [K][ny][nx] (float32 radians) as a new CUDA tensor."""
        import torch
        phi = torch.empty((K, ny, nx), dtype=torch.float32, device=f"cuda:{self.device}")
        _check(self.lib.hpt_grf_build(self.h, C.c_uint64(phase_seed), int(hologram_offset), int(K), int(nx), int(ny),
                                      float(pitch), C.c_void_p(phi.data_ptr()), _stream_ptr(stream)))
        return phi

    def asm_propagate(self, U, lambdas, pitch: float, z: float, out=None, stream=None):
        """Angular-spectrum propagation by z of fields U [n_lambda][K][H][W] (complex64, CUDA)."""
        if not (U.is_cuda and U.dtype.is_complex and U.element_size() == 8 and U.is_contiguous() and U.dim() == 4):
            raise ValueError("U must be a contiguous complex64 CUDA tensor [n_lambda][K][H][W]")
        nl, K, H, W = (int(x) for x in U.shape)
        if len(lambdas) != nl:
            raise ValueError("one wavelength per field group")
        if out is None:
            out = U.new_empty(U.shape)
        lam = (C.c_double * nl)(*[float(x) for x in lambdas])
        _check(self.lib.hpt_asm_propagate(self.h, C.c_void_p(U.data_ptr()), C.c_void_p(out.data_ptr()), W, H, nl, K,
                                          lam, float(pitch), float(z), _stream_ptr(stream)))
        return out

    def autotune(self, sid: int, r, precision=PREC_DF32) -> dict:
        """Pick the trace launch shape (wave size, lanes, grid sizes) by timing a band of this
        render; returns the choice (kept for the scene's size class)."""
        d = render_desc(r, precision)
        t = Tuning()
        _check(self.lib.hpt_autotune(self.h, C.c_uint64(sid), C.byref(d), C.byref(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def sync(self):
        _check(self.lib.hpt_sync(self.h))

    # ---------------------------------------------------------------- serving
    def submit(self, sid: int, r, out, precision=PREC_DF32) -> int:
        ptr, nbytes = _dev_buffer(out, r) if out is not None else (0, 0)
        d = render_desc(r, precision)
        rid = C.c_uint64()
        _check(self.lib.hpt_submit(self.h, C.c_uint64(sid), C.byref(d), C.c_void_p(ptr), nbytes, C.byref(rid)))
        return rid.value

    def poll(self, rid: int) -> bool:
        done = C.c_int()
        _check(self.lib.hpt_poll(self.h, C.c_uint64(rid), C.byref(done)))
        return bool(done.value)

    def wait(self, rid: int, timeout_ms: int = 0):
        _check(self.lib.hpt_wait(self.h, C.c_uint64(rid), int(timeout_ms)))

    def request_times(self, rid: int):
        t = (C.c_double * 3)()
        _check(self.lib.hpt_request_times(self.h, C.c_uint64(rid), t))
        return tuple(t)

    def cancel(self, rid: int):
        _check(self.lib.hpt_cancel(self.h, C.c_uint64(rid)))

    def request_output(self, rid: int, dst):
        """Copy a finished request's library-owned output into dst (a numpy complex64 array or a
        contiguous torch tensor, host or device, of at least the output's size)."""
        if isinstance(dst, np.ndarray):
            assert dst.flags.c_contiguous
            ptr, n = dst.ctypes.data, dst.nbytes
        else:
            assert dst.is_contiguous()
            ptr, n = dst.data_ptr(), dst.numel() * dst.element_size()
        _check(self.lib.hpt_request_output(self.h, C.c_uint64(rid), C.c_void_p(ptr), n))

    def request_release(self, rid: int):
        _check(self.lib.hpt_request_release(self.h, C.c_uint64(rid)))


def _dev_buffer(out, r):
    need = out_bytes(r)
    if isinstance(out, int):
        return out, need
    import torch  # device memory only
    if not isinstance(out, torch.Tensor) or not out.is_cuda or not out.is_contiguous():
        raise TypeError("out must be a contiguous CUDA tensor or a device pointer")
    nbytes = out.numel() * out.element_size()
    if nbytes < need:
        raise ValueError(f"output buffer has {nbytes} bytes, need {need}")
    return out.data_ptr(), nbytes


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def alloc_output(r, device="cuda"):
    import torch
    return torch.empty((len(r.lambdas), int(r.K), int(r.H), int(r.W)), dtype=torch.complex64, device=device)
