"""Seeded synthetic inputs for the wave path tracer.

This module only *makes inputs*: triangle meshes, materials, textures, lights,
an ambient-cache blob and render descriptors.  It contains none of the
estimator's arithmetic, and both the FP64 oracle (``oracle/``) and the CUDA
library read exactly the arrays it returns.

The paper renders Mitsuba scenes edited in Blender (Sec. 5.1); those scenes are
not available, so the workloads below stand in for them:

* ``config0``  - two emissive textured quads (4 triangles), 256x256 SLM, 8 um
  pitch, 520 nm, direct lighting only, K = 1.
* ``config1``  - 30 icospheres (~24k triangles) on a textured ground plane with
  one rectangular area light; Lambertian / GGX / mirror / dielectric spheres
  in equal shares; 1920x1080 SLM, 6.4 um pitch, RGB, depth 4, 64 spp.
* ``config2``  - the config-1 scene and SLM with K = 8 holograms.
* ``config3``  - ~200k triangles (500 icospheres + 20 subdivided slabs), a
  128^3 FP16 ambient-radiance cache, 3840x2160 SLM at 3.74 um, 256 spp, K = 8.

Units are SI metres.  Every vertex coordinate is a float32 value, so a float32
kernel and a float64 oracle see bit-identical triangles.  The SLM sits in the
z = 0 plane, pixels face +z, and hologram space equals world space unless a
transform is given.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Material kinds (the C-ABI and the oracle use the same numbering).
LAMBERT, GGX, MIRROR, DIELECTRIC, EMITTER = 0, 1, 2, 3, 4
MATERIAL_NAMES = {LAMBERT: "lambert", GGX: "ggx", MIRROR: "mirror",
                  DIELECTRIC: "dielectric", EMITTER: "emitter"}

PHASE_HASH, PHASE_ZERO, PHASE_GRF = 0, 1, 2
MM = 1e-3
UM = 1e-6
NM = 1e-9


# ---------------------------------------------------------------------------
# scene container
# ---------------------------------------------------------------------------
@dataclass
class Scene:
    verts: np.ndarray            # float32 [nv,3]  metres
    normals: np.ndarray          # float32 [nv,3]  per-vertex shading normals
    uvs: np.ndarray              # float32 [nv,2]
    tris: np.ndarray             # uint32  [nt,3]
    tri_mat: np.ndarray          # uint32  [nt]
    mat_type: np.ndarray         # int32   [nm]
    mat_albedo: np.ndarray       # float32 [nm,3]  (mirror reflectance, GGX F0)
    mat_rough: np.ndarray        # float32 [nm]    GGX roughness (alpha = r^2)
    mat_ior: np.ndarray          # float32 [nm]
    mat_Le: np.ndarray           # float32 [nm,3]  emitted radiance
    mat_tex: np.ndarray          # int32   [nm]    albedo texture id or -1
    mat_emit_tex: np.ndarray     # int32   [nm]    1: Le is scaled by the texture
    mat_light: np.ndarray        # int32   [nm]    rect light id for EMITTER, else -1
    tex_data: np.ndarray         # float32 [sum(w*h*3)]  row-major RGB texels
    tex_info: np.ndarray         # int32   [ntex,3] (offset in floats, w, h)
    lights: np.ndarray           # float32 [nl,12] corner, edge_u, edge_v, Le
    points: np.ndarray           # float64 [np,4]  position, amplitude
    cache_bmin: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))
    cache_bmax: np.ndarray = field(default_factory=lambda: np.ones(3, np.float32))
    cache_res: int = 0
    cache_E: np.ndarray | None = None   # float16 [res,res,res,3] (z, y, x, c)
    name: str = ""

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    def validate(self) -> None:
        nv, nt, nm = len(self.verts), len(self.tris), len(self.mat_type)
        assert self.verts.dtype == np.float32 and self.verts.shape == (nv, 3)
        assert self.normals.dtype == np.float32 and self.normals.shape == (nv, 3)
        assert self.uvs.dtype == np.float32 and self.uvs.shape == (nv, 2)
        assert self.tris.dtype == np.uint32 and self.tris.shape == (nt, 3)
        assert int(self.tris.max(initial=0)) < nv
        assert self.tri_mat.dtype == np.uint32 and int(self.tri_mat.max(initial=0)) < nm
        for a in (self.mat_albedo, self.mat_Le):
            assert a.dtype == np.float32 and a.shape == (nm, 3)
        assert self.lights.dtype == np.float32 and self.lights.ndim == 2 and self.lights.shape[1] == 12
        assert self.points.dtype == np.float64 and self.points.shape[1] == 4
        if self.cache_res:
            assert self.cache_E is not None and self.cache_E.dtype == np.float16
            assert self.cache_E.shape == (self.cache_res,) * 3 + (3,)


@dataclass
class Render:
    W: int
    H: int
    pitch: float                       # metres
    lambdas: tuple                     # metres, 1..3 entries
    channels: tuple                    # RGB channel read by each wavelength
    spp: int
    max_depth: int
    K: int = 1
    hologram_offset: int = 0
    seed: int = 1
    phase_seed: int = 2
    phase_mode: int = PHASE_HASH
    facet_size: float = 16 * UM        # edge of the cubic facet cells of the hash phase
    T: np.ndarray = field(default_factory=lambda: np.eye(4))  # world -> hologram
    use_cache: int = 0
    grf: object = None                 # phase mode 2: device phase maps [K][ny][nx] (float32 radians)
    omit_obliquity: int = 0            # 1: leave out the cos(theta) factor of Eq. 2

    @property
    def n_lambda(self) -> int:
        return len(self.lambdas)

    def path_samples(self) -> int:
        return self.W * self.H * self.n_lambda * self.spp

    def out_shape(self) -> tuple:
        return (self.n_lambda, self.K, self.H, self.W)


# ---------------------------------------------------------------------------
# geometry helpers
# ---------------------------------------------------------------------------
def icosphere(level: int):
    """Unit icosphere: 20 * 4**level triangles, outward winding."""
    g = (1.0 + math.sqrt(5.0)) / 2.0
    base = []
    for a in (-1.0, 1.0):
        for b in (-g, g):
            base += [(a, b, 0.0), (0.0, a, b), (b, 0.0, a)]
    v = np.array(base, np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    # faces = triples of mutually nearest neighbours (edge length of the icosahedron)
    d = np.linalg.norm(v[:, None] - v[None], axis=2)
    e = d[d > 1e-9].min()
    adj = np.abs(d - e) < 1e-6
    faces = []
    for i in range(12):
        for j in range(i + 1, 12):
            if not adj[i, j]:
                continue
            for k in range(j + 1, 12):
                if adj[i, k] and adj[j, k]:
                    f = [i, j, k]
                    n = np.cross(v[j] - v[i], v[k] - v[i])
                    if np.dot(n, v[i] + v[j] + v[k]) < 0:
                        f = [i, k, j]
                    faces.append(f)
    verts = list(map(tuple, v))
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = np.add(verts[a], verts[b])
                m /= np.linalg.norm(m)
                cache[key] = len(verts)
                verts.append(tuple(m))
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        faces = nf
    return np.array(verts, np.float64), np.array(faces, np.uint32)


class _Builder:
    """Accumulates meshes, materials and textures into one Scene."""

    def __init__(self, name):
        self.name = name
        self.V, self.N, self.UV, self.F, self.FM = [], [], [], [], []
        self.nv = 0
        self.mats = []
        self.tex = []
        self.lights = []
        self.points = []

    def material(self, kind, albedo=(0.0, 0.0, 0.0), rough=0.0, ior=1.5,
                 Le=(0.0, 0.0, 0.0), tex=-1, emit_tex=0, light=-1):
        self.mats.append((kind, albedo, rough, ior, Le, tex, emit_tex, light))
        return len(self.mats) - 1

    def texture(self, arr):
        self.tex.append(np.asarray(arr, np.float32))
        return len(self.tex) - 1

    def mesh(self, verts, normals, uvs, faces, mat):
        self.V.append(verts)
        self.N.append(normals)
        self.UV.append(uvs)
        self.F.append(np.asarray(faces, np.int64) + self.nv)
        self.FM.append(np.full(len(faces), mat, np.uint32))
        self.nv += len(verts)

    def quad(self, corner, eu, ev, mat, flip=False):
        """Quad corner, corner+eu, corner+eu+ev, corner+ev; normal = eu x ev (or its opposite)."""
        c, eu, ev = (np.asarray(x, np.float64) for x in (corner, eu, ev))
        v = np.array([c, c + eu, c + eu + ev, c + ev])
        n = np.cross(eu, ev)
        n /= np.linalg.norm(n)
        f = [[0, 1, 2], [0, 2, 3]]
        if flip:
            n = -n
            f = [[0, 2, 1], [0, 3, 2]]
        uv = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float64)
        self.mesh(v, np.tile(n, (4, 1)), uv, f, mat)

    def sphere(self, centre, radius, level, mat):
        v, f = icosphere(level)
        self.mesh(np.asarray(centre) + radius * v, v.copy(), np.zeros((len(v), 2)), f, mat)

    def box(self, lo, hi, n_sub, mat):
        """Axis-aligned box, each face split into an n_sub x n_sub grid (flat normals)."""
        lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
        ext = hi - lo
        for axis in range(3):
            for side in (0, 1):
                u_ax, v_ax = (axis + 1) % 3, (axis + 2) % 3
                if side == 0:
                    u_ax, v_ax = v_ax, u_ax     # keep the winding outward
                nrm = np.zeros(3)
                nrm[axis] = 1.0 if side else -1.0
                base = lo.copy()
                base[axis] = hi[axis] if side else lo[axis]
                g = np.linspace(0.0, 1.0, n_sub + 1)
                verts = []
                for b in g:
                    for a in g:
                        p = base.copy()
                        p[u_ax] = lo[u_ax] + a * ext[u_ax]
                        p[v_ax] = lo[v_ax] + b * ext[v_ax]
                        verts.append(p)
                faces = []
                m = n_sub + 1
                for j in range(n_sub):
                    for i in range(n_sub):
                        a0, a1, a2, a3 = j * m + i, j * m + i + 1, (j + 1) * m + i + 1, (j + 1) * m + i
                        faces += [[a0, a1, a2], [a0, a2, a3]]
                verts = np.array(verts)
                uv = np.zeros((len(verts), 2))
                tri = np.array(faces)
                # orient outward
                e1 = verts[tri[0, 1]] - verts[tri[0, 0]]
                e2 = verts[tri[0, 2]] - verts[tri[0, 0]]
                if np.dot(np.cross(e1, e2), nrm) < 0:
                    tri = tri[:, [0, 2, 1]]
                self.mesh(verts, np.tile(nrm, (len(verts), 1)), uv, tri, mat)

    def rect_light(self, corner, eu, ev, Le):
        """Rectangular one-sided area light; emits toward eu x ev."""
        li = len(self.lights)
        self.lights.append(np.concatenate([corner, eu, ev, Le]).astype(np.float32))
        # the light's geometry is built from the float32-rounded record
        rec = self.lights[-1].astype(np.float64)
        m = self.material(EMITTER, Le=tuple(Le), light=li)
        self.quad(rec[0:3], rec[3:6], rec[6:9], m)
        return li

    def build(self) -> Scene:
        V = np.concatenate(self.V).astype(np.float32)
        N = np.concatenate(self.N)
        N = (N / np.linalg.norm(N, axis=1, keepdims=True)).astype(np.float32)
        UV = np.concatenate(self.UV).astype(np.float32)
        F = np.concatenate(self.F).astype(np.uint32)
        FM = np.concatenate(self.FM).astype(np.uint32)
        nm = len(self.mats)
        mt = np.array([m[0] for m in self.mats], np.int32)
        alb = np.array([m[1] for m in self.mats], np.float32).reshape(nm, 3)
        rough = np.array([m[2] for m in self.mats], np.float32)
        ior = np.array([m[3] for m in self.mats], np.float32)
        Le = np.array([m[4] for m in self.mats], np.float32).reshape(nm, 3)
        tex = np.array([m[5] for m in self.mats], np.int32)
        etex = np.array([m[6] for m in self.mats], np.int32)
        light = np.array([m[7] for m in self.mats], np.int32)
        data, info, off = [], [], 0
        for t in self.tex:
            h, w, _ = t.shape
            data.append(t.reshape(-1))
            info.append((off, w, h))
            off += w * h * 3
        tex_data = np.concatenate(data).astype(np.float32) if data else np.zeros(3, np.float32)
        tex_info = np.array(info, np.int32).reshape(-1, 3)
        lights = np.array(self.lights, np.float32).reshape(-1, 12)
        points = np.array(self.points, np.float64).reshape(-1, 4)
        s = Scene(V, N, UV, F, FM, mt, alb, rough, ior, Le, tex, etex, light,
                  tex_data, tex_info, lights, points, name=self.name)
        s.validate()
        return s


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def config0_scene(seed: int = 1000) -> Scene:
    """Two emissive Lambertian quads facing the SLM (-z), each with a 64x64 U[0,1] texture."""
    rng = np.random.default_rng(seed)
    b = _Builder("cfg0-two-quads")
    for (x0, x1, y0, y1, z) in ((-1.0, 0.2, -0.6, 0.6, 5.0), (-1.5, 1.5, -1.5, 1.5, 10.0)):
        t = b.texture(rng.uniform(0.0, 1.0, (64, 64, 3)))
        m = b.material(LAMBERT, albedo=(1.0, 1.0, 1.0), Le=(1.0, 1.0, 1.0), tex=t, emit_tex=1)
        # eu along +x, ev along +y -> eu x ev = +z; flip so the front faces -z
        b.quad(np.array([x0, y0, z]) * MM, np.array([x1 - x0, 0, 0]) * MM,
               np.array([0, y1 - y0, 0]) * MM, m, flip=True)
    return b.build()


def config0_render(**kw) -> Render:
    base = dict(W=256, H=256, pitch=8 * UM, lambdas=(520 * NM,), channels=(1,),
                spp=16, max_depth=1, K=1)
    base.update(kw)
    return Render(**base)


RGB_LAMBDAS = (638 * NM, 520 * NM, 450 * NM)


def _place_spheres(rng, n, rmin, rmax, xr, yr, zr, on_ground=None, gap=0.1 * MM, tries=20000):
    out = []
    for _ in range(tries):
        if len(out) == n:
            break
        r = rng.uniform(rmin, rmax)
        x = rng.uniform(*xr)
        z = rng.uniform(*zr)
        y = on_ground + r if on_ground is not None else rng.uniform(*yr)
        c = np.array([x, y, z])
        if all(np.linalg.norm(c - c2) > r + r2 + gap for c2, r2 in out):
            out.append((c, r))
    return out


def config1_scene(seed: int = 1001) -> Scene:
    """30 icospheres on a textured ground plane, one 10x10 mm area light (~24k triangles)."""
    rng = np.random.default_rng(seed)
    b = _Builder("cfg1-30-icospheres")
    ground_y = -3.0 * MM
    gt = b.texture(rng.uniform(0.2, 0.8, (64, 64, 3)))
    gm = b.material(LAMBERT, albedo=(1.0, 1.0, 1.0), tex=gt)
    # eu = +z, ev = +x -> normal +y
    b.quad(np.array([-20 * MM, ground_y, 0.0]), np.array([0, 0, 40 * MM]),
           np.array([40 * MM, 0, 0]), gm)
    b.rect_light(np.array([-5 * MM, 15 * MM, 12.5 * MM]), np.array([10 * MM, 0, 0]),
                 np.array([0, 0, 10 * MM]), np.array([20.0, 20.0, 20.0]))
    spheres = _place_spheres(rng, 30, 0.5 * MM, 2.0 * MM, (-8 * MM, 8 * MM), None,
                             (5 * MM, 30 * MM), on_ground=ground_y + 1e-6)
    kinds = (LAMBERT, GGX, MIRROR, DIELECTRIC)
    for i, (c, r) in enumerate(spheres):
        kind = kinds[i % 4]
        alb = tuple(rng.uniform(0.2, 0.9, 3))
        rough = float(rng.uniform(0.05, 0.5))
        m = b.material(kind, albedo=alb, rough=rough, ior=1.5)
        b.sphere(c, r, 3 if r >= 1.25 * MM else 2, m)
    return b.build()


def config1_render(**kw) -> Render:
    base = dict(W=1920, H=1080, pitch=6.4 * UM, lambdas=RGB_LAMBDAS, channels=(0, 1, 2),
                spp=64, max_depth=4, K=1)
    base.update(kw)
    return Render(**base)


def config2_render(**kw) -> Render:
    base = dict(K=8)
    base.update(kw)
    return config1_render(**base)


def smooth_cache(bmin, bmax, res, rng):
    """Smooth positive irradiance field on a res^3 grid, stored as float16 (z, y, x, c)."""
    g = (np.arange(res) + 0.5) / res
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    E = np.empty((res, res, res, 3), np.float64)
    for c in range(3):
        a = rng.uniform(0.5, 1.5, 3)
        ph = rng.uniform(0, 2 * np.pi, 3)
        E[..., c] = 2.0 + 0.8 * np.sin(2 * np.pi * a[0] * x + ph[0]) * np.cos(2 * np.pi * a[1] * y + ph[1]) \
            + 0.5 * np.sin(2 * np.pi * a[2] * z + ph[2])
    return E.astype(np.float16)


def config3_scene(seed: int = 1003, cache_res: int = 128) -> Scene:
    """500 icospheres + 20 subdivided slabs (~200k triangles) with a 128^3 ambient cache."""
    rng = np.random.default_rng(seed)
    b = _Builder("cfg3-500-icospheres-20-slabs")
    ground_y = -5.0 * MM
    gt = b.texture(rng.uniform(0.2, 0.8, (64, 64, 3)))
    gm = b.material(LAMBERT, albedo=(1.0, 1.0, 1.0), tex=gt)
    b.quad(np.array([-20 * MM, ground_y, 0.0]), np.array([0, 0, 40 * MM]),
           np.array([40 * MM, 0, 0]), gm)
    b.rect_light(np.array([-6 * MM, 15 * MM, 11.5 * MM]), np.array([12 * MM, 0, 0]),
                 np.array([0, 0, 12 * MM]), np.array([20.0, 20.0, 20.0]))
    kinds = (LAMBERT, GGX, MIRROR, DIELECTRIC)
    slabs = []
    for i in range(20):
        size = np.array([rng.uniform(2, 3.5), rng.uniform(1.5, 2.5), rng.uniform(0.4, 0.8)]) * MM
        c = np.array([rng.uniform(-7, 7), rng.uniform(-4, 3), rng.uniform(6, 29)]) * MM
        slabs.append((c - size / 2, c + size / 2))
    spheres = _place_spheres(rng, 500, 0.3 * MM, 0.8 * MM, (-8 * MM, 8 * MM), (-4.5 * MM, 4.5 * MM),
                             (5 * MM, 30 * MM))
    for i, (lo, hi) in enumerate(slabs):
        kind = GGX if i % 2 == 0 else DIELECTRIC
        m = b.material(kind, albedo=tuple(rng.uniform(0.3, 0.9, 3)), rough=float(rng.uniform(0.1, 0.4)))
        b.box(lo, hi, 13, m)
    for i, (c, r) in enumerate(spheres):
        lo_c, hi_c = c - r, c + r
        if any(np.all(hi_c > lo) and np.all(lo_c < hi) for lo, hi in slabs):
            continue  # keep dielectrics from nesting: no sphere overlaps a slab
        m = b.material(kinds[i % 4], albedo=tuple(rng.uniform(0.2, 0.9, 3)),
                       rough=float(rng.uniform(0.05, 0.5)))
        b.sphere(c, r, 2, m)
    s = b.build()
    lo = s.verts.min(0).astype(np.float64) - 0.5 * MM
    hi = s.verts.max(0).astype(np.float64) + 0.5 * MM
    s.cache_bmin = lo.astype(np.float32)
    s.cache_bmax = hi.astype(np.float32)
    s.cache_res = cache_res
    s.cache_E = smooth_cache(lo, hi, cache_res, rng)
    return s


def config3_render(**kw) -> Render:
    base = dict(W=3840, H=2160, pitch=3.74 * UM, lambdas=RGB_LAMBDAS, channels=(0, 1, 2),
                spp=256, max_depth=4, K=8, use_cache=1)
    base.update(kw)
    return Render(**base)


# ---------------------------------------------------------------------------
# config 4: the serving stream
# ---------------------------------------------------------------------------
SCENE_MEDIAN_DEPTH = {"cfg0": 7.5 * MM, "cfg1": 17.5 * MM, "cfg3": 17.5 * MM}
CONFIG4_SLM_SIZES = ((512, 512), (1920, 1080), (3840, 2160))
CONFIG4_SPP = (16, 32, 64, 128, 256)
CONFIG4_K = (1, 4, 8)


def pose_T(dx, dy, dz):
    """Rigid world -> hologram transform of an eye offset (dx, dy) and an axial shift dz."""
    T = np.eye(4)
    T[0, 3], T[1, 3], T[2, 3] = -dx, -dy, -dz
    return T


def config4_requests(n, seed=4242):
    """n render requests of the serving stream: a workload drawn uniformly from configs 0-3 (its
    scene and its own pitch, wavelengths, depth and cache use; configs 1 and 2 share the scene),
    an SLM size drawn from 512x512, 1920x1080 and 3840x2160, spp from {16, ..., 256}, K from
    {1, 4, 8}, an eye offset U[-5, 5] mm in x and y and a focal depth U[5, 30] mm (the axial shift
    that puts the scene's median depth there).  Returns [(scene key, Render)]: the keys are
    "cfg0", "cfg1" and "cfg3".  Arrival times are drawn by the caller."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        cfg = int(rng.integers(0, 4))
        W, H = CONFIG4_SLM_SIZES[int(rng.integers(0, 3))]
        spp = int(rng.choice(CONFIG4_SPP))
        K = int(rng.choice(CONFIG4_K))
        dx, dy = rng.uniform(-5 * MM, 5 * MM, 2)
        df = rng.uniform(5 * MM, 30 * MM)
        key = "cfg0" if cfg == 0 else ("cfg1" if cfg in (1, 2) else "cfg3")
        T = pose_T(dx, dy, SCENE_MEDIAN_DEPTH[key] - df)
        make = {0: config0_render, 1: config1_render, 2: config2_render, 3: config3_render}[cfg]
        out.append((key, make(W=W, H=H, spp=spp, K=K, T=T, seed=100 + k)))
    return out


# ---------------------------------------------------------------------------
# small scenes used by tests
# ---------------------------------------------------------------------------
def emissive_plane_scene(z=5 * MM, half=3 * MM, Le=1.0) -> Scene:
    """One large uniform one-sided emitter parallel to the SLM, facing -z (no texture)."""
    b = _Builder("emissive-plane")
    m = b.material(LAMBERT, albedo=(0.0, 0.0, 0.0), Le=(Le, Le, Le))
    b.quad(np.array([-half, -half, z]), np.array([2 * half, 0, 0]), np.array([0, 2 * half, 0]), m, flip=True)
    return b.build()


def point_emitter_scene(points) -> Scene:
    """No geometry except a far-away dummy triangle; only deterministic point emitters."""
    b = _Builder("point-emitters")
    m = b.material(LAMBERT, albedo=(0.0, 0.0, 0.0))
    b.mesh(np.array([[1.0, 1.0, -1.0], [1.001, 1.0, -1.0], [1.0, 1.001, -1.0]]),
           np.tile([0.0, 0.0, 1.0], (3, 1)), np.zeros((3, 2)), [[0, 1, 2]], m)
    b.points = [tuple(p) for p in points]
    return b.build()


def furnace_scene(albedo=0.5, Le=1.0, half=4 * MM, zmin=-2 * MM, zmax=6 * MM) -> Scene:
    """Closed Lambertian box around the SLM, every wall emitting Le with albedo rho, normals inward."""
    b = _Builder("furnace-box")
    m = b.material(LAMBERT, albedo=(albedo,) * 3, Le=(Le,) * 3)
    lo = np.array([-half, -half, zmin])
    hi = np.array([half, half, zmax])
    b.box(lo, hi, 2, m)
    s = b.build()
    # walls face inward: reverse the winding and the normals
    s.tris = s.tris[:, [0, 2, 1]].copy()
    s.normals = (-s.normals).astype(np.float32)
    s.validate()
    return s


def mirror_pair_scenes(seed=7):
    """(A) textured emitter behind the SLM seen through a flat mirror at z = 5 mm;
    (B) the same emitter placed at its mirror image z = 15 mm, facing the SLM.

    With zero facet phase the two fields are equal (the virtual image point of Sec. 4.2)."""
    rng = np.random.default_rng(seed)
    tex = rng.uniform(0.0, 1.0, (32, 32, 3))
    half = 2 * MM
    # A: mirror at z = 5 mm facing -z, emitter at z = -5 mm facing +z
    a = _Builder("mirror-A")
    mm = a.material(MIRROR, albedo=(1.0, 1.0, 1.0))
    a.quad(np.array([-4 * MM, -4 * MM, 5 * MM]), np.array([8 * MM, 0, 0]), np.array([0, 8 * MM, 0]), mm, flip=True)
    ta = a.texture(tex)
    me = a.material(LAMBERT, albedo=(1, 1, 1), Le=(1, 1, 1), tex=ta, emit_tex=1)
    a.quad(np.array([-half, -half, -5 * MM]), np.array([2 * half, 0, 0]), np.array([0, 2 * half, 0]), me)
    # B: emitter at z = 15 mm facing -z with the same (x, y) -> uv map
    bb = _Builder("mirror-B")
    tb = bb.texture(tex)
    me2 = bb.material(LAMBERT, albedo=(1, 1, 1), Le=(1, 1, 1), tex=tb, emit_tex=1)
    bb.quad(np.array([-half, -half, 15 * MM]), np.array([2 * half, 0, 0]), np.array([0, 2 * half, 0]), me2, flip=True)
    return a.build(), bb.build()


def random_tri_soup(n, seed, extent=2 * MM, size=0.4 * MM, z0=3 * MM) -> Scene:
    """Random small triangles in front of the SLM (closest-hit brute-force tests)."""
    rng = np.random.default_rng(seed)
    b = _Builder(f"soup-{n}")
    m = b.material(LAMBERT, albedo=(0.5, 0.5, 0.5), Le=(1, 1, 1))
    c = np.stack([rng.uniform(-extent, extent, n), rng.uniform(-extent, extent, n),
                  rng.uniform(z0, z0 + 2 * extent, n)], 1)
    V = c[:, None, :] + rng.uniform(-size, size, (n, 3, 3))
    F = np.arange(3 * n).reshape(n, 3)
    e1, e2 = V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]
    nrm = np.cross(e1, e2)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    b.mesh(V.reshape(-1, 3), np.repeat(nrm, 3, 0), np.zeros((3 * n, 2)), F, m)
    return b.build()


def scene_bytes(s: Scene) -> int:
    n = 0
    for v in vars(s).values():
        if isinstance(v, np.ndarray):
            n += v.nbytes
    return n


def lit_receiver_scene(kind=LAMBERT, albedo=0.6, rough=0.3, z=5 * MM, Le=10.0) -> Scene:
    """A receiver plane facing the SLM, lit by a rectangular light placed off to the side
    (outside every pixel's cone) that faces the receiver."""
    b = _Builder("lit-receiver")
    m = b.material(kind, albedo=(albedo,) * 3, rough=rough)
    b.quad(np.array([-3 * MM, -3 * MM, z]), np.array([6 * MM, 0, 0]), np.array([0, 6 * MM, 0]), m, flip=True)
    b.rect_light(np.array([2 * MM, -1 * MM, 2 * MM]), np.array([2 * MM, 0, 0]), np.array([0, 2 * MM, 0]),
                 np.array([Le, Le, Le]))
    return b.build()


def multi_light_receiver_scene(kind=LAMBERT, albedo=0.6, rough=0.3, z=5 * MM) -> Scene:
    """The lit receiver with three rectangular lights of different sizes, positions and
    emission, all outside every pixel's cone and facing the receiver: light selection for NEE
    and its MIS weight over more than one light."""
    b = _Builder("lit-receiver-3-lights")
    m = b.material(kind, albedo=(albedo,) * 3, rough=rough)
    b.quad(np.array([-3 * MM, -3 * MM, z]), np.array([6 * MM, 0, 0]), np.array([0, 6 * MM, 0]), m, flip=True)
    b.rect_light(np.array([2 * MM, -1 * MM, 2 * MM]), np.array([2 * MM, 0, 0]), np.array([0, 2 * MM, 0]),
                 np.array([10.0, 10.0, 10.0]))
    b.rect_light(np.array([-4 * MM, -2.5 * MM, 3 * MM]), np.array([1.5 * MM, 0, 0]), np.array([0, 1 * MM, 0]),
                 np.array([30.0, 20.0, 5.0]))
    b.rect_light(np.array([-1 * MM, 2 * MM, 1.5 * MM]), np.array([0.5 * MM, 0, 0]), np.array([0, 0.5 * MM, 0.5 * MM]),
                 np.array([5.0, 40.0, 80.0]))
    return b.build()


def slab_scene(z0=3 * MM, thick=1 * MM, ze=8 * MM, ior=1.5) -> Scene:
    """A dielectric slab (parallel faces z0 and z0 + thick) in front of a uniform emitter at ze."""
    b = _Builder("dielectric-slab")
    md = b.material(DIELECTRIC, albedo=(1, 1, 1), ior=ior)
    b.box(np.array([-3 * MM, -3 * MM, z0]), np.array([3 * MM, 3 * MM, z0 + thick]), 1, md)
    me = b.material(LAMBERT, albedo=(0, 0, 0), Le=(1, 1, 1))
    b.quad(np.array([-4 * MM, -4 * MM, ze]), np.array([8 * MM, 0, 0]), np.array([0, 8 * MM, 0]), me, flip=True)
    return b.build()


def rotate_z90(s: Scene) -> Scene:
    """The same scene turned by +90 degrees about z: (x, y, z) -> (-y, x, z), exact in float32."""
    def rot(a):
        a = np.array(a, copy=True)
        x = a[:, 0].copy()
        a[:, 0] = -a[:, 1]
        a[:, 1] = x
        return a
    L = s.lights.copy()
    for k in (0, 3, 6):
        if len(L):
            L[:, k:k + 3] = rot(L[:, k:k + 3])
    P = s.points.copy()
    if len(P):
        P[:, 0:3] = rot(P[:, 0:3])
    out = Scene(rot(s.verts), rot(s.normals), s.uvs.copy(), s.tris.copy(), s.tri_mat.copy(), s.mat_type.copy(),
                s.mat_albedo.copy(), s.mat_rough.copy(), s.mat_ior.copy(), s.mat_Le.copy(), s.mat_tex.copy(),
                s.mat_emit_tex.copy(), s.mat_light.copy(), s.tex_data.copy(), s.tex_info.copy(), L, P,
                name=s.name + "-rotz90")
    out.validate()
    return out


ROT_Z_MINUS_90 = np.array([[0.0, 1.0, 0.0, 0.0], [-1.0, 0.0, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0],
                           [0.0, 0.0, 0.0, 1.0]])   # world -> hologram for a scene turned by +90 deg
