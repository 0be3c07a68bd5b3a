"""The seeded synthetic inputs follow the benchmark configurations they stand in for (CPU):
scene contents, sizes and value ranges, render settings, and the serving stream's mix."""
import numpy as np
import pytest

from paper_2606_14173_gb300 import scenes as S

MM, UM, NM = S.MM, S.UM, S.NM


def _tri_normals(s):
    v = s.verts.astype(np.float64)[s.tris.astype(np.int64)]
    n = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    return n / np.linalg.norm(n, axis=1, keepdims=True), v


def _meshes_by_material(s):
    """Triangle vertex boxes grouped by material id (every sphere has a material of its own)."""
    v = s.verts[s.tris.astype(np.int64)]
    out = {}
    for m in np.unique(s.tri_mat):
        pts = v[s.tri_mat == m].reshape(-1, 3)
        out[int(m)] = (pts.min(0).astype(np.float64), pts.max(0).astype(np.float64))
    return out


def test_config0_two_textured_emissive_quads():
    s = S.config0_scene()
    s.validate()
    assert s.n_tris == 4
    n, v = _tri_normals(s)
    assert np.allclose(n, [0.0, 0.0, -1.0])                       # both quads face the SLM
    assert sorted(set(np.round(v[:, :, 2].ravel() / MM, 6))) == [5.0, 10.0]
    assert np.all(s.mat_type == S.LAMBERT) and np.all(s.mat_emit_tex == 1)
    assert s.tex_info.shape == (2, 3) and np.all(s.tex_info[:, 1:] == 64)
    tex = s.tex_data.reshape(2, 64, 64, 3)
    assert tex.min() >= 0.0 and tex.max() < 1.0 and abs(float(tex.mean()) - 0.5) < 0.02
    r = S.config0_render()
    assert (r.W, r.H, r.pitch, r.lambdas, r.spp, r.max_depth, r.K) == (256, 256, 8 * UM, (520 * NM,), 16, 1, 1)


def test_config1_icosphere_scene():
    s = S.config1_scene()
    s.validate()
    assert 18_000 <= s.n_tris <= 26_000                          # ~20k triangles
    kinds = s.mat_type
    assert list(kinds[:2]) == [S.LAMBERT, S.EMITTER]              # textured ground, the light
    sphere_kinds = kinds[2:]
    assert len(sphere_kinds) == 30
    counts = np.bincount(sphere_kinds, minlength=4)[:4]
    assert counts.max() - counts.min() <= 1                       # equal shares of the four materials
    ggx = sphere_kinds == S.GGX
    assert np.all((s.mat_rough[2:][ggx] >= 0.05) & (s.mat_rough[2:][ggx] <= 0.5))
    assert np.all(s.mat_ior[2:][sphere_kinds == S.DIELECTRIC] == np.float32(1.5))
    # spheres: radius 0.5-2 mm, centres x in [-8, 8] mm, z in [5, 30] mm, resting on the ground
    for m, (lo, hi) in _meshes_by_material(s).items():
        if m < 2:
            continue
        c, rad = (lo + hi) / 2, (hi - lo) / 2
        assert 0.45 * MM <= rad.max() <= 2.0 * MM + 1e-9, (m, rad)
        assert -8 * MM - 1e-9 <= c[0] <= 8 * MM + 1e-9 and 5 * MM - 1e-9 <= c[2] <= 30 * MM + 1e-9
        assert lo[1] >= -3 * MM - 1e-6
    ground = s.verts[s.tris[s.tri_mat == 0].astype(np.int64)].reshape(-1, 3)
    assert np.allclose(ground[:, 1], -3 * MM)
    assert np.allclose([ground[:, 0].min(), ground[:, 0].max()], [-20 * MM, 20 * MM])
    assert np.allclose([ground[:, 2].min(), ground[:, 2].max()], [0.0, 40 * MM])
    # one 10 x 10 mm rectangular light at y = 15 mm facing down, Le = 20
    assert s.lights.shape == (1, 12)
    L = s.lights[0].astype(np.float64)
    assert np.isclose(L[1], 15 * MM) and np.allclose(L[9:12], 20.0)
    nl = np.cross(L[3:6], L[6:9])
    assert np.isclose(np.linalg.norm(nl), 100 * MM * MM) and nl[1] < 0
    r = S.config1_render()
    assert (r.W, r.H, r.pitch, r.lambdas, r.spp, r.max_depth, r.K) == (1920, 1080, 6.4 * UM, S.RGB_LAMBDAS, 64, 4, 1)
    assert S.RGB_LAMBDAS == (638 * NM, 520 * NM, 450 * NM)
    assert S.config2_render().K == 8 and S.config2_render().path_samples() == 398_131_200


def test_config3_scene_at_scale():
    s = S.config3_scene()
    s.validate()
    assert 150_000 <= s.n_tris <= 210_000                        # ~200k triangles
    assert s.cache_res == 128 and s.cache_E.shape == (128, 128, 128, 3) and s.cache_E.dtype == np.float16
    assert np.all(np.isfinite(s.cache_E.astype(np.float32))) and float(s.cache_E.min()) >= 0.0
    lo = s.verts.min(0)
    hi = s.verts.max(0)
    assert np.all(s.cache_bmin <= lo) and np.all(s.cache_bmax >= hi)   # the grid covers the scene
    kinds = s.mat_type
    slabs = kinds[2:22]
    assert np.all(slabs[0::2] == S.GGX) and np.all(slabs[1::2] == S.DIELECTRIC)
    assert 400 <= len(kinds) - 22 <= 500                             # spheres kept (none inside a slab)
    r = S.config3_render()
    assert (r.W, r.H, r.pitch, r.spp, r.max_depth, r.K, r.use_cache) == (3840, 2160, 3.74 * UM, 256, 4, 8, 1)
    assert r.path_samples() == 6_370_099_200


def test_config4_stream_mix():
    reqs = S.config4_requests(2000)
    assert len(reqs) == 2000
    keys = [k for k, _ in reqs]
    frac = {k: keys.count(k) / 2000 for k in ("cfg0", "cfg1", "cfg3")}
    # configs 0-3 uniformly, configs 1 and 2 sharing the scene
    assert abs(frac["cfg0"] - 0.25) < 0.04 and abs(frac["cfg1"] - 0.5) < 0.05 and abs(frac["cfg3"] - 0.25) < 0.04
    sizes = {(r.W, r.H) for _, r in reqs}
    assert sizes == {(512, 512), (1920, 1080), (3840, 2160)}
    assert {r.spp for _, r in reqs} == {16, 32, 64, 128, 256}
    assert {r.K for _, r in reqs} == {1, 4, 8}
    for key, r in reqs:
        T = r.T
        assert np.allclose(T[:3, :3], np.eye(3))                       # poses translate only
        assert abs(T[0, 3]) <= 5 * MM and abs(T[1, 3]) <= 5 * MM      # eye offsets within +-5 mm
        df = S.SCENE_MEDIAN_DEPTH[key] + T[2, 3]                       # focal depth (T shifts z by df - median)
        assert 5 * MM - 1e-12 <= df <= 30 * MM + 1e-12
    assert len({r.seed for _, r in reqs}) == 2000                      # every request its own draws
    for (ka, ra), (kb, rb) in zip(S.config4_requests(50), S.config4_requests(50)):   # seeded
        assert ka == kb and (ra.W, ra.H, ra.spp, ra.K, ra.seed) == (rb.W, rb.H, rb.spp, rb.K, rb.seed)
        assert np.array_equal(ra.T, rb.T)


@pytest.mark.parametrize("fn", [S.config0_scene, S.config1_scene])
def test_scenes_are_seeded(fn):
    a, b = fn(), fn()
    assert np.array_equal(a.verts, b.verts) and np.array_equal(a.tris, b.tris)
    assert np.array_equal(a.mat_albedo, b.mat_albedo) and np.array_equal(a.tex_data, b.tex_data)
