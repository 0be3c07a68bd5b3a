"""Pins of the oracle's texture and ambient-cache lookups (CPU only).

Both lookups are interpolations with a plain definition, so they are pinned by what
interpolation must reproduce exactly:

* bilinear filtering of the samples of a function affine in the texel index reproduces that
  function between the texel centres and holds the edge value in the clamp band; with
  different slopes along the two axes and per channel, a half-texel offset, a flipped or
  transposed axis or a wrong channel stride changes the value;
* at the texel centres (i + 1/2) / w the lookup returns the texel itself;
* the same for the trilinear cache read of a grid affine in the cell index, on a box that is
  not a cube, which fixes the [z][y][x][c] order and the cell-centre convention;
* through whole samples: an emitting textured quad seen at depth 1 radiates Le times the
  affine texture at the hit point's (u, v); in a closed Lambertian box with a constant cache,
  the path ends at its second vertex with L = Le + rho Le + rho^2 E / pi exactly (the ambient
  read-out of the hot-path table, Sec. 4.2), and without the cache L = Le + rho Le.
"""
import math

import numpy as np
import pytest

from paper_2606_14173_gb300 import scenes as S

MM = S.MM


def _affine_texture(w, h, a, bx, by):
    """T[j][i][c] = a_c + bx_c i + by_c j (row j along v, column i along u)."""
    i = np.arange(w)[None, :, None]
    j = np.arange(h)[:, None, None]
    return (np.asarray(a)[None, None, :] + np.asarray(bx)[None, None, :] * i +
            np.asarray(by)[None, None, :] * j).astype(np.float32)


def _textured_quad_scene(tex, z=5 * MM, half=1.5 * MM, Le=(1.0, 2.0, 3.0)):
    """One emitting quad facing the SLM; u runs along +x, v along +y."""
    b = S._Builder("textured-quad")
    t = b.texture(tex)
    m = b.material(S.LAMBERT, albedo=(1.0, 1.0, 1.0), Le=Le, tex=t, emit_tex=1)
    b.quad(np.array([-half, -half, z]), np.array([2 * half, 0, 0]), np.array([0, 2 * half, 0]), m, flip=True)
    return b.build()


A, BX, BY = (1.0, 0.5, 0.125), (0.03125, -0.015625, 0.0078125), (-0.0625, 0.046875, 0.09375)


def _affine_value(u, v, w, h, c):
    x = min(max(u * w - 0.5, 0.0), w - 1.0)
    y = min(max(v * h - 0.5, 0.0), h - 1.0)
    return A[c] + BX[c] * x + BY[c] * y


def test_texture_lookup_reproduces_an_affine_texture(oracle_mod):
    w, h = 11, 7
    orc = oracle_mod.Oracle(_textured_quad_scene(_affine_texture(w, h, A, BX, BY)))
    rng = np.random.default_rng(5)
    # the interior, the clamp bands of all four edges, and coordinates outside [0, 1]
    uv = np.concatenate([rng.uniform(0, 1, (300, 2)), rng.uniform(-0.2, 0.06, (60, 2)),
                         rng.uniform(0.94, 1.3, (60, 2)), [[0.0, 0.0], [1.0, 1.0], [0.5 / w, 0.5 / h]]])
    for u, v in uv:
        for c in range(3):
            got = orc.tex_lookup(0, u, v, c)
            assert abs(got - _affine_value(u, v, w, h, c)) <= 1e-12, (u, v, c)


def test_texture_lookup_at_texel_centres_is_the_texel(oracle_mod):
    w, h = 3, 2
    tex = np.random.default_rng(9).uniform(0, 1, (h, w, 3)).astype(np.float32)
    orc = oracle_mod.Oracle(_textured_quad_scene(tex))
    for j in range(h):
        for i in range(w):
            for c in range(3):
                assert orc.tex_lookup(0, (i + 0.5) / w, (j + 0.5) / h, c) == float(tex[j, i, c])
    # halfway between the centres of columns 0 and 1 on row 0: their mean
    assert abs(orc.tex_lookup(0, 1.0 / w, 0.5 / h, 1) - 0.5 * (float(tex[0, 0, 1]) + float(tex[0, 1, 1]))) <= 1e-12


C0, CX, CY, CZ = (3.0, 40.0, 100.0), (1.0, -2.0, 0.5), (4.0, 0.25, -1.0), (-3.0, 1.5, 8.0)


def _affine_cache_scene(res, bmin, bmax):
    """The textured quad plus a res^3 cache E[z][y][x][c] = C0 + CX x + CY y + CZ z, every value
    exact in binary16."""
    sc = _textured_quad_scene(_affine_texture(2, 2, A, BX, BY))
    k = np.arange(res, dtype=np.float64)
    z, y, x = np.meshgrid(k, k, k, indexing="ij")
    E = np.stack([C0[c] + CX[c] * x + CY[c] * y + CZ[c] * z for c in range(3)], axis=-1)
    assert np.array_equal(E.astype(np.float16).astype(np.float64), E)
    sc.cache_res = res
    sc.cache_bmin = np.asarray(bmin, np.float32)
    sc.cache_bmax = np.asarray(bmax, np.float32)
    sc.cache_E = E.astype(np.float16)
    sc.validate()
    return sc


def test_cache_lookup_reproduces_an_affine_grid(oracle_mod):
    res = 6
    bmin = np.array([-2e-3, 1e-3, 4e-3], np.float32)
    bmax = np.array([3e-3, 2.5e-3, 12e-3], np.float32)
    orc = oracle_mod.Oracle(_affine_cache_scene(res, bmin, bmax))
    lo, hi = bmin.astype(np.float64), bmax.astype(np.float64)
    rng = np.random.default_rng(17)
    ext = hi - lo
    pts = np.concatenate([lo + rng.uniform(0, 1, (300, 3)) * ext,             # inside
                          lo + rng.uniform(-0.3, 1.3, (200, 3)) * ext,        # across the clamp bands
                          [lo + (np.array([2, 0, 5]) + 0.5) * ext / res]])    # a cell centre
    for p in pts:
        g = np.clip((p - lo) / ext * res - 0.5, 0.0, res - 1.0)
        for c in range(3):
            want = C0[c] + CX[c] * g[0] + CY[c] * g[1] + CZ[c] * g[2]
            assert abs(orc.cache_lookup(p, c) - want) <= 1e-9 * max(1.0, abs(want)), (p, c)
    # at the centre of cell (x, y, z) = (2, 0, 5) the stored value itself
    assert orc.cache_lookup(pts[-1], 0) == C0[0] + 2 * CX[0] + 0 * CY[0] + 5 * CZ[0]


def _render(**kw):
    base = dict(W=24, H=16, pitch=8 * S.UM, lambdas=(638e-9, 520e-9, 450e-9), channels=(0, 1, 2), spp=4,
                max_depth=1, K=1, phase_mode=S.PHASE_ZERO)
    base.update(kw)
    return S.Render(**base)


def test_textured_emitter_radiates_the_affine_texture(oracle_mod):
    """Depth 1: every sample's radiance is Le times the bilinear texture at the uv of its hit."""
    w, h = 9, 13
    half, Le = 1.5 * MM, (1.0, 2.0, 3.0)
    sc = _textured_quad_scene(_affine_texture(w, h, A, BX, BY), half=half, Le=Le)
    orc = oracle_mod.Oracle(sc)
    lo, hi = sc.verts.min(0).astype(np.float64), sc.verts.max(0).astype(np.float64)   # float32 corners
    r = _render()
    n = 0
    for lam in range(3):
        for pix in range(0, r.W * r.H, 37):
            for s in range(r.spp):
                rec = orc.sample(r, lam, pix, s)
                if not rec["ok"]:
                    continue
                u = (rec["Px"] - lo[0]) / (hi[0] - lo[0])
                v = (rec["Py"] - lo[1]) / (hi[1] - lo[1])
                want = Le[lam] * _affine_value(u, v, w, h, lam)
                assert abs(rec["L"] - want) <= 1e-12 * want, (lam, pix, s, rec["L"], want)
                n += 1
    assert n > 100


@pytest.mark.parametrize("depth", [2, 3])
def test_constant_cache_read_out_in_a_closed_box(oracle_mod, depth):
    rho, Le = 0.5, 0.25
    E = (0.75, 2.5, 6.0)
    sc = S.furnace_scene(albedo=rho, Le=Le)
    res = 4
    sc.cache_res = res
    sc.cache_bmin = np.array([-5e-3, -5e-3, -3e-3], np.float32)
    sc.cache_bmax = np.array([5e-3, 5e-3, 7e-3], np.float32)
    sc.cache_E = np.broadcast_to(np.asarray(E, np.float16), (res, res, res, 3)).copy()
    sc.validate()
    orc = oracle_mod.Oracle(sc)
    for use_cache in (1, 0):
        r = _render(W=8, H=8, spp=3, max_depth=depth, use_cache=use_cache)
        for lam in range(3):
            for pix in range(0, 64, 5):
                for s in range(r.spp):
                    rec = orc.sample(r, lam, pix, s)
                    assert rec["ok"]
                    if use_cache:
                        want = Le + rho * Le + rho * rho * E[lam] / math.pi
                    else:
                        want = sum(Le * rho ** k for k in range(depth))
                    assert abs(rec["L"] - want) <= 1e-12 * want, (use_cache, lam, pix, s, rec["L"], want)
