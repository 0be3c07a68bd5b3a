"""Pins of the ambient-cache construction in the FP64 oracle (no GPU): E(x) = pi/N sum L_i(x, w_s)
over directions uniform on the sphere, L_i the incoherent radiance arriving at the cell centre.
Checked against closed forms: the furnace, the solid angle of a rectangular emitter, darkness."""
import math

import numpy as np
import pytest

from paper_2606_14173_gb300 import scenes as S

MM = 1e-3


@pytest.mark.parametrize("depth", [1, 2, 3, 4])
def test_bake_furnace_is_exact(oracle_mod, depth):
    """Inside a closed box whose walls emit Le and reflect rho, every direction brings
    Le (1 - rho^D) / (1 - rho) at depth D, so E = pi Le (1 - rho^D) / (1 - rho) in every cell."""
    rho, Le = 0.5, 1.0
    o = oracle_mod.Oracle(S.furnace_scene(albedo=rho, Le=Le))
    E = o.bake(3, [-3 * MM, -3 * MM, -1 * MM], [3 * MM, 3 * MM, 5 * MM], 8, depth, seed=9)
    want = math.pi * Le * (1 - rho ** depth) / (1 - rho)
    assert np.max(np.abs(E - want)) < 1e-12 * want


def test_bake_dark_box(oracle_mod):
    o = oracle_mod.Oracle(S.furnace_scene(albedo=0.7, Le=0.0))
    E = o.bake(2, [-3 * MM, -3 * MM, -1 * MM], [3 * MM, 3 * MM, 5 * MM], 16, 4)
    assert np.all(E == 0.0)


def _rect_solid_angle(px, py, d, x0, x1, y0, y1):
    """Solid angle of the rectangle [x0, x1] x [y0, y1] in a plane at distance d from the point
    whose foot is (px, py): inclusion-exclusion over corner quadrants,
    Omega(a, b) = atan(a b / (d sqrt(a^2 + b^2 + d^2)))."""
    def om(a, b):
        return math.atan(a * b / (d * math.sqrt(a * a + b * b + d * d)))
    xs, ys = (x0 - px, x1 - px), (y0 - py, y1 - py)
    return om(xs[1], ys[1]) - om(xs[0], ys[1]) - om(xs[1], ys[0]) + om(xs[0], ys[0])


def test_bake_rectangular_emitter_solid_angle(oracle_mod):
    """Below a one-sided emitting square (radiance Le, no reflection), L_i is Le inside the
    square's solid angle Omega and 0 outside, so E = Le Omega / 4, within the binomial error."""
    Le, z, half = 2.0, 5 * MM, 3 * MM
    o = oracle_mod.Oracle(S.emissive_plane_scene(z=z, half=half, Le=Le))
    res, N = 2, 4096
    bmin, bmax = [-4 * MM, -2 * MM, 0.0], [4 * MM, 6 * MM, 4 * MM]
    E = o.bake(res, bmin, bmax, N, 1, seed=3)
    for cell in range(res ** 3):
        ix, iy, iz = cell % res, (cell // res) % res, cell // (res * res)
        x = [bmin[k] + (i + 0.5) * (bmax[k] - bmin[k]) / res for k, i in enumerate((ix, iy, iz))]
        om = _rect_solid_angle(x[0], x[1], z - x[2], -half, half, -half, half)
        p = om / (4 * math.pi)
        want = Le * om / 4
        sigma = math.pi * Le * math.sqrt(p * (1 - p) / N)
        for c in range(3):
            assert abs(E[cell, c] - want) < 4.5 * sigma + 1e-12, (cell, E[cell, c], want, sigma)


def test_bake_subset_equals_full_grid(oracle_mod):
    """Cells are independent: baking a subset gives the same values as the full grid."""
    o = oracle_mod.Oracle(S.config1_scene())
    lo, hi = [-8 * MM, -3 * MM, 5 * MM], [8 * MM, 5 * MM, 30 * MM]
    full = o.bake(4, lo, hi, 4, 3, seed=5)
    cells = np.array([0, 17, 63, 40])
    sub = o.bake(4, lo, hi, 4, 3, seed=5, cells=cells)
    assert np.array_equal(sub, full[cells])
    assert np.all(full >= 0) and full.max() > 0


def test_bake_sensitivity_bound(oracle_mod):
    """The float32-sensitivity bound of the bake: zero where the arriving radiance does not
    depend on the start point (the furnace: every direction brings the same radiance), and below
    a square emitter only the directions that pass within a few float32 ulps of its edges count,
    each by at most its full radiance: 0 <= sens <= pi Le, and the values E are those of or_bake."""
    rho, Le = 0.5, 1.0
    o = oracle_mod.Oracle(S.furnace_scene(albedo=rho, Le=Le))
    E, sens = o.bake(3, [-3 * MM, -3 * MM, -1 * MM], [3 * MM, 3 * MM, 5 * MM], 8, 3, seed=9, with_sens=True)
    assert np.all(sens == 0.0)
    assert np.array_equal(E, o.bake(3, [-3 * MM, -3 * MM, -1 * MM], [3 * MM, 3 * MM, 5 * MM], 8, 3, seed=9))
    Le = 2.0
    o = oracle_mod.Oracle(S.emissive_plane_scene(z=5 * MM, half=3 * MM, Le=Le))
    E, sens = o.bake(2, [-4 * MM, -2 * MM, 0.0], [4 * MM, 6 * MM, 4 * MM], 512, 1, seed=3, with_sens=True)
    assert np.all(sens >= 0.0) and np.all(sens <= math.pi * Le)
    # a direction within 32 ulps (~4e-6 relative) of an edge is rare among 512 uniform ones
    assert np.median(sens / np.maximum(E, 1e-30)) < 1e-2
