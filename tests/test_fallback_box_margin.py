"""The widened float box test of the double-precision fallback traversal is conservative.

The fallback decides a coherent ray's hit exactly (double Moller-Trumbore), but visits the BVH
with float slab tests against boxes widened by w = 2^-17 (|o|_inf + M), M the largest coordinate
magnitude of the scene bounds.  The claim: for any double ray (o, d) and any point X = o + t d
with t >= 0 inside a box whose coordinates are floats of magnitude <= M, the float test of the
widened box passes with tfar >= t's float image.  This emulates that test in float32 arithmetic
(FMA rounded once, from the exact float64 product) on points placed on box faces, edges and
corners, with axis-parallel and nearly axis-parallel directions and origins far from the box."""
import numpy as np

f32 = np.float32


def fma32(a, b, c):
    # a * b is exact in float64 (48 significant bits); the sum is rounded to float64 then float32,
    # which can differ from one rounding by 1 ulp of float32: far inside the margin tested here
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def widened_test(o, d, lo, hi, M, tl=f32(1e30)):
    of = o.astype(f32)
    df = d.astype(f32)
    w = f32(f32(np.max(np.abs(of)) + f32(M)) * f32(2.0 ** -17))
    inv = np.array([f32(1.0) / x if abs(x) > f32(1e-20) else np.copysign(f32(1e20), x) for x in df], f32)
    oa = np.array([f32(f32(of[k] + w) * inv[k]) for k in range(3)], f32)
    ob = np.array([f32(f32(of[k] - w) * inv[k]) for k in range(3)], f32)
    a = [fma32(lo[k], inv[k], -oa[k]) for k in range(3)]
    b = [fma32(hi[k], inv[k], -ob[k]) for k in range(3)]
    tn = max(max(min(a[0], b[0]), min(a[1], b[1])), max(min(a[2], b[2]), f32(0)))
    tf = min(min(max(a[0], b[0]), max(a[1], b[1])), min(max(a[2], b[2]), tl))
    return tn <= tf, tn, tf


def _cases(rng, n):
    for i in range(n):
        M = 10.0 ** rng.uniform(-3, 0)                       # scene bounds from 1 mm to 1 m
        c = rng.uniform(-0.8, 0.8, 3) * M
        half = (10.0 ** rng.uniform(-7, -1)) * M * rng.uniform(0.0, 1.0, 3)
        lo = np.clip(c - half, -M, M).astype(f32)
        hi = np.clip(c + half, -M, M).astype(f32)
        hi = np.maximum(hi, lo)
        # X on a face, an edge or a corner of the box (the hardest places)
        X = rng.uniform(lo.astype(float), hi.astype(float))
        for k in rng.choice(3, size=rng.integers(1, 4), replace=False):
            X[k] = float(lo[k] if rng.random() < 0.5 else hi[k])
        d = rng.normal(size=3)
        mode = i % 4
        if mode == 1:
            d[rng.integers(3)] = 0.0                         # axis-parallel in one coordinate
        elif mode == 2:
            d[rng.integers(3)] *= 1e-9                       # nearly parallel
        d /= np.linalg.norm(d)
        dist = (10.0 ** rng.uniform(-4, 0.5)) * M            # origin up to 3 M before X
        o = X - dist * d
        if mode == 3:
            o = o + rng.normal(size=3) * 1e-12 * M           # origin off the float grid
        yield o, d, lo, hi, M, dist


def test_widened_float_box_never_misses_a_box_the_double_ray_meets():
    rng = np.random.default_rng(17)
    misses = 0
    for o, d, lo, hi, M, dist in _cases(rng, 20000):
        ok, tn, tf = widened_test(o, d, lo, hi, M)
        # the culling bound of the fallback: the double t rounded up with a margin of 2^-16
        tl = f32(np.nextafter(f32(dist), f32(np.inf)) * f32(1.0 + 2.0 ** -16))
        ok2, _, _ = widened_test(o, d, lo, hi, M, tl)
        misses += (not ok) + (not ok2)
    assert misses == 0


def test_widening_is_small():
    """The widened test does not accept boxes far from the ray: a box 1e-4 M beside the ray
    (about 1500 w) is rejected."""
    rng = np.random.default_rng(3)
    for _ in range(2000):
        M = 10.0 ** rng.uniform(-3, 0)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        o = rng.uniform(-0.5, 0.5, 3) * M
        X = o + 0.3 * M * d
        n = np.cross(d, rng.normal(size=3))
        n /= np.linalg.norm(n)
        C = X + n * 1e-4 * M
        half = 1e-5 * M
        lo, hi = (C - half).astype(f32), (C + half).astype(f32)
        assert not widened_test(o, d, lo, hi, M)[0]
