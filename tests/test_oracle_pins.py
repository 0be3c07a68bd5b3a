"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms (Snell/Fresnel, Lambert's polygon
irradiance, the RS integral of a uniform plane in ring coordinates), brute
force, library routines, invariants of the method (virtual image point of
Sec. 4.2, Path Reuse of Sec. 4.3, the rigid transform of Eq. 3) and the Monte
Carlo convergence rate.  A plausible mistake (dropped cosine, wrong pdf,
transposed transform, wrong sign of the phase, off-by-one depth, wrong
refractive index in the OPL) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from paper_2606_14173_gb300 import scenes as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- RNG
def test_philox_known_answers(oracle_mod):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle_mod.philox4x32_10(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_half_decode_matches_numpy(oracle_mod):
    bits = np.array([0, 1, 1023, 1024, 15360, 31743, 32768 | 15360, 0x3555, 0x7BFF, 0x0400], np.uint16)
    for b in bits:
        assert oracle_mod.half_to_double(int(b)) == float(np.array([b], np.uint16).view(np.float16)[0])


# ------------------------------------------------------------------ cone sampling
@pytest.mark.parametrize("lam,pitch", [(520e-9, 8e-6), (638e-9, 6.4e-6), (450e-9, 3.74e-6)])
def test_cone_limits_and_pdf(oracle_mod, lam, pitch):
    d0, pdf = oracle_mod.cone_dir(lam, pitch, 0.0, 0.3)
    assert np.allclose(d0, [0, 0, 1], atol=0, rtol=0)
    # at u0 -> 1 the polar angle reaches theta_max = asin(lambda / 2p) (Sec. 4.1)
    d1, _ = oracle_mod.cone_dir(lam, pitch, 1.0, 0.0)
    sin_max = lam / (2 * pitch)
    assert d1[2] == pytest.approx(math.sqrt(1 - sin_max ** 2), rel=1e-14)
    assert math.hypot(d1[0], d1[1]) == pytest.approx(sin_max, rel=1e-12)
    # uniform in solid angle: pdf = 1 / cone solid angle
    omega = 2 * math.pi * (1 - math.sqrt(1 - sin_max ** 2))
    assert pdf == pytest.approx(1 / omega, rel=1e-12)


def test_cone_distribution_uniform_in_solid_angle(oracle_mod):
    rng = np.random.default_rng(0)
    lam, pitch = 520e-9, 8e-6
    cmax = math.sqrt(1 - (lam / (2 * pitch)) ** 2)
    n = 20000
    u = rng.random((n, 2))
    d = np.array([oracle_mod.cone_dir(lam, pitch, a, b)[0] for a, b in u])
    assert np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-15)
    # cos(theta) is uniform on [cos theta_max, 1]; azimuth uniform on [0, 2 pi)
    q = (1 - d[:, 2]) / (1 - cmax)
    h, _ = np.histogram(q, bins=20, range=(0, 1))
    chi2 = ((h - n / 20) ** 2 / (n / 20)).sum()
    assert chi2 < 45  # 19 dof, p ~ 1e-3
    az = (np.arctan2(d[:, 1], d[:, 0]) + 2 * np.pi) % (2 * np.pi)
    h, _ = np.histogram(az, bins=20, range=(0, 2 * np.pi))
    assert ((h - n / 20) ** 2 / (n / 20)).sum() < 45


# ----------------------------------------------------------------- ray queries
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bvh_closest_hit_equals_brute_force(oracle_mod, seed):
    sc = S.random_tri_soup(600, seed)
    o = oracle_mod.Oracle(sc)
    rng = np.random.default_rng(100 + seed)
    hits = 0
    for _ in range(1500):
        org = np.array([rng.uniform(-2e-3, 2e-3), rng.uniform(-2e-3, 2e-3), 0.0])
        d = rng.normal(size=3)
        d[2] = abs(d[2]) + 0.5
        d /= np.linalg.norm(d)
        a = o.closest_hit(org, d, brute=False)
        b = o.closest_hit(org, d, brute=True)
        assert a == b
        hits += a[1] >= 0
    assert hits > 250


# ------------------------------------------------------------------- materials
def test_fresnel_closed_forms(oracle_mod):
    n = 1.5
    assert oracle_mod.fresnel_dielectric(1.0, 1.0, n) == pytest.approx(((n - 1) / (n + 1)) ** 2, rel=1e-14)
    # Brewster: p-polarised reflectance vanishes, F = Rs / 2
    tb = math.atan(n)
    ci, ct = math.cos(tb), math.cos(math.asin(math.sin(tb) / n))
    rs = ((ci - n * ct) / (ci + n * ct)) ** 2
    assert oracle_mod.fresnel_dielectric(ci, 1.0, n) == pytest.approx(rs / 2, rel=1e-12)
    # total internal reflection beyond the critical angle
    crit = math.asin(1 / n)
    assert oracle_mod.fresnel_dielectric(math.cos(crit + 0.01), n, 1.0) == 1.0
    # reciprocity F(theta_i; n1 -> n2) == F(theta_t; n2 -> n1)
    for th in (0.1, 0.5, 0.9, 1.3):
        tt = math.asin(math.sin(th) / n)
        assert oracle_mod.fresnel_dielectric(math.cos(th), 1.0, n) == pytest.approx(
            oracle_mod.fresnel_dielectric(math.cos(tt), n, 1.0), rel=1e-12)


def _hemi_grid(n_t=400, n_p=200):
    t = (np.arange(n_t) + 0.5) / n_t * (np.pi / 2)
    p = (np.arange(n_p) + 0.5) / n_p * (2 * np.pi)
    T, P = np.meshgrid(t, p, indexing="ij")
    dw = (np.pi / 2 / n_t) * (2 * np.pi / n_p) * np.sin(T)
    w = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1)
    return w.reshape(-1, 3), dw.reshape(-1)


@pytest.mark.parametrize("alpha", [0.2, 0.5, 0.8])
def test_ggx_pdf_normal_incidence_closed_form(oracle_mod, alpha):
    """At wo = n the visible-normal pdf is D(h)/4 per unit wi, so its integral over the upper
    hemisphere is the GGX mass with theta_h <= 45 deg: tan^2 CDF t/(alpha^2 + t) at t = 1."""
    w, dw = _hemi_grid(800, 64)
    pdf = np.array([oracle_mod.ggx_eval(alpha, 1.0, np.array([0.0, 0.0, 1.0]), wi)[1] for wi in w])
    assert float((pdf * dw).sum()) == pytest.approx(1.0 / (1.0 + alpha ** 2), abs=2e-3)


@pytest.mark.parametrize("alpha", [0.2, 0.5])
def test_ggx_sampling_matches_evaluation(oracle_mod, alpha):
    """E[sample weight] = int f cos dwi (sampler and evaluator agree), pdf integrates to <= 1."""
    wo = np.array([math.sin(0.6), 0.0, math.cos(0.6)])
    w, dw = _hemi_grid(300, 150)
    ev = np.array([oracle_mod.ggx_eval(alpha, 1.0, wo, wi) for wi in w])
    albedo_quad = float((ev[:, 0] * w[:, 2] * dw).sum())
    pdf_int = float((ev[:, 1] * dw).sum())
    rng = np.random.default_rng(3)
    ws = []
    for a, b in rng.random((40000, 2)):
        ok, wi, wgt, pdf = oracle_mod.ggx_sample(alpha, 1.0, wo, a, b)
        ws.append(wgt if ok else 0.0)
        if ok:
            f, p2 = oracle_mod.ggx_eval(alpha, 1.0, wo, wi)
            assert p2 == pytest.approx(pdf, rel=1e-9)
            assert f * wi[2] / pdf == pytest.approx(wgt, rel=1e-9)
    ws = np.array(ws)
    assert ws.mean() == pytest.approx(albedo_quad, abs=4 * ws.std() / math.sqrt(len(ws)) + 2e-3)
    assert albedo_quad <= 1.0 + 1e-3 and 0.5 < pdf_int <= 1.0 + 1e-3


# --------------------------------------------------------------- the estimator
def _plane_exact(z, lam, pitch, Le):
    """RS integral (Eq. 2) of a uniform incoherent plane at distance z over the cone footprint:
    (sqrt(Le)/(i lam)) * 2 pi z * int_z^R e^{ikr}/r dr, R = z / cos(theta_max)."""
    k = 2 * np.pi / lam
    R = z / math.sqrt(1 - (lam / (2 * pitch)) ** 2)
    re = integrate.quad(lambda r: math.cos(k * r) / r, z, R, limit=400, epsabs=0, epsrel=1e-12)[0]
    im = integrate.quad(lambda r: math.sin(k * r) / r, z, R, limit=400, epsabs=0, epsrel=1e-12)[0]
    return math.sqrt(Le) / (1j * lam) * 2 * np.pi * z * (re + 1j * im)


@pytest.mark.parametrize("z", [5e-3, 7.5e-3])
def test_emissive_plane_matches_ring_integral(oracle_mod, z):
    sc = S.emissive_plane_scene(z=z, half=3e-3, Le=2.0)
    o = oracle_mod.Oracle(sc)
    r = S.config0_render(W=256, H=256, spp=512, phase_mode=S.PHASE_ZERO)
    U = o.trace_full(r)[0, 0].reshape(-1)
    exact = _plane_exact(z, r.lambdas[0], r.pitch, 2.0)
    mean = U.mean()
    sem = math.sqrt(U.real.var() + U.imag.var()) / math.sqrt(U.size)
    assert abs(mean - exact) < 4 * sem, (mean, exact, sem)
    assert sem < 0.015 * abs(exact)


def test_monte_carlo_error_falls_as_inverse_sqrt_n(oracle_mod):
    sc = S.emissive_plane_scene(z=5e-3, half=3e-3, Le=1.0)
    o = oracle_mod.Oracle(sc)
    sds, ns = [], [4, 16, 64, 256]
    for n in ns:
        U = o.trace_full(S.config0_render(W=48, H=48, spp=n, phase_mode=S.PHASE_ZERO))[0, 0].reshape(-1)
        sds.append(math.sqrt(U.real.var() + U.imag.var()))
    slope = np.polyfit(np.log(ns), np.log(sds), 1)[0]
    assert abs(slope + 0.5) < 0.05, slope


@pytest.mark.parametrize("depth", [1, 2, 3, 4])
def test_furnace_closed_form(oracle_mod, depth):
    """Closed emissive Lambertian box: every path returns L = Le (1 - rho^D) / (1 - rho) (Eq. 1)."""
    rho, Le = 0.6, 1.5
    o = oracle_mod.Oracle(S.furnace_scene(albedo=rho, Le=Le))
    r = S.config0_render(W=16, H=16, max_depth=depth, spp=4)
    rho = float(np.float32(rho))          # the scene stores float32 material values
    want = Le * (1 - rho ** depth) / (1 - rho)
    for pix in (0, 37, 255):
        for s in range(4):
            rec = o.sample(r, 0, pix, s)
            assert rec["ok"] and rec["L"] == pytest.approx(want, rel=1e-12)


def _polygon_irradiance(x, n, poly, Le):
    """Lambert's formula for a uniform polygonal source: E = Le/2 * sum_i Theta_i (n . g_i)."""
    E = 0.0
    m = len(poly)
    for i in range(m):
        a, b = poly[i] - x, poly[(i + 1) % m] - x
        th = math.acos(np.clip(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)), -1, 1))
        g = np.cross(a, b)
        E += th * np.dot(n, g / np.linalg.norm(g))
    return abs(0.5 * Le * E)


@pytest.mark.parametrize("depth", [1, 2])
def test_nee_matches_polygon_irradiance(oracle_mod, depth):
    """Depth 1: NEE alone; depth 2: NEE + BSDF sampling with MIS.  Both estimate rho/pi * E(P)."""
    rho, Le = 0.6, 10.0
    sc = S.lit_receiver_scene(S.LAMBERT, albedo=rho, Le=Le)
    o = oracle_mod.Oracle(sc)
    L = sc.lights[0].astype(np.float64)
    poly = [L[0:3], L[0:3] + L[3:6], L[0:3] + L[3:6] + L[6:9], L[0:3] + L[6:9]]
    r = S.config0_render(W=32, H=32, max_depth=depth, spp=1, phase_mode=S.PHASE_ZERO)
    ratios = []
    for pix in range(0, 1024, 3):
        for s in range(12):
            rec = o.sample(r, 0, pix, s)
            assert rec["ok"]
            P = np.array([rec["Px"], rec["Py"], rec["Pz"]])
            E = _polygon_irradiance(P, np.array([0, 0, -1.0]), poly, Le)
            ratios.append(rec["L"] / (rho / math.pi * E))
    ratios = np.array(ratios)
    assert ratios.mean() == pytest.approx(1.0, abs=4 * ratios.std() / math.sqrt(len(ratios)))


@pytest.mark.parametrize("depth", [1, 2])
def test_nee_over_three_lights_matches_polygon_irradiance(oracle_mod, depth):
    """Three lights of different sizes, tilts and emission: NEE picks one uniformly and weights it
    by the light count (depth 2 adds BSDF sampling with MIS over all three); the estimate of
    rho/pi * sum of the lights' irradiances E(P) must be unbiased."""
    rho = 0.6
    sc = S.multi_light_receiver_scene(S.LAMBERT, albedo=rho)
    o = oracle_mod.Oracle(sc)
    polys = []
    for L in sc.lights.astype(np.float64):
        polys.append(([L[0:3], L[0:3] + L[3:6], L[0:3] + L[3:6] + L[6:9], L[0:3] + L[6:9]], L[9 + 1]))
    r = S.config0_render(W=32, H=32, max_depth=depth, spp=1, phase_mode=S.PHASE_ZERO)
    ratios = []
    for pix in range(0, 1024, 3):
        for s in range(24):
            rec = o.sample(r, 0, pix, s)
            assert rec["ok"]
            P = np.array([rec["Px"], rec["Py"], rec["Pz"]])
            E = sum(_polygon_irradiance(P, np.array([0, 0, -1.0]), poly, Le) for poly, Le in polys)
            ratios.append(rec["L"] / (rho / math.pi * E))
    ratios = np.array(ratios)
    assert ratios.mean() == pytest.approx(1.0, abs=4 * ratios.std() / math.sqrt(len(ratios)))


def test_ggx_nee_and_mis_agree(oracle_mod):
    """A GGX receiver: NEE alone (depth 1) and NEE + BSDF sampling with MIS (depth 2) are two
    estimators of the same integral and must agree in expectation."""
    sc = S.lit_receiver_scene(S.GGX, albedo=0.9, rough=0.7, Le=10.0)
    o = oracle_mod.Oracle(sc)
    means = []
    for depth in (1, 2):
        r = S.config0_render(W=32, H=32, max_depth=depth, spp=1, phase_mode=S.PHASE_ZERO)
        v = np.array([o.sample(r, 0, pix, s)["L"] for pix in range(0, 1024, 2) for s in range(16)])
        means.append((v.mean(), v.std() / math.sqrt(len(v))))
    (m1, e1), (m2, e2) = means
    assert m1 > 0 and abs(m1 - m2) < 4 * math.hypot(e1, e2)


def test_mirror_virtual_image_equivalence(oracle_mod):
    """Sec. 4.2: through a flat mirror the virtual image point P' = O + d_OPL v reproduces the
    field of the emitter placed at its mirror image."""
    a, b = S.mirror_pair_scenes()
    r = S.config0_render(W=64, H=64, spp=8, max_depth=2, phase_mode=S.PHASE_ZERO)
    Ua = oracle_mod.Oracle(a).trace_full(r)
    Ub = oracle_mod.Oracle(b).trace_full(r)
    assert np.abs(Ub).mean() > 1.0
    assert np.max(np.abs(Ua - Ub)) <= 1e-9 * np.max(np.abs(Ub))


def test_slab_refraction_opl_closed_form(oracle_mod):
    """Two refractions through a parallel slab: d_OPL = (z0 + gap)/cos(theta) + n t / cos(theta_t)."""
    z0, th_, ze, n = 3e-3, 1e-3, 8e-3, 1.5
    sc = S.slab_scene(z0=z0, thick=th_, ze=ze, ior=n)
    o = oracle_mod.Oracle(sc)
    # the planes as stored (float32 coordinates)
    zs = sorted(set(float(v) for v in sc.verts[:, 2]))
    z0, z1, ze = zs[0], zs[1], zs[2]
    n = float(np.float32(n))
    th_ = z1 - z0
    r = S.config0_render(W=16, H=16, spp=64, max_depth=3, phase_mode=S.PHASE_ZERO)
    checked = 0
    for pix in range(0, 256, 5):
        for s in range(64):
            rec = o.sample(r, 0, pix, s)
            if not rec["ok"] or rec["vP"] != 3:
                continue
            ct = rec["cos"]
            st = math.sqrt(1 - ct * ct)
            ctt = math.sqrt(1 - (st / n) ** 2)
            want = z0 / ct + n * th_ / ctt + (ze - z1) / ct
            assert rec["opl"] == pytest.approx(want, rel=1e-13)
            assert rec["beta"] == pytest.approx(1.0, rel=1e-13)   # (n_i/n_t)^2 in, then out
            checked += 1
    assert checked > 2000


def test_emitter_inside_a_dielectric_closed_form(oracle_mod):
    """An emitter inside a dielectric slab seen through its front face: one refraction into the
    medium, so the path throughput is (n_i/n_t)^2 = 1/n^2 (radiance emitted in the medium loses
    n^2 on the way out into air) and d_OPL = z0/cos(theta) + n (ze - z0)/cos(theta_t).  Fixes the
    direction of the radiance scaling, which the slab's in-and-out case leaves open."""
    z0, thick, n = 3e-3, 2e-3, 1.5
    sc = S.slab_scene(z0=z0, thick=thick, ze=z0 + 0.8e-3, ior=n)
    o = oracle_mod.Oracle(sc)
    zs = sorted(set(float(v) for v in sc.verts[:, 2]))     # front face, emitter, back face (float32)
    z0, ze = zs[0], zs[1]
    n = float(np.float32(n))
    r = S.config0_render(W=16, H=16, spp=64, max_depth=3, phase_mode=S.PHASE_ZERO)
    checked = 0
    for pix in range(0, 256, 5):
        for s in range(64):
            rec = o.sample(r, 0, pix, s)
            if not rec["ok"] or rec["vP"] != 2:
                continue
            ct = rec["cos"]
            st = math.sqrt(1 - ct * ct)
            ctt = math.sqrt(1 - (st / n) ** 2)
            assert rec["opl"] == pytest.approx(z0 / ct + n * (ze - z0) / ctt, rel=1e-13)
            assert rec["beta"] == pytest.approx(1.0 / n ** 2, rel=1e-13)
            assert rec["L"] == pytest.approx(1.0, rel=1e-13)   # Le of the emitter, albedo 0
            checked += 1
    assert checked > 2000


def test_path_reuse_hologram_index_invariance(oracle_mod):
    """Sec. 4.3: only the facet phase depends on m; hologram m of a K = 8 run equals a K = 1 run
    offset to m, and zero phase makes all holograms equal."""
    sc = S.config0_scene()
    o = oracle_mod.Oracle(sc)
    r8 = S.config0_render(W=32, H=24, spp=4, K=8)
    U8 = o.trace_full(r8)
    for m in (0, 3, 7):
        U1 = o.trace_full(S.config0_render(W=32, H=24, spp=4, K=1, hologram_offset=m))
        assert np.array_equal(U8[:, m], U1[:, 0])
    assert not np.allclose(U8[:, 0], U8[:, 1])
    Uz = o.trace_full(S.config0_render(W=32, H=24, spp=4, K=4, phase_mode=S.PHASE_ZERO))
    for m in range(1, 4):
        assert np.array_equal(Uz[:, m], Uz[:, 0])


def test_rigid_transform_invariance(oracle_mod):
    """Eq. 3: turning the scene by +90 deg about z and mapping it back with T gives the same field."""
    sc = S.config0_scene()
    rot = S.rotate_z90(sc)
    r = S.config0_render(W=48, H=40, spp=6, phase_mode=S.PHASE_ZERO)
    U0 = oracle_mod.Oracle(sc).trace_full(r)
    r.T = S.ROT_Z_MINUS_90.copy()
    U1 = oracle_mod.Oracle(rot).trace_full(r)
    assert np.max(np.abs(U1 - U0)) <= 1e-10 * np.max(np.abs(U0))


def test_point_emitter_spherical_wave(oracle_mod):
    """A deterministic point emitter adds a e^{ikr} cos(theta)/r inside the cone, zero outside."""
    pts = [(1e-4, -2e-4, 5e-3, 1e-3), (3e-3, 0.0, 4e-3, 2e-3)]   # second one outside every cone
    sc = S.point_emitter_scene(pts)
    r = S.config0_render(W=64, H=48, spp=1)
    U = oracle_mod.Oracle(sc).trace_full(r)[0, 0]
    lam = r.lambdas[0]
    ii, jj = np.meshgrid(np.arange(r.W), np.arange(r.H))
    x = (ii + 0.5 - r.W / 2) * r.pitch
    y = (jj + 0.5 - r.H / 2) * r.pitch
    cmax = math.sqrt(1 - (lam / (2 * r.pitch)) ** 2)
    want = np.zeros_like(U)
    for (px, py, pz, a) in pts:
        rr = np.sqrt((px - x) ** 2 + (py - y) ** 2 + pz ** 2)
        c = pz / rr
        want += np.where(c >= cmax, a * np.exp(2j * np.pi * rr / lam) * c / rr, 0)
    assert np.count_nonzero(want) > 100
    assert np.max(np.abs(U - want)) <= 1e-9 * np.max(np.abs(want))


def test_point_emitter_without_obliquity_is_the_spherical_wave(oracle_mod):
    """With the obliquity factor left out, a point emitter gives exactly a e^{ikr} / r inside the
    cone (the analytic spherical wave), and every traced sample loses exactly its cos(theta)."""
    pts = [(1e-4, -2e-4, 5e-3, 1e-3)]
    sc = S.point_emitter_scene(pts)
    r = S.config0_render(W=48, H=40, spp=1, omit_obliquity=1)
    U = oracle_mod.Oracle(sc).trace_full(r)[0, 0]
    lam = r.lambdas[0]
    ii, jj = np.meshgrid(np.arange(r.W), np.arange(r.H))
    x = (ii + 0.5 - r.W / 2) * r.pitch
    y = (jj + 0.5 - r.H / 2) * r.pitch
    cmax = math.sqrt(1 - (lam / (2 * r.pitch)) ** 2)
    px, py, pz, a = pts[0]
    rr = np.sqrt((px - x) ** 2 + (py - y) ** 2 + pz ** 2)
    want = np.where(pz / rr >= cmax, a * np.exp(2j * np.pi * rr / lam) / rr, 0)
    assert np.count_nonzero(want) > 100
    assert np.max(np.abs(U - want)) <= 1e-9 * np.max(np.abs(want))
    o = oracle_mod.Oracle(S.config1_scene())
    r1 = S.config1_render(W=32, H=24, spp=4, K=1)
    r0 = S.config1_render(W=32, H=24, spp=4, K=1, omit_obliquity=1)
    for pix, smp in [(3, 0), (300, 2), (700, 3)]:
        a1, a0 = o.sample(r1, 0, pix, smp), o.sample(r0, 0, pix, smp)
        if a1["ok"] and a1["re"] != 0:
            assert abs((a1["re"] + 1j * a1["im"]) / (a0["re"] + 1j * a0["im"]) - a1["cos"]) < 1e-12


def test_conditioning_flags_and_bound(oracle_mod):
    """Per-pixel flags: bits 16-31 count ill-conditioned samples, bits 32-47 samples whose
    incoherent path met a mirror or dielectric; sens bounds the field change that float32-sized
    moves of the image points cause.  A diffuse receiver under an area light and a slab whose
    refractions belong to the coherent part of the path (Sec. 4.2: the chain up to the first
    non-delta vertex) are smooth: no ill-conditioned samples, no incoherent delta vertices and a
    bound mostly well below the 1e-4 tolerance.  In the scene with ~185k triangles and many small mirror
    and glass spheres, ill-conditioning is common but mostly comes with delta vertices."""
    r = S.config0_render(W=16, H=16, spp=8, max_depth=4)
    for sc in (S.lit_receiver_scene(S.LAMBERT), S.slab_scene()):
        U, fl, sens = oracle_mod.Oracle(sc).trace(r, with_flags=True)
        assert np.all((fl >> 16) == 0)
        assert np.median(sens / np.abs(U[:, 0])) <= 5e-5
    r3 = S.config3_render(W=24, H=24, spp=8, K=1)
    U, fl, sens = oracle_mod.Oracle(S.config3_scene()).trace(r3, with_flags=True)
    ill = (fl >> 16) & 0xFFFF
    delta = (fl >> 32) & 0xFFFF
    assert np.all(ill <= r3.spp) and np.all(delta <= r3.spp)
    assert 0 < ill.sum() < delta.sum()
    assert np.all(sens >= 0)
    # where no sample is ill-conditioned the bound mostly stays well below the tolerance
    assert np.median(sens[ill == 0] / np.abs(U[:, 0])[ill == 0]) <= 5e-5
