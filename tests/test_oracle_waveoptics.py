"""Pins of the FP64 wave-optics oracle (no GPU): the GRF phase maps of Eq. 4 and the angular
spectrum propagation of the two-stage scheme (Sec. 5), each checked against what the paper and
the mathematics fix rather than against the oracle's own formulas."""
import math

import numpy as np
import pytest

from paper_2606_14173_gb300 import scenes as S


@pytest.fixture(scope="module")
def wo(oracle_mod):
    from oracle import waveoptics
    return waveoptics


def test_grf_equals_the_direct_spectral_sum(wo):
    """r_m(x, y) = sum over the passband of exp(i xi) exp(2 pi i (fx x + fy y)) (Eq. 4), written
    out point by point on a small grid: pins the transform's sign, scale, frequency order and
    the passband radius sin(theta_max)/lambda = 1/(2 pitch)."""
    from oracle.oracle import grf_phases
    nx, ny, p, seed, m = 12, 10, 8e-6, 7, 3
    r = wo.grf_field(seed, m, nx, ny, p)
    xi = grf_phases(seed, m, nx, ny)
    for (jx, jy) in [(0, 0), (3, 7), (11, 9), (6, 5)]:
        acc = 0j
        for iy in range(ny):
            ky = iy if iy < ny / 2 else iy - ny
            fy = ky / (ny * p)
            for ix in range(nx):
                kx = ix if ix < nx / 2 else ix - nx
                fx = kx / (nx * p)
                # |f| <= 1/(2p) in exact rational arithmetic: (kx/nx)^2 + (ky/ny)^2 <= 1/4
                from fractions import Fraction
                if Fraction(kx, nx) ** 2 + Fraction(ky, ny) ** 2 <= Fraction(1, 4):
                    acc += np.exp(1j * xi[iy, ix]) * np.exp(2j * math.pi * (fx * jx * p + fy * jy * p))
        assert abs(r[jy, jx] - acc) <= 1e-9 * max(1.0, abs(acc))


def test_grf_statistics(wo):
    """Random spectral phases make r_m a circular complex Gaussian (Sec. 4.3): E|r|^2 equals the
    number of passband frequencies, arg r is uniform on (-pi, pi], and maps differ with m."""
    nx = ny = 128
    p = 6.4e-6
    n_pass = int(wo.grf_passband(nx, ny, p).sum())
    # the disk of radius 1/(2p) covers pi/4 of the square frequency grid
    assert abs(n_pass / (nx * ny) - math.pi / 4) < 0.01
    phis, pw = [], []
    for m in range(4):
        r = wo.grf_field(2, m, nx, ny, p)
        pw.append(np.mean(np.abs(r) ** 2) / n_pass)
        phis.append(np.angle(r).ravel())
    assert abs(np.mean(pw) - 1) < 1e-9          # Parseval: |exp(i xi)| = 1 on the passband
    ph = np.concatenate(phis)
    hist, _ = np.histogram(ph, bins=16, range=(-math.pi, math.pi))
    exp = len(ph) / 16
    chi2 = float(np.sum((hist - exp) ** 2 / exp))
    assert chi2 < 40                            # 15 dof, p ~ 1e-3
    assert abs(np.mean(np.exp(1j * (phis[0] - phis[1])))) < 0.05


def test_asm_plane_wave_is_exact(wo):
    """A periodic plane wave exp(2 pi i (fx x + fy y)) only gains exp(2 pi i z sqrt(1/lambda^2 -
    fx^2 - fy^2)) over z (the angular spectrum of a plane wave is one coefficient)."""
    Wp, Hp, p, lam, z = 64, 32, 8e-6, 520e-9, 12e-3
    kx, ky = 5, -3
    fx, fy = kx / (Wp * p), ky / (Hp * p)
    x = np.arange(Wp) * p
    y = np.arange(Hp) * p
    P = np.exp(2j * math.pi * (fx * x[None, :] + fy * y[:, None]))
    Q = wo.asm_periodic(P, p, lam, z)
    g = np.exp(2j * math.pi * z * math.sqrt(1 / lam ** 2 - fx ** 2 - fy ** 2))
    assert np.max(np.abs(Q - g * P)) < 1e-10


def test_asm_composes_and_reverses(wo):
    """Propagation by z1 then z2 equals propagation by z1 + z2, and by -z undoes +z."""
    rng = np.random.default_rng(3)
    P = rng.normal(size=(32, 64)) + 1j * rng.normal(size=(32, 64))
    p, lam = 6.4e-6, 638e-9
    a = wo.asm_periodic(wo.asm_periodic(P, p, lam, 4e-3), p, lam, 7e-3)
    b = wo.asm_periodic(P, p, lam, 11e-3)
    assert np.max(np.abs(a - b)) < 1e-9 * np.max(np.abs(P))
    c = wo.asm_periodic(wo.asm_periodic(P, p, lam, 9e-3), p, lam, -9e-3)
    assert np.max(np.abs(c - P)) < 1e-9 * np.max(np.abs(P))
    # no evanescent components at these pitches: the step is unitary (Parseval)
    assert abs(np.sum(np.abs(b) ** 2) / np.sum(np.abs(P) ** 2) - 1) < 1e-12


def test_two_stage_point_source(wo):
    """Two-stage scheme (Sec. 5): the spherical wave exp(ikr)/r of a point 20 mm from the SLM,
    recorded on a wave recording plane 5 mm from the point and inside the cone the pitch can
    carry, propagated 15 mm to the SLM by the padded ASM, matches the spherical wave there in
    the centre of the cone (mean ratio 1, phase 0, high correlation).  A wrong sign of z or a
    wrong transfer function scatters the ratio."""
    lam, p, N = 520e-9, 8e-6, 256
    zs, zw = 20e-3, 15e-3
    x = (np.arange(N) + 0.5 - N / 2) * p
    X, Y = np.meshgrid(x, x)
    rho = np.hypot(X, Y)

    def sph(d):
        r = np.sqrt(rho ** 2 + d ** 2)
        return np.exp(2j * math.pi * r / lam) / r

    th = math.asin(lam / (2 * p))
    Uw = sph(zs - zw) * (rho < (zs - zw) * math.tan(th))
    Us = wo.asm_propagate(Uw[None], p, [lam], zw)[0]
    ref = sph(zs)
    c = rho < 0.3 * zs * math.tan(th)
    ratio = np.mean(Us[c] / ref[c])
    assert abs(ratio - 1) < 0.03
    corr = abs(np.vdot(ref[c], Us[c])) / (np.linalg.norm(ref[c]) * np.linalg.norm(Us[c]))
    assert corr > 0.95
    bad = wo.asm_propagate(Uw[None], p, [lam], -zw)[0]
    assert abs(np.mean(bad[c] / ref[c]) - 1) > 0.5


def test_asm_padding_rule(wo):
    assert wo.pad_shape(1920, 1080) == (4096, 4096)
    assert wo.pad_shape(3840, 2160) == (8192, 8192)
    assert wo.pad_shape(100, 3) == (256, 8)


def test_trace_with_grf_maps(oracle_mod, wo):
    """Phase mode 2 samples map m at the image point's hologram-plane position Q (Eq. 4): with
    all-zero maps it equals the zero-phase mode; with a constant map c every hologram is the
    zero-phase field times exp(ic); with a ramp map the phase of one sample follows the grid
    cell of Q."""
    sc = S.config0_scene()
    o = oracle_mod.Oracle(sc)
    nx, ny = 64, 48
    r0 = S.config0_render(W=24, H=20, spp=4, K=3, phase_mode=S.PHASE_ZERO)
    U0 = o.trace(r0)
    rg = S.config0_render(W=24, H=20, spp=4, K=3, phase_mode=S.PHASE_GRF)
    zero = np.zeros((3, ny, nx))
    assert np.array_equal(o.trace(rg, grf=zero), U0)
    const = np.full((3, ny, nx), 0.7)
    assert np.max(np.abs(o.trace(rg, grf=const) - U0 * np.exp(0.7j))) < 1e-12 * np.max(np.abs(U0))
    ramp = np.broadcast_to((np.arange(nx) * 0.37)[None, None, :], (3, ny, nx)).copy()
    for pix, s in [(5, 0), (123, 2), (300, 3)]:
        a = o.sample(r0, 0, pix, s)
        b = o.sample(rg, 0, pix, s, grf=ramp)
        if not a["ok"]:
            continue
        jx = math.floor(a["Qx"] / rg.pitch + nx / 2) % nx
        got = np.angle((b["re"] + 1j * b["im"]) / (a["re"] + 1j * a["im"]))
        assert abs(np.angle(np.exp(1j * (got - 0.37 * jx)))) < 1e-9


def _target(wo, rng, W, H, p, lam, z):
    phi = rng.uniform(-math.pi, math.pi, (H, W))
    return wo.asm_propagate(np.exp(1j * phi)[None, None], p, [lam], z)[0, 0], phi


def test_encode_gradient_is_the_derivative(wo):
    """Central finite differences of the loss at a few pixels equal the analytic gradient
    (pins the adjoint ASM, the Wirtinger factor and the sign)."""
    rng = np.random.default_rng(1)
    W, H, p, lam, z = 24, 16, 8e-6, 520e-9, 2e-3
    T = rng.normal(size=(H, W)) + 1j * rng.normal(size=(H, W))
    phi = rng.uniform(-math.pi, math.pi, (H, W))
    L0, g, _ = wo.encode_loss_grad(phi, T, p, lam, z)
    h = 1e-6
    for (y, x) in [(0, 0), (5, 17), (15, 23), (8, 3)]:
        e = np.zeros_like(phi)
        e[y, x] = h
        fd = (wo.encode_loss_grad(phi + e, T, p, lam, z)[0] - wo.encode_loss_grad(phi - e, T, p, lam, z)[0]) / (2 * h)
        assert abs(fd - g[y, x]) <= 1e-6 * max(1.0, abs(fd)), (y, x, fd, g[y, x])


def test_encode_scale_is_phase_shift_invariant(wo):
    """A global phase of the target changes nothing, a global amplitude c scales the loss and
    its gradient by |c|^2 (the scale factor absorbs both; with the step divided by |c|^2 the
    iterates are the same)."""
    rng = np.random.default_rng(2)
    W, H, p, lam, z = 20, 12, 8e-6, 638e-9, 3e-3
    T, _ = _target(wo, rng, W, H, p, lam, z)
    phi0 = rng.uniform(-math.pi, math.pi, (H, W))
    a, la = wo.encode(phi0, T, p, lam, z, 5, 0.05)
    b, lb = wo.encode(phi0, T * np.exp(1.1j), p, lam, z, 5, 0.05)
    assert np.max(np.abs(a - b)) < 1e-9 and np.allclose(lb, la, rtol=1e-9)
    c, lc = wo.encode(phi0, T * 0.3, p, lam, z, 5, 0.05 / 0.09)
    assert np.max(np.abs(a - c)) < 1e-9 and np.allclose(lc, la * 0.09, rtol=1e-9)


def test_encode_descends_towards_a_reachable_target(wo):
    """A target made by propagating a phase-only field is reachable: the loss falls steadily."""
    rng = np.random.default_rng(3)
    W, H, p, lam, z = 32, 32, 8e-6, 520e-9, 1e-3
    T, _ = _target(wo, rng, W, H, p, lam, z)
    phi0 = rng.uniform(-math.pi, math.pi, (H, W))
    lr = 0.1 / float(np.sum(np.abs(T) ** 2) / (W * H))
    _, L = wo.encode(phi0, T, p, lam, z, 60, lr)
    assert np.all(np.diff(L) <= 1e-12 * L[0]) and L[-1] < 0.5 * L[0]
