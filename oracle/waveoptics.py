"""FP64 oracle of the wave-optics steps around the path tracer (test infrastructure only).

- ``grf_maps``: the band-limited Gaussian random field phase maps of Eq. 4 (Sec. 4.3): for each
  hologram m, r_m = F^-1{ chi_Omega exp(i xi_m) } on a periodic grid of the SLM pitch, with the
  circular passband |f| <= sin(theta_max) / lambda = 1 / (2 pitch), and phi_m = arg r_m.
- ``asm_propagate``: the angular spectrum method (Sec. 3 "Angular Spectrum of Wave Field" and the
  two-stage scheme of Sec. 5): zero-pad the field to at least twice its size (next powers of
  two), multiply its spectrum by exp(i 2 pi z sqrt(1/lambda^2 - fx^2 - fy^2)) (evanescent
  components dropped), transform back and crop the original window.

numpy's FFT is the library primitive; everything else is written out here.  Only tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use this module.
"""
from __future__ import annotations

import numpy as np

from .oracle import grf_phases


def freqs(n: int, pitch: float) -> np.ndarray:
    """Spatial frequencies of an n-point periodic grid of the given pitch, in FFT order."""
    k = np.arange(n)
    return np.where(k < n // 2, k, k - n) / (n * pitch)


def grf_passband(nx: int, ny: int, pitch: float) -> np.ndarray:
    """chi_Omega on the [ny][nx] frequency grid: fx^2 + fy^2 <= (1 / (2 pitch))^2, decided
    exactly in integers: with fx = kx / (nx pitch), fy = ky / (ny pitch) the test is
    4 (kx^2 ny^2 + ky^2 nx^2) <= nx^2 ny^2 (frequencies on the circle are inside)."""
    k = lambda n: np.where(np.arange(n) < n // 2, np.arange(n), np.arange(n) - n).astype(np.int64)
    kx, ky = k(nx), k(ny)
    return 4 * (kx[None, :] ** 2 * ny ** 2 + ky[:, None] ** 2 * nx ** 2) <= nx ** 2 * ny ** 2


def grf_field(seed: int, m: int, nx: int, ny: int, pitch: float) -> np.ndarray:
    """r_m of Eq. 4 on the [ny][nx] grid (complex128; the inverse DFT without 1/N)."""
    spec = np.where(grf_passband(nx, ny, pitch), np.exp(1j * grf_phases(seed, m, nx, ny)), 0.0)
    return np.fft.ifft2(spec) * (nx * ny)


def grf_maps(seed: int, K: int, nx: int, ny: int, pitch: float, hologram_offset: int = 0) -> np.ndarray:
    """phi_m = arg r_m for m = hologram_offset .. hologram_offset + K - 1: [K][ny][nx] radians."""
    return np.stack([np.angle(grf_field(seed, hologram_offset + m, nx, ny, pitch)) for m in range(K)])


def pad_shape(W: int, H: int) -> tuple[int, int]:
    """(Wp, Hp): the next powers of two of at least twice the field size (double zero-padding)."""
    def p2(n):
        return 1 << max(0, int(np.ceil(np.log2(2 * n))))
    return p2(W), p2(H)


def transfer(Wp: int, Hp: int, pitch: float, lam: float, z: float) -> np.ndarray:
    """Angular-spectrum transfer function over distance z (m) on the padded grid, FFT order."""
    fx, fy = freqs(Wp, pitch), freqs(Hp, pitch)
    arg = 1.0 / lam ** 2 - fx[None, :] ** 2 - fy[:, None] ** 2
    return np.where(arg > 0, np.exp(2j * np.pi * z * np.sqrt(np.maximum(arg, 0.0))), 0.0)


def asm_periodic(P: np.ndarray, pitch: float, lam: float, z: float) -> np.ndarray:
    """One periodic angular-spectrum step on the whole grid P[Hp][Wp] (no padding)."""
    Hp, Wp = P.shape
    return np.fft.ifft2(np.fft.fft2(P) * transfer(Wp, Hp, pitch, lam, z))


def asm_propagate(U: np.ndarray, pitch: float, lambdas, z: float, K: int | None = None) -> np.ndarray:
    """Propagate fields U[..., H, W] by z; lambdas gives the wavelength of each field along the
    first axis (the layout [n_lambda][K][H][W] of the tracer's output)."""
    U = np.asarray(U, np.complex128)
    H, W = U.shape[-2:]
    Wp, Hp = pad_shape(W, H)
    ox, oy = (Wp - W) // 2, (Hp - H) // 2
    out = np.empty_like(U)
    lead = U.shape[:-2]
    flat = U.reshape(-1, H, W)
    res = out.reshape(-1, H, W)
    per_lam = flat.shape[0] // len(lambdas)
    for f in range(flat.shape[0]):
        lam = lambdas[f // per_lam]
        P = np.zeros((Hp, Wp), np.complex128)
        P[oy:oy + H, ox:ox + W] = flat[f]
        Q = asm_periodic(P, pitch, lam, z)
        res[f] = Q[oy:oy + H, ox:ox + W]
    return out.reshape(lead + (H, W))


# ---------------------------------------------------------------------------------------------
# Phase-only encoding with complex supervision (Sec. 2 and 5): gradient descent on the SLM
# phase phi so that the field exp(i phi) propagated by z matches the complex target T up to the
# phase-shift-invariant scale s = <A, T> / <A, A> (the least-squares complex factor, which
# absorbs a global amplitude and phase).  Loss L = sum |s A - T|^2 with A = P_z(exp(i phi));
# at the optimal s, dL/dphi = -2 Im(u conj(G)) with u = exp(i phi) and G = P_z^H(conj(s) R),
# R = s A - T, and P_z^H the same padded ASM over -z (the transfer function is unitary on the
# propagating components).  The supplementary section with the optimiser's details is not
# available: plain gradient descent with a fixed step is the reading.
# ---------------------------------------------------------------------------------------------
def encode_loss_grad(phi, T, pitch, lam, z):
    """(loss, gradient, s) of the complex-supervised phase-only objective at phi [H][W]."""
    u = np.exp(1j * phi)
    A = asm_propagate(u[None, None], pitch, [lam], z)[0, 0]
    s = np.vdot(A, T) / np.vdot(A, A)
    R = s * A - T
    G = asm_propagate((np.conj(s) * R)[None, None], pitch, [lam], -z)[0, 0]
    return float(np.sum(np.abs(R) ** 2)), -2.0 * np.imag(u * np.conj(G)), s


def encode(phi0, T, pitch, lam, z, iters, lr):
    """iters gradient steps phi <- phi - lr dL/dphi from phi0; returns (phi, losses before each step)."""
    phi = np.array(phi0, np.float64)
    losses = []
    for _ in range(iters):
        L, g, _ = encode_loss_grad(phi, T, pitch, lam, z)
        losses.append(L)
        phi = phi - lr * g
    return phi, np.array(losses)
