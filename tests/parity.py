"""Per-pixel comparison of complex fields against the FP64 oracle.

Bar: relative error |dU| / |U_ref| <= 1e-4 and phase error <= 1e-3 rad per pixel, on at
least 99.9 % of the pixels of every (wavelength, hologram) output.  Where |U_ref| is tiny
because random facet phases cancel (|U_ref| < 1e-3 RMS), the bound is |dU| <= 1e-4 RMS
instead; the phase is only checked where |U_ref| >= 0.1 RMS (it is undefined at zero).
"""
import numpy as np

REL_TOL = 1e-4
PHASE_TOL = 1e-3
PASS_FRAC = 0.999


def compare(U, ref):
    U = np.asarray(U, np.complex128).reshape(-1)
    ref = np.asarray(ref, np.complex128).reshape(-1)
    rms = float(np.sqrt(np.mean(np.abs(ref) ** 2))) if ref.size else 0.0
    a = np.abs(ref)
    d = np.abs(U - ref)
    if rms == 0.0:
        ok = d == 0.0
        return {"n": U.size, "frac_fail": float(1 - ok.mean()) if U.size else 0.0, "max_rel": 0.0,
                "max_phase": 0.0, "rms": 0.0, "fail_idx": np.nonzero(~ok)[0]}
    small = a < 1e-3 * rms
    rel = np.where(small, d / rms, d / np.maximum(a, 1e-300))
    ok = rel <= REL_TOL
    ph_mask = a >= 0.1 * rms
    ph = np.zeros_like(a)
    ph[ph_mask] = np.abs(np.angle(U[ph_mask] / ref[ph_mask]))
    ok &= ph <= PHASE_TOL
    return {"n": U.size, "frac_fail": float(1 - ok.mean()), "max_rel": float(rel.max()),
            "p999_rel": float(np.quantile(rel, 0.999)), "median_rel": float(np.median(rel)),
            "max_phase": float(ph.max()), "rms": rms, "fail_idx": np.nonzero(~ok)[0]}


def assert_parity(U, ref, label=""):
    """Every (lambda, m) output passes the bar; returns the per-output reports."""
    U = np.asarray(U)
    ref = np.asarray(ref)
    assert U.shape == ref.shape, (U.shape, ref.shape)
    reps = []
    for l in range(U.shape[0]):
        for m in range(U.shape[1]):
            r = compare(U[l, m], ref[l, m])
            reps.append(r)
            assert r["frac_fail"] <= 1 - PASS_FRAC, (
                f"{label} lambda {l} hologram {m}: {r['frac_fail'] * 100:.3f}% pixels out of tolerance "
                f"(max rel {r['max_rel']:.2e}, p99.9 rel {r['p999_rel']:.2e}, max phase {r['max_phase']:.2e})")
    return reps
