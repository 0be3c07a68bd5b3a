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


def attribute(U, ref, flags, sens):
    """Per (lambda, m) output: the pixels out of the bar and how the oracle accounts for each.

    A failing pixel is attributed when the oracle flags one of its samples -- a triangle edge
    or tie met within the float error band (flag bits 0-15), an ill-conditioned incoherent part
    (bits 16-31), an incoherent path through a mirror or dielectric (bits 32-47) -- or when its
    sensitivity bound sens, the largest change of its field under moves of its samples' image
    points by up to 32 float32 ulps (the error budget of a float32 incoherent path: one rounding
    of P, then a few ulps of direction and hit-point error at each of at most three incoherent
    vertices), reaches the strict tolerance of the pixel.  An attributed pixel is explained when
    it is near an edge or |dU| <= tolerance + sens.  Returns one dict per output."""
    U = np.asarray(U)
    ref = np.asarray(ref)
    flags = np.asarray(flags)
    sens = np.asarray(sens)
    reps = []
    for l in range(U.shape[0]):
        near = (flags[l].reshape(-1) & 0xFFFF) > 0
        ill = ((flags[l].reshape(-1) >> 16) & 0xFFFF) > 0
        delta = ((flags[l].reshape(-1) >> 32) & 0xFFFF) > 0
        sl = sens[l].reshape(-1)
        for m in range(U.shape[1]):
            r = compare(U[l, m], ref[l, m])
            u = np.asarray(U[l, m], np.complex128).reshape(-1)
            q = np.asarray(ref[l, m], np.complex128).reshape(-1)
            tol = REL_TOL * np.maximum(np.abs(q), 1e-3 * r["rms"])
            sensitive = near | (sl >= tol)
            flagged = near | ill | delta | (sl >= tol)
            bad = r["fail_idx"]
            d = np.abs(u[bad] - q[bad])
            explained = near[bad] | (flagged[bad] & (d <= tol[bad] + sl[bad]))
            r.update({"failing": int(len(bad)), "attributed": int(flagged[bad].sum()),
                      "failing_not_sensitive": int((~sensitive[bad]).sum()),
                      "explained": int(explained.sum()), "unexplained": int((~explained).sum()),
                      "failing_near_edge": int(near[bad].sum()), "failing_ill_conditioned": int(ill[bad].sum()),
                      "failing_incoherent_delta": int(delta[bad].sum()),
                      "sensitive_frac": float(sensitive.mean()) if sensitive.size else 0.0,
                      "sens_median_rel": float(np.median(sl / np.maximum(np.abs(q), 1e-300))) if q.size else 0.0})
            reps.append(r)
    return reps


def assert_parity_explained(U, ref, flags, sens, label="", sensitive_only=False):
    """The bar with its stated exception for float32-sensitive incoherent paths.

    The incoherent radiance is computed in float32 (its error budget is about 32 ulps of image-
    point displacement); where reflection and refraction at curved mirrors and lenses, shadow
    boundaries or near-specular lobes magnify that by 1e2-1e4, no float32 evaluation reproduces
    the FP64 radiance to 1e-4.  A pixel out of the bar is excused only when the oracle itself
    flags it (attribute()) and the disagreement stays within tolerance + its sensitivity bound;
    unexplained pixels <= 0.1 % of every output.  The excused pixels are therefore a subset of
    the pixels the oracle alone flags.  sensitive_only: moreover, the pixels out of the bar whose
    sensitivity bound stays below the tolerance (flagged only as ill-conditioned or as passing an
    incoherent delta vertex) must be <= 0.1 % of every output, so that the failures lie where the
    oracle's own float32 probes predict them.  Returns the per-output reports."""
    U = np.asarray(U)
    ref = np.asarray(ref)
    assert U.shape == ref.shape, (U.shape, ref.shape)
    reps = attribute(U, ref, flags, sens)
    k = 0
    for l in range(U.shape[0]):
        for m in range(U.shape[1]):
            r = reps[k]
            k += 1
            msg = (f"{label} lambda {l} hologram {m}: {r['failing']} of {r['n']} pixels out of tolerance, "
                   f"{r['unexplained']} unexplained, max rel {r['max_rel']:.2e}, sensitive pixels "
                   f"{100 * r['sensitive_frac']:.2f} %, median sens/|U| {r['sens_median_rel']:.2e}")
            assert r["unexplained"] <= (1 - PASS_FRAC) * r["n"], msg
            if sensitive_only:
                assert r["failing_not_sensitive"] <= (1 - PASS_FRAC) * r["n"], (
                    msg + f", {r['failing_not_sensitive']} of them outside the oracle's float32-sensitive set")
    return reps
