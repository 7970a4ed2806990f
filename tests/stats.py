"""Statistical acceptance of a sampled P(m) against a reference.

Reading of "agrees within sampling error" used throughout the tests:
  * bulk bins (reference P > bulk): |dP| <= zmax * sigma, and the mean of
    (dP/sigma)^2 over the bulk is below chi2_max.  Adjacent bins share the
    same trajectories, so their errors are strongly correlated and the mean
    z^2 has few effective degrees of freedom: no lower bound is imposed;
  * far-tail bins: |dP| <= zmax * sigma + tail_frac * max_m sigma, because a
    handful of rare trajectories feed both the estimate and its sigma there.
The scale of sigma itself is checked from both sides by pooled_z2 over
several independent runs (an over-estimated sigma would pass the one-run
bounds above).
"""
import numpy as np


def agreement(P, sigma, Pref, bulk=1e-5, zmax=5.0, chi2_max=2.5, tail_frac=0.05,
              sigma_floor=1e-13):
    P = np.asarray(P, dtype=np.float64)
    s = np.maximum(np.asarray(sigma, dtype=np.float64), sigma_floor)
    Pref = np.asarray(Pref, dtype=np.float64)
    d = P - Pref
    z = d / s
    sel = Pref > bulk
    out = {
        "max_z_bulk": float(np.max(np.abs(z[sel]))) if sel.any() else 0.0,
        "chi2_bulk": float(np.mean(z[sel] ** 2)) if sel.any() else 0.0,
        "tail_excess": float(np.max(np.abs(d) - zmax * s - tail_frac * s.max())),
        "frac_within_1sigma": float(np.mean(np.abs(z[sel]) <= 1.0)) if sel.any() else 1.0,
    }
    out["ok"] = (out["max_z_bulk"] <= zmax and out["chi2_bulk"] <= chi2_max
                 and out["tail_excess"] <= 0.0)
    return out


def pooled_z2(runs, bulk=1e-5, sigma_floor=1e-13):
    """Mean of (dP / sigma)^2 over the bulk bins (reference P > bulk) of
    several independent runs [(P, sigma, Pref), ...], and the fraction of
    those bins within one sigma.  The bins of one run share its trajectories
    (few effective degrees of freedom); independent runs add theirs.  With
    sigma the standard error of P the pooled mean is near 1 (t-distributed
    z with N_R - 1 degrees of freedom: (N_R - 1) / (N_R - 3)); a sigma too
    large by a factor f pulls it to 1 / f^2, too small to f^2."""
    z2, within = [], []
    for P, sigma, Pref in runs:
        P = np.asarray(P, dtype=np.float64)
        s = np.maximum(np.asarray(sigma, dtype=np.float64), sigma_floor)
        Pref = np.asarray(Pref, dtype=np.float64)
        sel = Pref > bulk
        z = (P[sel] - Pref[sel]) / s[sel]
        z2.append(z ** 2)
        within.append(np.abs(z) <= 1.0)
    z2 = np.concatenate(z2)
    within = np.concatenate(within)
    return {"mean_z2": float(np.mean(z2)), "frac_within_1sigma": float(np.mean(within)),
            "bins": int(z2.size)}
