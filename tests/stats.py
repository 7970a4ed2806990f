"""Statistical acceptance of a sampled P(m) against a reference.

Reading of "agrees within sampling error" used throughout the tests:
  * bulk bins (reference P > bulk): |dP| <= zmax * sigma, and the mean of
    (dP/sigma)^2 over the bulk is below chi2_max.  Adjacent bins share the
    same trajectories, so their errors are strongly correlated and the mean
    z^2 has few effective degrees of freedom: no lower bound is imposed;
  * far-tail bins: |dP| <= zmax * sigma + tail_frac * max_m sigma, because a
    handful of rare trajectories feed both the estimate and its sigma there.
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
