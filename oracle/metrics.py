"""Reductions of traced photons (test infrastructure, plain numpy).

Fig. 1 (g)-(i) of the paper are spot diagrams at a field angle; Fig. 2 (b)
is collection efficiency against incidence angle.  The paper quotes no
number for either; the readings used here are
  PSF centroid = mean focal-plane (x, y) of the DETECTED photons;
  R80 = nearest-rank 80th percentile of their radial distance to the
        centroid (sorted index ceil(0.8 N) - 1);
  A_eff = N_detected / N_emitted * pi R_b^2 (bundle radius R_b);
  CE = N_detected / N_emitted.
"""
import math

import numpy as np

DETECTED = 1


def psf(status, focal_xy):
    det = status == DETECTED
    n = int(det.sum())
    if n == 0:
        return {"n_detected": 0, "cx": float("nan"), "cy": float("nan"), "r80": float("nan")}
    x = focal_xy[0][det].astype(np.float64)
    y = focal_xy[1][det].astype(np.float64)
    cx, cy = x.mean(), y.mean()
    r = np.sort(np.hypot(x - cx, y - cy))
    k = int(math.ceil(0.8 * n)) - 1
    return {"n_detected": n, "cx": float(cx), "cy": float(cy), "r80": float(r[k])}


def effective_area(status, bundle_radius):
    return float((status == DETECTED).sum()) / status.shape[0] * math.pi * bundle_radius ** 2


def collection_efficiency(status):
    return float((status == DETECTED).sum()) / status.shape[0]
