"""FP64 post-processing of the oracle's raw observable sums (test infrastructure).

Definitions follow arXiv 2207.09431:
  rise velocity and centroid   V = sum C_g v / sum C_g,  y = sum C_g y / sum C_g   (Sec. 4.2, Eq. 43-44)
  drag coefficient             C_D = 4 d g (rho_l - rho_g) / (3 rho_l U^2)          (Sec. 4.1, Eq. 37)
  Reynolds number              Re = rho_l U^(2-n) d^n / k                           (Eq. 38)
  Morton number                Mo = g drho / (rho_l^2 sigma^3) [k (U/d)^(n-1)]^4    (Eq. 39)
  Eotvos number                Eo = drho g d^2 / sigma                              (Eq. 40)
  aspect ratio                 E = vertical / horizontal extent of the bubble       (Sec. 4.1, below Eq. 41)
  thresholded mass             sum of C_i over nodes with C_i > 0.5                 (Sec. 3.1)

Reading: the paper's equivalent diameter is the 3-D cube-root formula; in this
2-D model the area-equivalent diameter d = 2 sqrt(A / pi) with A = sum C_g is
used instead.
"""
from __future__ import annotations

import math


def drag_coefficient(d, g, rho_l, rho_g, U):
    """Eq. 37: buoyancy-balanced drag coefficient at terminal velocity U."""
    return 4.0 * d * g * (rho_l - rho_g) / (3.0 * rho_l * U * U)


def reynolds(rho_l, U, d, n, k):
    """Eq. 38: power-law Reynolds number."""
    return rho_l * abs(U) ** (2.0 - n) * d ** n / k


def morton(g, rho_l, rho_g, sigma, k, U, d, n):
    """Eq. 39: power-law Morton number."""
    return g * (rho_l - rho_g) / (rho_l ** 2 * sigma ** 3) * (k * (abs(U) / d) ** (n - 1.0)) ** 4


def eotvos(rho_l, rho_g, g, d, sigma):
    """Eq. 40: Eotvos number."""
    return (rho_l - rho_g) * g * d * d / sigma


def li_correlation(Re, n, E):
    """Eq. 41 (Li et al. correlation, used only to cross-check printed tables)."""
    return 16.0 / Re * (1.0 + 0.43 * Re ** 0.44) * (1.0 + 3.868 * n ** 0.7528 * (1.0 - E) ** 0.6810)


def postprocess(params: dict, raw, gas_comp=None) -> dict:
    """Turn the 15 raw sums of ``orc_observables`` into the observables."""
    gc = int(params.get("gas_comp", 3) if gas_comp is None else gas_comp)
    rho = params["rho"]
    rho_l, rho_g = float(rho[0]), float(rho[gc - 1])
    sigma = float(params["sigma13"] if gc == 3 else params["sigma12"])
    g = float(params.get("gravity", 0.0))
    n = float(params.get("pl_n", 1.0)) if params.get("powerlaw", 0) else 1.0
    if params.get("powerlaw", 0):
        k = float(params["pl_k"])
    else:
        k = rho_l * float(params["tau"][0]) / 3.0
    A = raw[6]
    out = {
        "mass": [raw[0], raw[1], raw[2]],
        "mass_thr": [raw[3], raw[4], raw[5]],
        "area": A,
    }
    if A > 0:
        cx, cy = raw[7] / A, raw[8] / A
        vx, vy = raw[9] / A, raw[10] / A
    else:
        cx = cy = vx = vy = float("nan")
    out["centroid"] = [cx, cy]
    out["velocity"] = [vx, vy]
    out["rise_velocity"] = vy
    d = 2.0 * math.sqrt(A / math.pi) if A > 0 else float("nan")
    out["d_eq"] = d
    xmin, xmax, ymin, ymax = raw[11:15]
    if xmin >= 0:
        E = (ymax - ymin + 1.0) / (xmax - xmin + 1.0)
    else:
        E = float("nan")
    out["aspect_E"] = E
    U = vy
    if A > 0 and U != 0 and g != 0:
        out["drag_coefficient"] = drag_coefficient(d, g, rho_l, rho_g, U)
    else:
        out["drag_coefficient"] = float("nan")
    out["Re"] = reynolds(rho_l, U, d, n, k) if A > 0 else float("nan")
    out["Eo"] = eotvos(rho_l, rho_g, g, d, sigma) if A > 0 else float("nan")
    out["Mo"] = morton(g, rho_l, rho_g, sigma, k, U, d, n) if (A > 0 and U != 0) else float("nan")
    return out
