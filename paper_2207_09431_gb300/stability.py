"""Stability of the two directional-derivative schemes (reading R2 of Sec. 2.2:
central, or the mean of central and second-order biased differences) on the
rising-bubble grid of Sec. 4.3 at density ratio 1000.

Every case runs on its own lattice through the C ABI; the library's watchdog
(non-finite rho, p, u or tau) ends a case.  This module only orchestrates.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs, lbm


def survival(cases, steps=20000, chunk=1000, stream=None, device="cuda"):
    """Runs each (params, discs, meta) case for up to `steps` steps.  Returns
    per-case dicts: steps survived, diverged flag, the largest Mach number
    max|u| / cs and the fraction of liquid nodes whose tau sits at a clamp at
    the last finite state, and the wall time."""
    out = []
    for p, discs, meta in cases:
        lat = lbm.Lattice(p, device=device, stream=stream)
        lat.set_fields(inputs.bubble_fields(p["nx"], p["ny"], 2, p["xi"], discs, seed=0, noise=1e-8))
        t0 = time.perf_counter()
        done, diverged = 0, False
        ma, clamp = 0.0, 0.0
        while done < steps:
            n = min(chunk, steps - done)
            try:
                lat.step(n)
            except lbm.LbmError as err:
                if err.status != -4:
                    raise
                diverged = True
                break
            done += n
            ux, uy, tau, C1 = lat.field("ux"), lat.field("uy"), lat.field("tau"), lat.field("C1")
            ma = float(np.sqrt(3.0) * np.max(np.hypot(ux, uy)))
            liquid = C1 > 0.5
            at = (np.abs(tau - p["tau_min"]) < 1e-6 * p["tau_min"]) | (np.abs(tau - p["tau_max"]) < 1e-6 * p["tau_max"])
            clamp = float(np.mean(at[liquid])) if liquid.any() else 0.0
        out.append(dict(meta, fd_scheme=p["fd_scheme"], steps=done, diverged=diverged, mach=ma,
                        tau_clamped=clamp, wall_s=round(time.perf_counter() - t0, 3)))
        del lat
    return out


def compare(steps=20000, density_ratio=1000.0, mobility=0, stream=None, **grid):
    """Both schemes on the same grid of cases; returns (rows, summary)."""
    rows = []
    for fd in (0, 1):
        rows += survival(inputs.paper_grid_cases(density_ratio=density_ratio, mobility=mobility, fd_scheme=fd, **grid),
                         steps=steps, stream=stream)
    summary = {}
    for fd in (0, 1):
        r = [x for x in rows if x["fd_scheme"] == fd]
        summary[f"fd{fd}"] = {"cases": len(r), "survived": sum(not x["diverged"] for x in r),
                              "flagged_mach_gt_0.1": sum(x["mach"] > 0.1 for x in r),
                              "flagged_tau_clamp_gt_half": sum(x["tau_clamped"] > 0.5 for x in r)}
    return rows, summary
