"""Surrogate of the rising-bubble terminal state, with the solver as fallback.

The network (CUDA kernels behind ``surr_*`` in include/lbm.h) maps
(n, Eo, log10 Mo, density ratio, viscosity ratio) to (log U_t, log C_D).  Its
training data are terminal states computed by the batched lattice Boltzmann
solver (``lbm_batch_*``); its answer is used only when the input lies inside
the box of the training inputs and the ensemble agrees within ``max_spread``;
otherwise the case is solved directly.  This module only orchestrates: every
time step and every network evaluation runs in the CUDA library.

Terminal state (reading of Sec. 4.2-4.3, which gives no criterion): the rise
velocity of Eq. 43 averaged over windows of ``window`` steps changes by less
than ``rtol`` of itself between two consecutive windows, or the centroid has
come within 1.5 diameters of the top wall, or ``max_steps`` is reached (then
the case is reported as not converged).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs, lbm


def features(params: dict, meta: dict) -> np.ndarray:
    """(n, Eo, log10 Mo, density ratio, viscosity ratio k / eta_gas), with
    eta_gas = rho_gas cs^2 tau_gas."""
    rho_l, rho_g = params["rho"][0], params["rho"][2]
    eta_g = rho_g * params["tau"][2] / 3.0
    return np.array([meta["n"], meta["Eo"], meta["log10_Mo"], rho_l / rho_g, params["pl_k"] / eta_g])


def run_to_terminal(cases, window=1000, rtol=2e-3, max_steps=30000, stream=None, device="cuda"):
    """Advances cases [(params, discs, meta), ...] together until each reaches
    its terminal state.  Returns per-case dicts with U_t, C_D, steps,
    converged, finite, and the wall time."""
    batch = lbm.Batch([c[0] for c in cases], device=device, stream=stream)
    for i, (p, b, _) in enumerate(cases):
        batch.case(i).set_fields(inputs.bubble_fields(p["nx"], p["ny"], 2, p["xi"], b, seed=i, noise=1e-8))
    batch.autotune(reps=2)
    n = len(cases)
    done = [False] * n
    out = [dict(U_t=math.nan, C_D=math.nan, steps=0, converged=False, finite=True) for _ in range(n)]
    hist = [[] for _ in range(n)]
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps and not all(done):
        try:
            batch.step(window)
        except lbm.LbmError as err:
            if err.status != -4:
                raise
        steps += window
        for i in range(n):
            if done[i]:
                continue
            ob = batch.case(i).observables()
            v, y = ob["rise_velocity"], ob["centroid"][1]
            if not (np.isfinite(v) and np.isfinite(y)):
                out[i].update(finite=False, steps=steps)
                done[i] = True
                batch.set_active(i, False)
                continue
            hist[i].append(v)
            p = cases[i][0]
            top = p["ny"] - 1.5 * 2.0 * cases[i][1][0][2]
            steady = (len(hist[i]) >= 3 and abs(hist[i][-1] - hist[i][-2]) < rtol * abs(hist[i][-1])
                      and abs(hist[i][-2] - hist[i][-3]) < rtol * abs(hist[i][-2]))
            if steady or y > top or steps >= max_steps:
                out[i].update(U_t=v, C_D=ob["drag_coefficient"], steps=steps, converged=bool(steady or y > top))
                done[i] = True
                batch.set_active(i, False)
    wall = time.perf_counter() - t0
    return out, wall


class TerminalStateModel:
    """Ensemble surrogate with hull and agreement checks and solver fallback."""

    def __init__(self, members=5, seed=0, max_rows=4096, max_batch=512, max_spread=0.05):
        self.net = lbm.Surrogate(inputs.mlp_init(members, seed=seed), max_batch=max_batch, max_rows=max_rows)
        self.max_spread = max_spread

    def fit(self, X, U_t, C_D, epochs=400, batch=128, lr=2e-3, seed=0):
        Y = np.stack([np.log(U_t), np.log(C_D)], axis=1)
        return self.net.train(np.asarray(X, dtype=np.float64), Y, epochs=epochs, batch=batch, lr=lr, seed=seed)

    def predict(self, X):
        """(U_t, C_D, trusted) per row: trusted means inside the training box
        and an ensemble spread below max_spread in both outputs (relative)."""
        mean, spread, outside = self.net.predict(np.asarray(X, dtype=np.float64))
        U, CD = np.exp(mean[:, 0]), np.exp(mean[:, 1])
        # spread of log values = relative spread of the values
        trusted = (~outside) & (spread[:, 0] < self.max_spread) & (spread[:, 1] < self.max_spread)
        return U, CD, trusted

    def answer(self, cases, **run_kw):
        """Terminal states of cases: the network where trusted, the solver
        elsewhere.  Returns (U_t, C_D, used_solver, wall seconds)."""
        X = np.stack([features(p, m) for p, _, m in cases])
        t0 = time.perf_counter()
        U, CD, trusted = self.predict(X)
        fallback = [c for c, t in zip(cases, trusted) if not t]
        if fallback:
            res, _ = run_to_terminal(fallback, **run_kw)
            j = 0
            for i, t in enumerate(trusted):
                if not t:
                    U[i], CD[i] = res[j]["U_t"], res[j]["C_D"]
                    j += 1
        return U, CD, ~trusted, time.perf_counter() - t0
