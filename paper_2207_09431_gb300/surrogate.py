"""Surrogate of the rising-bubble terminal state, with the solver as fallback.

The network (CUDA kernels behind ``surr_*`` in include/lbm.h) maps
(n, Eo, log10 Mo, density ratio, log10 viscosity ratio) to (log U_t, log C_D).  Its
training data are terminal states computed by the batched lattice Boltzmann
solver (``lbm_batch_*``); its answer is used only when the input lies inside
the box of the training inputs, the ensemble agrees within ``max_spread`` and
the training cases nearest to the input were predicted within ``local_max``
when held out (cross validation); otherwise the case is solved directly.  This module only orchestrates: every
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
    """(n, Eo, log10 Mo, density ratio, log10 of the viscosity ratio
    k / eta_gas), with eta_gas = rho_gas cs^2 tau_gas (k spans decades over
    the Mo range)."""
    rho_l, rho_g = params["rho"][0], params["rho"][2]
    eta_g = rho_g * params["tau"][2] / 3.0
    return np.array([meta["n"], meta["Eo"], meta["log10_Mo"], rho_l / rho_g,
                     math.log10(params["pl_k"] / eta_g)])


def run_to_terminal(cases, window=2000, rtol=0.05, max_steps=40000, stream=None, device="cuda", persistent=False):
    """Advances cases [(params, discs, meta), ...] together until each reaches
    its terminal state (lbm_batch_run: the rise velocity measured as the
    centroid displacement per window, Eq. 44, because the instantaneous value
    oscillates with the bubble shape).  Returns per-case dicts with U_t, C_D
    (Eq. 37 at U_t), steps, converged and finite, and the wall time."""
    batch = lbm.Batch([c[0] for c in cases], device=device, stream=stream)
    if persistent:
        batch.set_persistent(True)
    for i, (p, b, _) in enumerate(cases):
        batch.case(i).set_fields(inputs.bubble_fields(p["nx"], p["ny"], 2, p["xi"], b, seed=i, noise=1e-8))
    t0 = time.perf_counter()  # lbm_batch_run tunes the launch configuration itself
    res = batch.run(window=window, rtol=rtol, max_steps=max_steps, top_margin=1.5)
    wall = time.perf_counter() - t0
    out = []
    for r in res:
        finite = r["outcome"] != "diverged"
        out.append(dict(U_t=r["rise_velocity"] if finite else math.nan,
                        C_D=r["drag_coefficient"] if finite else math.nan, steps=r["steps_run"],
                        converged=r["outcome"] in ("terminal", "top"), finite=finite, outcome=r["outcome"]))
    return out, wall


class TerminalStateModel:
    """Ensemble surrogate with hull, agreement and local-residual checks and
    solver fallback.

    Local residual: the ensemble is also trained with `folds`-fold cross
    validation on its own training set (surr_train_cv), and a case is trusted
    only where the `local_k` training cases nearest to it were all predicted
    within `local_max` (in log U_t and log C_D) when held out.  The labels are
    terminal states under a stopping rule, and near some inputs they scatter
    by more than the network's error; the members then agree with each other
    and only held-out residuals reveal it."""

    def __init__(self, members=5, seed=0, max_rows=4096, max_batch=512, max_spread=0.05, local_k=8,
                 local_max=0.03):
        self.init = inputs.mlp_init(members, seed=seed)
        self.net = lbm.Surrogate(self.init, max_batch=max_batch, max_rows=max_rows)
        self.max_spread = max_spread
        self.local_k, self.local_max = local_k, local_max
        self.cv = False

    def fit(self, X, U_t, C_D, epochs=400, batch=128, lr=2e-3, seed=0, folds=5):
        Y = np.stack([np.log(U_t), np.log(C_D)], axis=1)
        X = np.asarray(X, dtype=np.float64)
        self.cv = folds > 1
        if self.cv:
            loss = self.net.train_cv(X, Y, folds, epochs, batch, lr, seed, self.init)
        else:
            loss = self.net.train(X, Y, epochs=epochs, batch=batch, lr=lr, seed=seed)
        self.net.set_local_trust(self.local_k, self.local_max if self.cv else 0.0)
        return loss

    def predict(self, X, local=True):
        """(U_t, C_D, trusted) per row: trusted means inside the training box,
        no member farther than max_spread from the ensemble mean in either
        output (relative: the outputs are logarithms) and, after a
        cross-validated fit (unless local=False), a local residual below
        local_max."""
        X = np.asarray(X, dtype=np.float64)
        mean, spread, outside = self.net.predict(X)
        U, CD = np.exp(mean[:, 0]), np.exp(mean[:, 1])
        trusted = (~outside) & (spread[:, 0] < self.max_spread) & (spread[:, 1] < self.max_spread)
        if local and self.cv and self.local_max > 0:
            trusted &= self.net.local_residual(X, self.local_k) < self.local_max
        return U, CD, trusted

    def answer(self, cases, max_steps=40000, window=2000, rtol=0.05, stream=None):
        """Terminal states of cases: the network where trusted, the solver
        elsewhere, both inside the library (surr_answer).  Returns (U_t, C_D,
        used_solver, wall seconds)."""
        X = np.stack([features(p, m) for p, _, m in cases])
        t0 = time.perf_counter()
        y, used, _ = self.net.answer(X, [p for p, _, _ in cases], [b[0] for _, b, _ in cases],
                                     max_spread=self.max_spread, window=window, rtol=rtol, max_steps=max_steps)
        return y[:, 0], y[:, 1], used, time.perf_counter() - t0


def evaluate(n_train=1024, n_test=128, grid=(100, 200), members=5, epochs=1000, max_steps=30000, seed=1000,
             test_seed=9000, stream=None, max_spread=0.05, return_model=False, density_ratio=100.0):
    """Trains on solver terminal states of n_train seeded cases and judges the
    network on n_test held-out cases solved in full.  Returns a summary dict:
    C_D error of the network on every converged test case and on the trusted
    ones, the fallback count, and the time to answer with and without the
    network (and the trained model if return_model)."""
    train = inputs.ensemble_cases(n_train, seed=seed, grids=(grid,), density_ratio=density_ratio)
    res, wall_train = run_to_terminal(train, max_steps=max_steps, stream=stream)
    keep = [i for i, r in enumerate(res) if r["finite"] and r["converged"] and r["U_t"] > 0 and r["C_D"] > 0]
    X = np.stack([features(train[i][0], train[i][2]) for i in keep])
    U = np.array([res[i]["U_t"] for i in keep])
    CD = np.array([res[i]["C_D"] for i in keep])
    model = TerminalStateModel(members=members, seed=seed, max_rows=max(len(keep), 1), max_batch=512,
                               max_spread=max_spread)
    loss = model.fit(X, U, CD, epochs=epochs)
    test = inputs.ensemble_cases(n_test, seed=test_seed, grids=(grid,), density_ratio=density_ratio)
    ref, wall_solver = run_to_terminal(test, max_steps=max_steps, stream=stream)
    Xt = np.stack([features(p, m) for p, _, m in test])
    t0 = time.perf_counter()
    Up, CDp, trusted = model.predict(Xt)
    wall_net = time.perf_counter() - t0
    _, _, trusted_spread = model.predict(Xt, local=False)
    ok = np.array([r["finite"] and r["converged"] and r["U_t"] > 0 for r in ref])
    judged = trusted & ok
    cd_ref = np.array([r["C_D"] for r in ref])
    err = np.abs(CDp[judged] / cd_ref[judged] - 1.0)
    err_all = np.abs(CDp[ok] / cd_ref[ok] - 1.0)
    js = trusted_spread & ok
    err_spread = np.abs(CDp[js] / cd_ref[js] - 1.0)
    summary = {
        "train_cases": n_train, "train_converged": len(keep), "train_solver_s": round(wall_train, 2),
        "final_loss": loss, "test_cases": n_test, "test_converged": int(ok.sum()),
        "trusted": int(trusted.sum()), "judged": int(judged.sum()),
        "cd_rel_err_median": float(np.median(err)) if err.size else None,
        "cd_rel_err_p90": float(np.percentile(err, 90)) if err.size else None,
        "cd_within_5pct": float(np.mean(err < 0.05)) if err.size else None,
        "cd_rel_err_max": float(np.max(err)) if err.size else None,
        "trust_rule": f"inside the training box, members within {max_spread:g} of the mean, the "
                      f"{model.local_k} nearest training cases predicted within {model.local_max:g} out of fold",
        "trusted_spread_only": int(trusted_spread.sum()), "judged_spread_only": int(js.sum()),
        "cd_within_5pct_spread_only": float(np.mean(err_spread < 0.05)) if err_spread.size else None,
        "cd_rel_err_max_spread_only": float(np.max(err_spread)) if err_spread.size else None,
        "cd_rel_err_median_all_converged": float(np.median(err_all)) if err_all.size else None,
        "cd_rel_err_p90_all_converged": float(np.percentile(err_all, 90)) if err_all.size else None,
        "solver_s_for_test": round(wall_solver, 3), "network_s_for_test": round(wall_net, 5),
        "speedup_trusted": round(wall_solver / max(wall_net, 1e-9), 1),
    }
    return (summary, model) if return_model else summary
