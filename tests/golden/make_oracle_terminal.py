"""Writes oracle_terminal_table5_case<C>_r<R>.json: the rise of a Table 5 bubble
(Sec. 4.3; d = 50 on 200 x 400; case 6 by default: n = 0.8, k = 1e-2, g = 5e-7,
sigma = 2.61e-5) at density ratio R (1000 by default), computed by the FP64
oracle from the seeded initial fields rounded to FP32, up to its terminal
state.

Terminal state (the paper gives no criterion): the rise velocity averaged over
windows of 2000 steps (centroid displacement, Eq. 44) changes by less than 1 %
of itself between two consecutive pairs of windows.  Recorded every 1000 steps:
the gas area, the centroid (Eq. 44) and the mean velocity (Eq. 43); at the
terminal step the window-averaged rise velocity U_t and the drag coefficient of
Eq. 37 from it (oracle post-processing).

With a third argument "f32" it runs the same oracle source built with FP32
internals (the FP32 rounding floor of the scheme) and writes
oracle_terminal_table5_case<C>_r<R>_f32.json.

Calls only the oracle and the input generators.  Run from the repository root:
    python tests/golden/make_oracle_terminal.py [case] [density ratio] [f32]
(case 6: 5 minutes on 6 host cores with the OpenMP build of the oracle, which
gives the serial build's results bit for bit; case 4 needs twice the steps).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2207_09431_gb300 import inputs  # noqa: E402

CASE = int(sys.argv[1]) if len(sys.argv) > 1 else 6
RATIO = float(sys.argv[2]) if len(sys.argv) > 2 else 1000.0
EVERY, WINDOW, RTOL, MAX_STEPS = 1000, 2000, 0.01, 80000
PREC = "f32" if len(sys.argv) > 3 and sys.argv[3] == "f32" else "f64"
OUT = os.path.join(HERE, f"oracle_terminal_table5_case{CASE}_r{RATIO:g}" + ("_f32" if PREC == "f32" else "") + ".json")


def window_velocities(steps, ys):
    """Centroid displacement per step over consecutive windows of WINDOW steps."""
    k = WINDOW // EVERY
    ws = np.asarray(steps)[k - 1::k]
    yw = np.asarray(ys)[k - 1::k]
    return ws[1:], np.diff(yw) / WINDOW


def terminal(u):
    return len(u) >= 3 and all(abs(u[-j] - u[-j - 1]) < RTOL * abs(u[-j]) for j in (1, 2))


def main():
    p, discs = inputs.table5_case(CASE, density_ratio=RATIO)
    C = inputs.round_to_fp32(inputs.bubble_fields(p["nx"], p["ny"], 2, p["xi"], discs, seed=0, noise=1e-8))
    o = oracle.Oracle(p, PREC + "-omp")
    o.set_fields(C)
    steps, area, ybar, vbar = [], [], [], []
    t0 = time.time()
    U_t, step_t = None, None
    while o.step_count < MAX_STEPS:
        o.step(EVERY)
        raw = o.raw_observables()
        steps.append(o.step_count)
        area.append(raw[6])
        ybar.append(raw[8] / raw[6])
        vbar.append(raw[10] / raw[6])
        if len(steps) % (WINDOW // EVERY) == 0:
            ws, u = window_velocities(steps, ybar)
            print(f"step {o.step_count}: ybar {ybar[-1]:.4f}  U(window) {u[-1] if len(u) else float('nan'):.6e}  "
                  f"{time.time() - t0:.0f} s", flush=True)
            if terminal(u):
                U_t, step_t = float(u[-1]), int(ws[-1])
                raw = np.array(raw)
                raw[10] = U_t * raw[6]
                post = oracle.postprocess(o.params, raw)
                break
    if U_t is None:
        raise SystemExit("no terminal state within MAX_STEPS")
    doc = {
        "source": ("FP64 oracle" if PREC == "f64" else "the oracle source built with FP32 internals")
                  + " (oracle/lbm_oracle.c) run by tests/golden/make_oracle_terminal.py",
        "case": f"Table 5 case {CASE} (Sec. 4.3) at density ratio {RATIO:g}, constant mobility, 200 x 400, "
                "bubble d = 50 at (100, 120), seeded noise 1e-8 (seed 0), fields rounded to FP32",
        "terminal_rule": f"windows of {WINDOW} steps, relative change < {RTOL} between two consecutive pairs",
        "every": EVERY, "window": WINDOW, "steps": steps, "area": area, "ybar": ybar, "vbar": vbar,
        "terminal_step": step_t, "U_t": U_t, "C_D": post["drag_coefficient"], "Re": post["Re"],
        "wall_s": round(time.time() - t0, 1),
    }
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", OUT, "U_t", U_t, "at step", step_t)


if __name__ == "__main__":
    main()
