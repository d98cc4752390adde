"""Parity with the FP64 oracle at density ratio 1000 on the paper's bubble.

The set-up is case 6 of Table 5 (Sec. 4.3: n = 0.8, k = 1e-2, g = 5e-7,
sigma = 2.61e-5, d = 50 on 200 x 400), run at density ratio 1000 instead of the
paper's 800.  Small bubbles (R <= 20 lattice units) diverge at that ratio under
the printed scheme; the paper-size bubble is stable for 150,000 steps.

1. Fields after 1000 steps: per field, relative L2 within max(1e-5, 2 x the
   deviation of the FP32 build of the oracle), the floor measured live.
2. Terminal velocity: the oracle's rises to their terminal states are stored in
   tests/golden/oracle_terminal_table5_case6_r1000.json and
   oracle_terminal_table5_case4_r1000.json (case 4: n = 0.6, k = 5e-4,
   g = 2e-7; written by tests/golden/make_oracle_terminal.py, which calls only
   the oracle); the CUDA path run from the same FP32-rounded fields must give
   the window-averaged rise velocity (centroid displacement over 2000 steps,
   Eq. 44) and drag coefficient (Eq. 37) at the oracle's terminal step, and
   meet the terminal criterion there too.  Case 6 is held to 0.5 %.  Case 4,
   the slowest rise (46,000 steps), is held to the deviation of the same
   oracle source built with FP32 internals (the *_f32.json goldens): that
   build loses 1.4 % of the gas area by its terminal step and ends 3.4 % off
   in U_t, so 0.5 % is below what FP32 arithmetic fixes for this case.  In
   both cases the CUDA path's drift of the gas area must stay within that of
   the FP32 build.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2207_09431_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "oracle_terminal_table5_case{}_r1000.json")


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_09431_gb300 import lbm as _lbm

    _lbm.load_library()
    return _lbm


def _case(case=6):
    p, discs = inputs.table5_case(case, density_ratio=1000.0)
    C = inputs.round_to_fp32(inputs.bubble_fields(p["nx"], p["ny"], 2, p["xi"], discs, seed=0, noise=1e-8))
    return p, C


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12 * b.size))


def test_fields_after_1000_steps_at_density_ratio_1000(lbm):
    p, C = _case()
    lat = lbm.Lattice(p)
    lat.set_fields(C)
    lat.step(1000)
    o64, o32 = oracle.Oracle(p, "f64-omp"), oracle.Oracle(p, "f32-omp")
    for o in (o64, o32):
        o.set_fields(C)
        o.step(1000)
    bad = {}
    for name in ("C1", "p", "ux", "uy", "tau", "g", "h"):
        ref = o64.field(name)
        err, floor = relerr(lat.field(name), ref), relerr(o32.field(name), ref)
        print(f"{name}: gpu {err:.2e}  fp32 floor {floor:.2e}  ratio {err / max(floor, 1e-30):.2f}")
        if not err <= max(1e-5, 2.0 * floor):
            bad[name] = (err, floor)
    assert not bad, bad


def _fp32_floor(case, gold):
    """Relative deviation of the FP32-internal oracle's terminal U_t and C_D."""
    g32 = json.load(open(GOLDEN.format(case).replace(".json", "_f32.json")))
    return abs(g32["U_t"] / gold["U_t"] - 1.0), abs(g32["C_D"] / gold["C_D"] - 1.0), g32


@pytest.mark.parametrize("case", [6, 4])
def test_terminal_velocity_matches_oracle(lbm, case):
    gold = json.load(open(GOLDEN.format(case)))
    fU, fCD, g32 = _fp32_floor(case, gold)
    tol_U, tol_CD = (0.005, 0.005) if case == 6 else (fU, fCD)
    p, C = _case(case)
    lat = lbm.Lattice(p)
    lat.set_fields(C)
    every, window = gold["every"], gold["window"]
    steps, ybar, area, raw = [], [], [], None
    while lat.observables()["step"] < gold["terminal_step"]:
        lat.step(every)
        ob = lat.observables()
        steps.append(ob["step"])
        ybar.append(ob["centroid"][1])
        area.append(ob["area"])
        raw = np.array(ob["raw"])
    assert steps == gold["steps"]
    k = window // every
    u_gpu = np.diff(np.asarray(ybar)[k - 1::k]) / window
    u_orc = np.diff(np.asarray(gold["ybar"])[k - 1::k]) / window
    U_t = float(u_gpu[-1])
    raw[10] = U_t * raw[6]
    C_D = lbm.lbm_postprocess(p, raw)["drag_coefficient"]
    n32 = min(len(g32["area"]), len(area))
    print(f"case {case}: U_t gpu {U_t:.6e} oracle {gold['U_t']:.6e} ({U_t / gold['U_t'] - 1:+.2e}, "
          f"fp32 floor {fU:.2e}); C_D gpu {C_D:.4f} oracle {gold['C_D']:.4f} ({C_D / gold['C_D'] - 1:+.2e}, "
          f"fp32 floor {fCD:.2e}); largest window difference {np.max(np.abs(u_gpu / u_orc - 1)):.2e}; "
          f"gas area change at step {steps[n32 - 1]}: gpu {area[n32 - 1] / gold['area'][0] - 1:+.2e}, "
          f"fp32 oracle {g32['area'][n32 - 1] / gold['area'][0] - 1:+.2e}")
    assert abs(U_t / gold["U_t"] - 1.0) < tol_U
    assert abs(C_D / gold["C_D"] - 1.0) < tol_CD
    # the gas area drifts in FP32 (FP64 keeps it to 1e-10); the CUDA path must
    # keep it at least as well as the FP32 build of the oracle
    assert abs(area[n32 - 1] / gold["area"][0] - 1.0) <= abs(g32["area"][n32 - 1] / gold["area"][0] - 1.0)
    # the terminal criterion holds at the oracle's terminal window
    rtol = 0.01

    def terminal(u):
        return len(u) >= 3 and all(abs(u[-j] - u[-j - 1]) < rtol * abs(u[-j]) for j in (1, 2))

    assert terminal(u_gpu)
