"""Three-component experiment of Sec. 3.1: constant against variable mobility.

256 x 256 fully periodic lattice, power-law matrix (component 1, n = 0.6),
two droplets of component 2 (R = 20 and 12) and a bubble of component 3
(R = 6) at seeded non-overlapping centres, pairwise sigma 1e-3, no gravity,
20,000 steps; the masses M_i and the thresholded masses M_i^{>0.5} (sum of C_i
over nodes with C_i > 0.5) summed in FP64 on the GPU every 100 steps.

The paper reports that the constant mobility dissipates the interfaces and
loses mass gradually while the variable one keeps each component (Sec. 3.1).
Measured here: the droplets of component 2 keep 98 % of their thresholded mass
with the variable mobility and 86 % with the constant one; the R = 6 bubble of
component 3 (1.5 interface widths) dissolves below C = 0.5 under both within
about 5,200 steps.  Parity of the three-component step with both mobilities
against the FP64 oracle is in test_gpu_parity.py.
"""
import numpy as np
import pytest

from paper_2207_09431_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def runs():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_09431_gb300 import lbm

    out = {}
    for mob in (0, 1):
        p, discs = inputs.three_comp_case(nx=256, mobility=mob, seed=0)
        lat = lbm.Lattice(p)
        lat.set_fields(inputs.bubble_fields(256, 256, 3, p["xi"], discs, seed=0, noise=1e-8, periodic_y=True))
        rows = []
        for _ in range(201):
            ob = lat.observables()
            rows.append([ob["step"]] + list(ob["mass"]) + list(ob["mass_thr"]))
            if ob["step"] < 20000:
                lat.step(100)
        out[mob] = np.array(rows)
    return out


def test_variable_mobility_keeps_the_droplets_thresholded_mass(runs):
    const, var = runs[0], runs[1]
    assert const[-1, 0] == var[-1, 0] == 20000
    keep_const = const[-1, 5] / const[0, 5]
    keep_var = var[-1, 5] / var[0, 5]
    print(f"component 2 above 0.5: constant {keep_const:.4f}, variable {keep_var:.4f} of the initial mass")
    assert keep_var > keep_const + 0.05
    # constant mobility loses it gradually: the thresholded mass falls at every
    # 2000-step checkpoint after the first
    assert np.all(np.diff(const[20::20, 5]) < 0)


def test_masses_and_the_small_bubble(runs):
    const, var = runs[0], runs[1]
    # the constant mobility conserves each transported component (FP32 sums
    # over 20,000 steps drift by a few parts in 1e5)
    for i in (1, 2):
        assert abs(const[-1, i] / const[0, i] - 1.0) < 1e-4
    # the variable mobility's split form is not a discrete divergence: its mass
    # moves with the summed sources, here by less than 0.5 %
    assert abs(var[-1, 2] / var[0, 2] - 1.0) < 5e-3
    # the R = 6 bubble of component 3 dissolves below C = 0.5 under both
    for r in (const, var):
        zero = r[r[:, 6] == 0.0, 0]
        assert zero.size and zero[0] <= 8000 and np.all(r[r[:, 0] >= zero[0], 6] == 0.0)
