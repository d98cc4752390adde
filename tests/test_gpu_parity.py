"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Both sides start from the same seeded input fields, rounded to FP32 so that the
starting states agree exactly; each builds its own populations.  Tolerance:
relative L2 <= 1e-5 on fields and populations (FP32 arithmetic against FP64),
with the denominator max(||ref||, 1e-12 N).
"""
import numpy as np
import pytest

import oracle
from paper_2207_09431_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12 * b.size))


@pytest.fixture(scope="module")
def lbm():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2207_09431_gb300 import lbm as _lbm

    _lbm.load_library()
    return _lbm


def _pair(lbm, p, C):
    lat = lbm.Lattice(p)
    lat.set_fields(C)
    orc = oracle.Oracle(p)
    orc.set_fields(C)
    return lat, orc


def _compare(lat, orc, names=("C1", "p", "ux", "uy", "tau", "g", "h"), tol=TOL):
    errs = {}
    for name in names:
        errs[name] = relerr(lat.field(name), orc.field(name))
    print("parity", {k: f"{v:.2e}" for k, v in errs.items()})
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"parity failures {bad} (all: {errs})"
    return errs


def _bubble_case(nx, ny, mobility=0, fd_scheme=0, ratio=100.0, R=8.0, seed=1):
    p, _ = inputs.small_case(mobility=mobility, density_ratio=ratio)
    p = dict(p, nx=nx, ny=ny, fd_scheme=fd_scheme)
    C = inputs.round_to_fp32(inputs.bubble_fields(nx, ny, 2, p["xi"], [(nx / 2, ny / 3, R, 3)], seed=seed,
                                                  noise=1e-8))
    return p, C


def test_initial_equilibria(lbm):
    """The state after set_fields (populations, tau, C).  The velocity read
    back at t = 0 is a cancellation of two O(F) terms and is not compared."""
    p, C = _bubble_case(50, 70)
    lat, orc = _pair(lbm, p, C)
    _compare(lat, orc, names=("C1", "tau", "g", "h"), tol=1e-6)


@pytest.mark.parametrize("nx,ny", [(50, 70), (64, 128), (33, 45)])
def test_ten_steps_ragged(lbm, nx, ny):
    p, C = _bubble_case(nx, ny, R=min(nx, ny) / 5)
    lat, orc = _pair(lbm, p, C)
    lat.step(10)
    orc.step(10)
    _compare(lat, orc)


@pytest.mark.parametrize("mobility,fd_scheme", [(1, 0), (0, 1), (1, 1)])
def test_variants_100_steps(lbm, mobility, fd_scheme):
    p, C = _bubble_case(48, 80, mobility=mobility, fd_scheme=fd_scheme)
    lat, orc = _pair(lbm, p, C)
    lat.step(100)
    orc.step(100)
    _compare(lat, orc)
    sv = lat.field("SV")
    svo = orc.field("S") + orc.field("V")
    assert relerr(sv, svo) < 1e-4


def test_small_rising_bubble_1000_steps(lbm):
    """64 x 128 rising bubble (R = 10, Eo = 10, n = 0.7, power law): fields and
    populations after 1000 steps."""
    p, b = inputs.small_case(mobility=0)
    C = inputs.round_to_fp32(inputs.bubble_fields(64, 128, 2, p["xi"], b, seed=0, noise=1e-8))
    lat, orc = _pair(lbm, p, C)
    lat.step(1000)
    orc.step(1000)
    _compare(lat, orc)
    og, oo = lat.observables(), orc.observables()
    assert abs(og["rise_velocity"] - oo["rise_velocity"]) <= 5e-3 * abs(oo["rise_velocity"]) + 1e-9
    assert abs(og["centroid"][1] - oo["centroid"][1]) < 1e-4
    for i in (0, 2):
        assert abs(og["mass"][i] - oo["mass"][i]) < 1e-5 * oo["mass"][i]


def test_three_components_periodic(lbm):
    p, b = inputs.three_comp_case(nx=64, mobility=0, seed=3)
    C = inputs.round_to_fp32(inputs.bubble_fields(64, 64, 3, p["xi"], b, seed=3, noise=1e-8, periodic_y=True))
    lat, orc = _pair(lbm, p, C)
    lat.step(200)
    orc.step(200)
    _compare(lat, orc, names=("C1", "C2", "p", "ux", "uy", "tau", "g", "h"))


def test_init_bubbles_matches_oracle(lbm):
    p, b = inputs.small_case()
    lat = lbm.Lattice(p)
    lat.init_bubbles(b, seed=7, noise=1e-8)
    orc = oracle.Oracle(p)
    orc.init_bubbles([list(x) for x in b], seed=7, noise=1e-8)
    assert np.max(np.abs(lat.field("C1") - orc.field("C1"))) < 1e-7
    assert relerr(lat.field("g"), orc.field("g")) < 1e-5


def test_observables_match_oracle(lbm):
    p, C = _bubble_case(64, 96)
    lat, orc = _pair(lbm, p, C)
    lat.step(50)
    orc.step(50)
    og, oo = lat.observables(), orc.raw_observables()
    raw = np.array(og["raw"])
    assert np.allclose(raw[:11], oo[:11], rtol=1e-5, atol=1e-9)
    assert np.array_equal(raw[11:], oo[11:])


def test_checkpoint_resume_bit_identical(lbm, tmp_path):
    p, C = _bubble_case(40, 60)
    a = lbm.Lattice(p)
    a.set_fields(C)
    a.step(20)
    path = str(tmp_path / "ck.bin")
    a.save(path)
    a.step(15)
    b = lbm.Lattice(p)
    b.load(path)
    b.step(15)
    for name in ("g", "h", "tau"):
        assert np.array_equal(a.field(name), b.field(name))


def test_divergence_is_reported(lbm):
    """A non-finite state is caught by the watchdog (injected on the host)."""
    p, C = _bubble_case(32, 48)
    C = C.copy()
    C[0, 10, 10] = np.nan
    lat = lbm.Lattice(p)
    lat.set_fields(C)
    with pytest.raises(lbm.LbmError) as ei:
        lat.step(2)
    assert ei.value.status == -4


def test_full_size_windows_one_step(lbm):
    """Bench workload (2048 x 4096 rising bubble) in the launch configuration the
    benchmark times: after one step, nodes at least 5 lattice units inside
    windows of the seeded input agree with the oracle run on those windows
    (the step reads at most 4 nodes away)."""
    p, b = inputs.sweep_case(2048)
    nx, ny = p["nx"], p["ny"]
    Cfull = inputs.round_to_fp32(inputs.bubble_fields(nx, ny, 2, p["xi"], b, seed=0, noise=1e-8))
    lat = lbm.Lattice(p)
    lat.set_fields(Cfull)
    lat.step(1)
    fields = {n: lat.field(n) for n in ("C1", "p", "uy", "tau")}
    cx, cy, R, _ = b[0]
    W = 48
    windows = [(int(cx + R) - W // 2, 0), (int(cx) - W // 2, int(cy - R) - W // 2), (0, int(cy) - W // 2)]
    m = 5
    for (x0, y0) in windows:
        x0 = max(0, min(nx - W, x0))
        y0 = max(0, min(ny - W, y0))
        pw = dict(p, nx=W, ny=W)
        orc = oracle.Oracle(pw)
        orc.set_fields(Cfull[:, y0:y0 + W, x0:x0 + W])
        orc.step(1)
        ylo = 0 if y0 == 0 else m   # the real bottom wall is inside the window
        for n in ("C1", "p", "uy", "tau"):
            got = fields[n][y0 + ylo:y0 + W - m, x0 + m:x0 + W - m]
            want = orc.field(n)[ylo:W - m, m:W - m]
            assert relerr(got, want) < TOL, (n, x0, y0)


@pytest.mark.parametrize("mobility", [0, 1])
def test_collapsed_state_form(lbm, mobility):
    """State holding C_i instead of h^i: same fields as the oracle, and the same
    as the population form up to FP32 summation order."""
    p, C = _bubble_case(56, 90, mobility=mobility)
    pc = dict(p, collapse_h=1)
    lat = lbm.Lattice(pc)
    lat.set_fields(C)
    full = lbm.Lattice(p)
    full.set_fields(C)
    orc = oracle.Oracle(p)
    orc.set_fields(C)
    lat.step(300)
    full.step(300)
    orc.step(300)
    _compare(lat, orc, names=("C1", "p", "ux", "uy", "tau", "g"))
    for name in ("C1", "p", "uy", "tau", "g"):
        assert relerr(lat.field(name), full.field(name)) < 1e-6, name
    with pytest.raises(lbm.LbmError):
        lat.field("h")
