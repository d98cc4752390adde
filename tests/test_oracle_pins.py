"""Pins of the FP64 oracle against things other than itself (arXiv 2207.09431).

Closed forms (power-law channel, hydrostatics, Laplace law, the modified
equation of the flat interface), conservation invariants, special cases, an
independent brute-force NumPy stepper on tiny grids, and values printed in the
paper's tables.  None of these runs on a GPU.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import channel_closed_form as ccf
import handstep_numpy as hs
from oracle import observables as obs
from paper_2207_09431_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _single_phase(nx, ny, **kw):
    p = dict(nx=nx, ny=ny, ncomp=2, rho=(1.0, 1.0, 1.0), tau=(0.8, 0.8, 0.8))
    p.update(kw)
    o = oracle.Oracle(p)
    o.set_fields(np.ones((1, ny, nx)))
    return o


# ------------------------------------------------------------------ P1
@pytest.mark.parametrize("n", [0.5, 0.8, 1.0, 1.5])
def test_powerlaw_channel_closed_form(n):
    """Sec. 3.2 / Eq. 34: body-force driven power-law channel between walls.

    Force balance k |du/dy|^n = F |y| gives u(y) = n/(n+1) (F/k)^(1/n)
    (H^((n+1)/n) - |y|^((n+1)/n)), the paper's profile with u_in its mean.
    Pins Eq. 25-33 (strain rate from the non-equilibrium part, power-law tau)."""
    table = _golden("paper_table2_channel.json")
    bound = dict(zip(table["n"], table["E_rel"]))[n]
    Ny, H, umax = 60, 30.0, 0.02
    r = (umax * (n + 1) / n / H ** ((n + 1) / n)) ** n   # F / k
    k = 0.8 / 3.0 / (r * H) ** ((n - 1.0) / n)             # tau = 0.8 at the wall
    F = r * k
    o = _single_phase(2, Ny, powerlaw=1, pl_n=n, pl_k=k, tau_min=0.02, tau_max=20.0, force_x=F)
    prev = None
    for _ in range(200):
        o.step(500)
        u = o.field("ux")[:, 0]
        # steady-state criterion in the spirit of Sec. 3.3
        if prev is not None and np.linalg.norm(u - prev) / np.linalg.norm(u) < 1e-9:
            break
        prev = u
    y = np.arange(Ny) + 0.5 - H
    ua = n / (n + 1) * (F / k) ** (1 / n) * (H ** ((n + 1) / n) - np.abs(y) ** ((n + 1) / n))
    err = np.linalg.norm(u - ua) / np.linalg.norm(ua)          # Eq. 35
    assert err <= bound
    # the strain rate the method computes locally vs |du/dy| of the closed form
    gd = o.field("shear")[:, 0]
    gda = (F * np.abs(y) / k) ** (1 / n)
    away = np.abs(y) > 5
    assert np.max(np.abs(gd[away] - gda[away]) / gda[away]) < 0.02


# ------------------------------------------------------------------ P1b
@pytest.mark.parametrize("n,tau_in", [(0.5, 0.8), (1.0, 0.24), (1.0, 0.8), (1.5, 0.8)])
def test_layered_two_phase_channel_closed_form(n, tau_in):
    """Sec. 3.3: two fluids in layers (power-law inside, Newtonian outside,
    equal densities, flat diffuse interfaces) driven by a body force.

    (a) Momentum balance: the steady velocity equals the profile that balances
    the force for the viscosity eta = tau / 3 the method holds at each node
    (to quadrature accuracy; the n = 0.5 case, whose tau varies like 1/|y|
    towards its clamp at the centreline, to 2 %).  (b) Where both fluids have
    the same viscosity at the interface, the sharp-interface closed form holds
    within the largest relative error Table 3 prints for the same inner index.
    With a viscosity jump (tau_in = 0.24, lambda = 0.3) the diffuse interface
    itself shifts the profile (7.8 % at H = 25, 4.7 % at H = 50 with the linear
    mixture law of tau), so (b) is not applied there.  Pins the mixture
    relaxation time, the power law in the inner fluid and the x-forcing of
    Eq. 12 with two components."""
    table = _golden("paper_table3_layered.json")["rows"]
    H, tau_out = 25, 0.8
    F, k, k_out = ccf.design(n, tau_in, tau_out, H, umax=0.005)
    p, C = inputs.layered_channel_case(n, k, F, tau_outer=tau_out, H=H)
    o = oracle.Oracle(p)
    o.set_fields(C)
    prev = None
    for _ in range(200):
        o.step(500)
        u = o.field("ux")[:, 0]
        if prev is not None and np.linalg.norm(u - prev) / np.linalg.norm(u) < 1e-9:
            break
        prev = u
    y = np.arange(2 * H) + 0.5 - H
    uq = ccf.stress_balance_profile(y, o.field("tau")[:, 0] / 3.0, F, H)
    assert np.linalg.norm(u - uq) / np.linalg.norm(uq) <= (2e-2 if n < 1 else 2e-3)
    if tau_in == tau_out:
        bound = max(r["E_rel"] for r in table if r["n3"] == n)
        ua = ccf.layered_profile(y, H, 0.5 * H, F, n, k, 1.0, k_out)
        assert np.linalg.norm(u - ua) / np.linalg.norm(ua) <= bound      # Eq. 35
    # the layers stay put: C is conserved and stays mirror-symmetric about the
    # centreline, with its 0.5 crossings at |y| = H/2 (the profile itself
    # widens to the width of the modified equation, see the flat-interface pin)
    c = o.field("C1")[:, 0]
    assert abs(c.sum() - C[0, :, 0].sum()) < 1e-10 * C[0].size
    assert np.max(np.abs(c - c[::-1])) < 1e-9
    j = int(np.argmax(c[: H] > 0.5))
    ycross = y[j - 1] + (0.5 - c[j - 1]) / (c[j] - c[j - 1])
    assert abs(abs(ycross) - 0.5 * H) < 0.05


# ------------------------------------------------------------------ P1c
@pytest.mark.parametrize("n,ny", [(0.5, 32), (1.0, 20), (1.5, 20)])
def test_open_channel_inlet_outlet(n, ny):
    """Sec. 3.2 in its own set-up: uniform inflow at x = 0, convective outflow
    at x = nx - 1 (reading R27), walls top and bottom.  At steady state the
    flow rate is the same in every column, the outlet pressure is the
    reference, and the profile three quarters down the channel has the fully
    developed power-law shape (2n+1)/(n+1) (1 - |y/H|^((n+1)/n)) times the mean
    velocity of that column within the Table 2 error for the same n."""
    table = _golden("paper_table2_channel.json")
    bound = dict(zip(table["n"], table["E_rel"]))[n]
    p, C, ux = inputs.open_channel_case(n, ny=ny)
    nx, uin = p["nx"], p["u_in"]
    o = oracle.Oracle(p)
    o.set_fields(C, ux=ux)
    prev = None
    for _ in range(200):
        o.step(250)
        u = o.field("ux")
        if prev is not None and np.linalg.norm(u - prev) / np.linalg.norm(u) < 1e-7:
            break
        prev = u
    flux = u.sum(axis=0)
    assert flux.max() / flux.min() - 1.0 < 1e-4
    assert abs(o.field("p")[:, -1].mean()) < 1e-12
    H = ny / 2.0
    y = np.arange(ny) + 0.5 - H
    col = u[:, 3 * nx // 4]
    ua = col.mean() * (2 * n + 1) / (n + 1) * (1.0 - np.abs(y / H) ** ((n + 1) / n))
    assert np.linalg.norm(col - ua) / np.linalg.norm(ua) <= bound          # Eq. 35
    # the inlet delivers nearly the imposed velocity (the wall rows of the
    # ghost column lose a few per cent)
    assert 0.95 < col.mean() / uin <= 1.0
    # the inflow carries the channel's own fluid: C moves by less than 1 % near
    # the inlet, where the equilibrium h at the imposed velocity meets the
    # slower wall rows
    c = o.field("C1")
    assert np.max(np.abs(c - 1.0)) < 1e-2 and np.mean(np.abs(c - 1.0)) < 2e-3


# ------------------------------------------------------------------ P8
def test_hydrostatic_pressure():
    """Gravity on a resting single phase between walls: p linear with slope -rho g."""
    g = 1e-5
    o = _single_phase(4, 40, gravity=g)
    o.step(20000)
    p = o.field("p")[:, 0]
    y = np.arange(40)
    slope, icpt = np.polyfit(y, p, 1)
    assert abs(slope + g) / g < 1e-6
    assert np.max(np.abs(p - (slope * y + icpt))) < 1e-6 * g * 40
    assert np.max(np.abs(o.field("uy"))) < 1e-12


# ------------------------------------------------------------------ P2
def test_laplace_law():
    """Static 2-D bubble: the pressure jump is sigma / R (the interface tension
    sigma_ij follows from the scaling of Eq. 2-5)."""
    sigma = 1e-3
    Rs, dps = [], []
    for R in (8.0, 10.0, 12.0):
        p = dict(nx=48, ny=48, ncomp=2, periodic_y=1, rho=(1.0, 1.0, 1.0), tau=(0.5, 0.5, 0.5),
                 sigma12=sigma, sigma13=sigma, sigma23=sigma, xi=4.0, D0=4.0 / 300.0)
        o = oracle.Oracle(p)
        o.init_bubbles([[24, 24, R, 3]])
        o.step(3000)
        pr = o.field("p")
        Reff = math.sqrt(o.observables()["area"] / math.pi)
        Rs.append(Reff)
        dps.append(pr[24, 24] - pr[0, 0])
        assert np.max(np.hypot(o.field("ux"), o.field("uy"))) < 1e-5
    slope = np.polyfit(1.0 / np.array(Rs), np.array(dps), 1)[0]
    assert abs(slope - sigma) / sigma < 0.05


# ------------------------------------------------------------------ P3
def test_chemical_potential_vanishes_on_tanh_profile():
    """The flat tanh profile of width xi (the shape of Eq. 42) is stationary for
    the free energy of Eq. 2-3: mu_1 - mu_3 (the potential of C1 when C2 = 0)
    vanishes up to the stencil error, here made small with a wide interface."""
    xi, sigma, nx = 24.0, 1e-3, 256
    p = dict(nx=nx, ny=2, ncomp=2, periodic_y=1, sigma12=sigma, sigma13=sigma, sigma23=sigma, xi=xi)
    o = oracle.Oracle(p)
    x = np.arange(nx, dtype=float)
    C = 0.5 + 0.5 * np.tanh(2 * (x - 64) / xi) - (0.5 + 0.5 * np.tanh(2 * (x - 192) / xi))
    o.set_fields(np.tile(C, (2, 1))[None])
    mu = o.field("mu1")[0] - o.field("mu3")[0]
    scale = 12 * sigma / xi          # magnitude of the double-well term
    assert np.max(np.abs(mu)) < 2e-3 * scale
    # a profile twice too wide is far from stationary
    C2 = 0.5 + 0.5 * np.tanh((x - 64) / xi) - (0.5 + 0.5 * np.tanh((x - 192) / xi))
    o.set_fields(np.tile(C2, (2, 1))[None])
    mu2 = o.field("mu1")[0] - o.field("mu3")[0]
    assert np.max(np.abs(mu2)) > 0.1 * scale


@pytest.mark.parametrize("D0", [4.0 / 300.0, 0.01])
def test_flat_interface_width_modified_equation(D0):
    """Flat interface dynamics.  With tau_h = 1/2 the collision of Eq. 18 sets
    h to its equilibrium, and streaming plus the central directional derivative
    add -(1/24) lap^2 C per step (Taylor expansion of the D2Q9 shift); the CH
    equation then has gradient coefficient (3/4) xi + 1/(24 D0), so the
    stationary tanh widens to xi sqrt(1 + 1/(18 D0 xi)).  A sign slip in the
    half forcing of Eq. 18-20 turns this into second-order diffusion."""
    xi, nx = 4.0, 64
    p = dict(nx=nx, ny=2, ncomp=2, periodic_y=1, xi=xi, D0=D0)
    o = oracle.Oracle(p)
    x = np.arange(nx, dtype=float)
    C = 0.5 + 0.5 * np.tanh(2 * (x - 16) / xi) - (0.5 + 0.5 * np.tanh(2 * (x - 48) / xi))
    o.set_fields(np.tile(C, (2, 1))[None])
    o.step(4000)
    c = o.field("C1")[0]
    width = 1.0 / np.max(np.gradient(c))       # tanh(2x/w)/2 has slope 1/w at its centre
    pred = xi * math.sqrt(1.0 + 1.0 / (18.0 * D0 * xi))
    assert abs(width - pred) / pred < 0.05
    assert abs(c.sum() - C.sum()) < 1e-10


# ------------------------------------------------------------------ P4
def test_mass_conservation_constant_mobility():
    """Constant mobility: every source of Eq. 18 sums to zero over directions
    and the discrete Laplacian telescopes (mirror ghosts at walls), so each
    component's mass is conserved to round-off."""
    p, b = inputs.small_case(mobility=0)
    p = dict(p, nx=32, ny=64)
    o = oracle.Oracle(p)
    o.init_bubbles([[16, 20, 6, 3]], seed=1, noise=1e-8)
    m0 = o.observables()["mass"]
    o.step(300)
    m1 = o.observables()["mass"]
    nodes = p["nx"] * p["ny"]
    for i in (0, 2):
        # round-off of a sum of `nodes` values of order 1, over 300 steps
        assert abs(m1[i] - m0[i]) < 1e-13 * nodes


def test_mass_balance_variable_mobility():
    """Variable mobility: the split form of Eq. 21 is not a discrete divergence,
    so mass changes by exactly the summed diffusion sources per step."""
    p, b = inputs.small_case(mobility=1)
    p = dict(p, nx=32, ny=64)
    o = oracle.Oracle(p)
    o.init_bubbles([[16, 20, 6, 3]], seed=1, noise=1e-8)
    o.step(50)
    for _ in range(5):
        m0 = o.observables()["mass"][0]
        o.step(1)
        src = o.field("S")[0].sum() + o.field("V")[0].sum()
        m1 = o.observables()["mass"][0]
        assert abs((m1 - m0) - src) < 1e-12 * abs(m0)


# ------------------------------------------------------------------ P5
def test_binary_reduction_three_sets():
    """With C2 = 0 the chemical potential mu_2 vanishes (Sigma_1 + Sigma_3 =
    2 sigma_13), so a three-set run stays binary and equals the two-set run."""
    p, b = inputs.small_case(mobility=0)
    p2 = dict(p, nx=24, ny=48, sigma12=1.2e-3, sigma23=0.9e-3)
    C = inputs.bubble_fields(24, 48, 2, 4.0, [(12, 16, 6, 3)], seed=2, noise=1e-8)
    a = oracle.Oracle(p2)
    a.set_fields(C)
    p3 = dict(p2, ncomp=3)
    b3 = oracle.Oracle(p3)
    b3.set_fields(np.stack([C[0], np.zeros_like(C[0])]))
    a.step(200)
    b3.step(200)
    assert np.max(np.abs(b3.field("C2"))) < 1e-14
    for f in ("C1", "p", "ux", "uy", "tau"):
        x, y = a.field(f), b3.field(f)
        # 200 steps of round-off through the power law (pow of a small shear rate)
        assert np.max(np.abs(x - y)) <= 1e-10 * max(1.0, np.max(np.abs(x)))


# ------------------------------------------------------------------ P6
@pytest.mark.parametrize("periodic_y", [1, 0])
@pytest.mark.parametrize("ncomp", [2, 3])
@pytest.mark.parametrize("mobility", [0, 1])
@pytest.mark.parametrize("fd_scheme", [0, 1])
@pytest.mark.parametrize("powerlaw", [0, 1])
def test_hand_step_4x4(periodic_y, ncomp, mobility, fd_scheme, powerlaw):
    """Brute force: an independent vectorised NumPy restatement of the step
    (tests/handstep_numpy.py) on a 4 x 4 grid for 3 steps."""
    rng = np.random.default_rng(100 + 16 * periodic_y + 8 * ncomp + 4 * mobility + 2 * fd_scheme + powerlaw)
    P = dict(oracle.DEFAULTS)
    P.update(nx=4, ny=4, ncomp=ncomp, periodic_y=periodic_y, rho=(1.0, 0.5, 0.1),
             tau=(0.6, 0.7, 0.55), powerlaw=powerlaw, pl_n=0.7, pl_k=0.05, gravity=1e-3,
             force_x=2e-4, mobility=mobility, fd_scheme=fd_scheme, D0=0.01, sigma12=1e-3,
             sigma13=1.5e-3, sigma23=2e-3)
    C = np.zeros((ncomp - 1, 4, 4))
    C[0] = 0.5 + 0.4 * rng.random((4, 4))
    if ncomp == 3:
        C[1] = 0.3 * rng.random((4, 4))
    o = oracle.Oracle(P)
    o.set_fields(C)
    g, h, tau = hs.init_state(P, C)
    assert np.max(np.abs(o.field("g") - g)) < 1e-15
    assert np.max(np.abs(o.field("h") - h)) < 1e-15
    for _ in range(3):
        o.step(1)
        g, h, tau = hs.step(P, g, h, tau)
    assert np.max(np.abs(o.field("g") - g)) < 1e-11
    assert np.max(np.abs(o.field("h") - h)) < 1e-11
    assert np.max(np.abs(o.field("tau") - tau)) < 1e-11


@pytest.mark.parametrize("ncomp", [2, 3])
def test_hand_step_4x4_order_parameter_outside_unit_interval(ncomp):
    """The same brute-force comparison with order parameters that leave [0, 1]
    at some nodes (as the Cahn-Hilliard bulk shift does inside bubbles): the
    clipped mixture weights and the clipped variable mobility with its
    derivative term switched off there (readings R1, R8)."""
    rng = np.random.default_rng(7 + ncomp)
    P = dict(oracle.DEFAULTS)
    P.update(nx=4, ny=4, ncomp=ncomp, periodic_y=0, rho=(1.0, 0.5, 0.1), tau=(0.6, 0.7, 0.55), powerlaw=1,
             pl_n=0.7, pl_k=0.05, gravity=1e-3, mobility=1, D0=0.01, sigma12=1e-3, sigma13=1.5e-3, sigma23=2e-3)
    C = np.zeros((ncomp - 1, 4, 4))
    C[0] = -0.06 + 1.12 * rng.random((4, 4))
    C[0, 0, 1], C[0, 2, 3], C[0, 3, 0] = -0.05, 1.04, -0.02
    if ncomp == 3:
        C[1] = -0.04 + 0.3 * rng.random((4, 4))
        C[1, 1, 2] = -0.03
    o = oracle.Oracle(P)
    o.set_fields(C)
    g, h, tau = hs.init_state(P, C)
    for _ in range(3):
        o.step(1)
        g, h, tau = hs.step(P, g, h, tau)
    assert np.max(np.abs(o.field("g") - g)) < 1e-11
    assert np.max(np.abs(o.field("h") - h)) < 1e-11
    assert np.max(np.abs(o.field("tau") - tau)) < 1e-11


# ------------------------------------------------------------------ P7
def test_uniform_rest_state_is_fixed_point():
    o = _single_phase(6, 5)
    g0 = o.field("g")
    o.step(50)
    assert np.max(np.abs(o.field("g") - g0)) < 1e-15


def test_newtonian_power_law_equals_fixed_tau():
    """n = 1 turns Eq. 31 into eta = k, i.e. tau = k / (rho cs^2)."""
    k = 0.25
    a = _single_phase(2, 20, powerlaw=1, pl_n=1.0, pl_k=k, tau_max=10.0, force_x=1e-6)
    b = _single_phase(2, 20, tau=(3 * k, 3 * k, 3 * k), force_x=1e-6)
    a.step(500)
    b.step(500)
    assert np.max(np.abs(a.field("ux") - b.field("ux"))) < 1e-13 * np.max(np.abs(b.field("ux")))


def test_mirror_symmetry_of_centred_bubble():
    p, _ = inputs.small_case(mobility=1)
    p = dict(p, nx=32, ny=48)
    o = oracle.Oracle(p)
    o.set_fields(inputs.bubble_fields(32, 48, 2, 4.0, [(15.5, 16, 7, 3)]))
    o.step(100)
    ux, uy = o.field("ux"), o.field("uy")
    # x -> 31 - x maps the lattice onto itself about the disc centre 15.5
    assert np.max(np.abs(ux + ux[:, ::-1])) < 1e-13
    assert np.max(np.abs(uy - uy[:, ::-1])) < 1e-13
    assert np.max(np.abs(uy)) > 1e-8


# ------------------------------------------------------------------ P9
def test_observable_formulas_against_tables_5_to_7():
    """Eo (Eq. 40) and Re (Eq. 38) recomputed from Table 5 and the terminal
    velocities of Table 7 (d = L/4 = 50) reproduce Table 6; the buoyancy drag of
    Eq. 37 agrees with the Li correlation of Eq. 41 where Table 7 reports 0 error."""
    t = _golden("paper_tables5to7_bubble.json")
    rho_l, rho_g, d = 1.0, 1.0 / t["density_ratio"], t["d"]
    for c in t["cases"]:
        Eo = obs.eotvos(rho_l, rho_g, c["g"], d, c["sigma"])
        assert abs(Eo - c["Eo"]) / c["Eo"] < 0.005
        Re = obs.reynolds(rho_l, c["Ut_present"], d, c["n"], c["k"])
        tol = 0.03 if c["case"] >= 4 else 0.10
        assert abs(Re - c["Re"]) / c["Re"] < tol
    c4 = t["cases"][3]
    cd_buoy = obs.drag_coefficient(d, c4["g"], rho_l, rho_g, c4["Ut_present"])
    Re4 = obs.reynolds(rho_l, c4["Ut_present"], d, c4["n"], c4["k"])
    cd_li = obs.li_correlation(Re4, c4["n"], c4["E"])
    assert abs(cd_buoy - cd_li) / cd_li < 0.05


# ------------------------------------------------------------------ inputs
# ------------------------------------------------------------------ P9b
@pytest.mark.parametrize("ncomp", [2, 3])
def test_observable_sums_of_prescribed_disc(ncomp):
    """Raw observable sums (Sec. 3.1 masses, Eq. 43-44 centroid and mean
    velocity, the C_g > 0.5 extents behind the aspect ratio of Eq. 41) of a
    state whose answers are fixed without the oracle.

    A gas disc centred between nodes, (31.5, 47.5), on a 64 x 96 lattice is
    mirror-symmetric about both centre lines, so its C_g-weighted centroid is
    the centre.  The state is set with a uniform velocity (u_x, u_y) =
    (0.011, -0.0037) and no step is taken: the equilibria of Eq. 16 return
    that velocity through Eq. 23 (their first moment is rho u minus half the
    force), so sum C_g u / sum C_g is the prescribed velocity.  C_g > 0.5
    exactly where the tanh profile has r < R, so the extents are those of the
    nodes inside the circle, counted here by brute force.  The masses are the
    plain sums of the fields that were set.  Different x and y (centre,
    velocity, lattice sides) catch a swap of the axes; the extents catch an
    off-by-one."""
    nx, ny, R, xi = 64, 96, 10.3, 4.0
    cx, cy = 31.5, 47.5
    ux0, uy0 = 0.011, -0.0037
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    r = np.hypot(x - cx, y - cy)
    cg = 0.5 - 0.5 * np.tanh((r - R) / (0.5 * xi))
    if ncomp == 2:
        C = (1.0 - cg)[None]
        comps = [1.0 - cg, np.zeros_like(cg), cg]
    else:  # a droplet of component 2 in the lower half, the gas disc as above
        c2 = 0.5 - 0.5 * np.tanh((np.hypot(x - 20.0, y - 15.0) - 6.2) / (0.5 * xi))
        C = np.stack([1.0 - cg - c2, c2])
        comps = [1.0 - cg - c2, c2, cg]
    p = dict(nx=nx, ny=ny, ncomp=ncomp, rho=(1.0, 1.0, 0.05), tau=(0.8, 0.8, 0.5), gravity=1e-6,
             sigma12=1e-3, sigma13=1e-3, sigma23=1e-3, xi=xi)
    o = oracle.Oracle(p)
    o.set_fields(C, ux=np.full((ny, nx), ux0), uy=np.full((ny, nx), uy0))
    raw = o.raw_observables(gas_comp=3)
    for i in range(3):
        assert raw[i] == pytest.approx(comps[i].sum(), rel=1e-13, abs=1e-10)
        assert raw[3 + i] == pytest.approx(comps[i][comps[i] > 0.5].sum(), rel=1e-13, abs=1e-10)
    A = raw[6]
    assert A == pytest.approx(cg.sum(), rel=1e-13)
    assert raw[7] / A == pytest.approx(cx, abs=1e-9)
    assert raw[8] / A == pytest.approx(cy, abs=1e-9)
    assert raw[9] / A == pytest.approx(ux0, rel=1e-9)
    assert raw[10] / A == pytest.approx(uy0, rel=1e-9)
    inside = [(i, j) for j in range(ny) for i in range(nx) if (i - cx) ** 2 + (j - cy) ** 2 < R * R]
    xs = [i for i, _ in inside]
    ys = [j for _, j in inside]
    assert list(raw[11:]) == [min(xs), max(xs), min(ys), max(ys)]
    assert (max(xs) - min(xs), max(ys) - min(ys)) == (19, 19)   # |dx|, |dy| <= 9.5 inside R = 10.3


def test_openmp_build_is_bit_identical():
    """The OpenMP build of the oracle (timed CPU baseline only) shares each
    whole-field pass's nodes among threads; every node keeps its own order of
    operations, so after several steps of a walled three-component variable-
    mobility case every field equals the serial build's bit for bit."""
    p, discs = inputs.three_comp_case(nx=48, mobility=1, seed=3)
    p = dict(p, periodic_y=0, gravity=1e-6)
    C = inputs.bubble_fields(48, 48, 3, p["xi"], discs, seed=1, noise=1e-8)
    runs = []
    for prec in ("f64", "f64-omp"):
        o = oracle.Oracle(p, prec)
        o.set_fields(C)
        o.step(7)
        runs.append({name: o.field(name) for name in ("g", "h", "tau", "p", "ux", "uy", "C1", "C2")})
    for name in runs[0]:
        assert np.array_equal(runs[0][name], runs[1][name]), name


def test_splitmix64_reference_vectors():
    t = _golden("splitmix64_vectors.json")
    for v in t["vectors"]:
        got = inputs.splitmix64_at(v["seed"], np.arange(len(v["outputs"])))
        assert [int(x) for x in got] == [int(h, 16) for h in v["outputs"]]


def test_oracle_bubble_init_matches_input_generator():
    p, b = inputs.small_case()
    o = oracle.Oracle(p)
    o.init_bubbles([list(x) for x in b], seed=5, noise=1e-8)
    C = inputs.bubble_fields(p["nx"], p["ny"], 2, p["xi"], b, seed=5, noise=1e-8)
    assert np.max(np.abs(o.field("C1") - C[0])) < 1e-15
    # disc profile of Eq. 42 at the centre and one radius out
    assert abs(C[0][32, 32] - (0.5 + 0.5 * math.tanh(-10 / 2.0))) < 2e-8
    assert abs(C[0][32, 42] - 0.5) < 2e-8


# ------------------------------------------------------------- surrogate MLP
def test_mlp_oracle_gradients_finite_differences():
    """Backward pass of the FP64 network against central finite differences."""
    from oracle import mlp

    w = inputs.mlp_init(1, seed=3)[0]
    params = inputs.mlp_unflatten(w)
    rng = np.random.default_rng(0)
    X, T = rng.normal(size=(6, 5)), rng.normal(size=(6, 2))
    Y, cache = mlp.forward(params, X, bf16=False)
    grads = mlp.backward(params, cache, Y, T, bf16=False)
    flat_g = inputs.mlp_flatten(grads)
    idx = rng.choice(w.size, size=40, replace=False)
    for i in idx:
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        lp = mlp.loss(mlp.forward(inputs.mlp_unflatten(wp), X, bf16=False)[0], T)
        lm = mlp.loss(mlp.forward(inputs.mlp_unflatten(wm), X, bf16=False)[0], T)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - flat_g[i]) <= 1e-7 + 1e-5 * abs(fd)


def test_mlp_oracle_adam_first_step_closed_form():
    """First Adam step: bias-corrected moments are g and g^2, so the update is
    -lr g / (|g| + eps) (Kingma and Ba 2015, Algorithm 1)."""
    from oracle import mlp

    params = inputs.mlp_unflatten(inputs.mlp_init(1, seed=4)[0])
    rng = np.random.default_rng(1)
    grads = [(rng.normal(size=W.shape), rng.normal(size=b.shape)) for W, b in params]
    lr, eps = 1e-3, 1e-8
    new, _ = mlp.adam(params, grads, mlp.adam_state(params), lr, eps=eps)
    for (W, b), (W2, b2), (gW, gb) in zip(params, new, grads):
        assert np.allclose(W2 - W, -lr * gW / (np.abs(gW) + eps), rtol=1e-12, atol=1e-15)
        assert np.allclose(b2 - b, -lr * gb / (np.abs(gb) + eps), rtol=1e-12, atol=1e-15)


def test_bf16_rounding_reference_values():
    """Round to nearest even at 8 mantissa bits (bfloat16)."""
    from oracle import mlp

    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, np.float32(np.pi), -2.5, 1.0 + 2.0 ** -7 + 2.0 ** -8])
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -7, 3.140625, -2.5, 1.0 + 2.0 ** -6])
    assert np.array_equal(mlp.round_bf16(vals), want)


def test_table5_inputs_are_the_printed_values():
    """The Table 5 set-ups the density-ratio-1000 tests run are the printed
    (n, k, g, sigma) of Sec. 4.3 (the golden file transcribes the tables)."""
    table = {c["case"]: c for c in _golden("paper_tables5to7_bubble.json")["cases"]}
    for case, (n, k, g, sigma) in inputs.TABLE5.items():
        assert (n, k, g, sigma) == (table[case]["n"], table[case]["k"], table[case]["g"], table[case]["sigma"])
        p, discs = inputs.table5_case(case)
        assert (p["nx"], p["ny"]) == (200, 400) and discs == [(100.0, 120.0, 25.0, 3)]
        assert p["rho"][2] == pytest.approx(1.0 / 800.0) and p["tau"][2] == 0.5


@pytest.mark.parametrize("case,suffix", [(6, ""), (4, ""), (6, "_f32"), (4, "_f32")])
def test_oracle_terminal_golden_is_self_consistent(case, suffix):
    """The stored oracle rise to the terminal state (FP64, and the FP32 build
    that gives the rounding floor): U_t is the last 2000-step window of the
    stored centroid series, the 1 % rule holds there and not a window earlier,
    and C_D is Eq. 37 at U_t through the oracle's post-processing (the drag of
    a rising bubble: 4 (rho_l - rho_g) g d / (3 rho_l U^2) with d from the gas
    area)."""
    gold = _golden(f"oracle_terminal_table5_case{case}_r1000{suffix}.json")
    k = gold["window"] // gold["every"]
    assert gold["steps"][-1] == gold["terminal_step"]
    y = np.asarray(gold["ybar"])[k - 1::k]
    u = np.diff(y) / gold["window"]
    assert u[-1] == pytest.approx(gold["U_t"], rel=1e-12)

    def terminal(v):
        return len(v) >= 3 and all(abs(v[-j] - v[-j - 1]) < 0.01 * abs(v[-j]) for j in (1, 2))

    assert terminal(u) and not terminal(u[:-1])
    p, _ = inputs.table5_case(case, density_ratio=1000.0)
    A = gold["area"][-1]
    d = 2.0 * math.sqrt(A / math.pi)
    rho_l, rho_g = p["rho"][0], p["rho"][2]
    cd = 4.0 * (rho_l - rho_g) * p["gravity"] * d / (3.0 * rho_l * gold["U_t"] ** 2)
    assert gold["C_D"] == pytest.approx(cd, rel=1e-9)
    if not suffix:
        # FP64 conserves the gas area (sum of C_g) to rounding over the rise
        assert max(gold["area"]) - min(gold["area"]) < 1e-9 * gold["area"][0]
