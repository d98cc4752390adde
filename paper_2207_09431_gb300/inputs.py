"""Seeded synthetic inputs: lattice set-ups, bubble discs and case parameters.

This module only builds inputs.  It holds none of the time-step arithmetic, and
both the CUDA library's callers and the CPU oracle's tests draw their inputs
from it.  Every array it returns is float64 on the host.

Workloads (rising bubble in a power-law liquid, arXiv 2207.09431 Sec. 4):
  small        64 x 128, one gas bubble R = 10 at (32, 32)
  paper        200 x 400, R = 25 at (100, 240)  (x = L/2, y = 0.6 L of Eq. 42)
  sweep        nx x 2 nx with R = nx / 8, same physics as `paper`
  three_comp   256 x 256 periodic, two droplets of component 2, one bubble of 3
  ensemble     cases with grids from {100x200, 150x300, 200x400, 300x600}
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_at(seed: int, counters) -> np.ndarray:
    """SplitMix64 (Steele, Lea and Flood 2014) output number i+1 of the stream
    that starts at state ``seed``: mix(seed + (i + 1) * 0x9E3779B97F4A7C15)."""
    i = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (i + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform_noise(seed: int, counters, amp: float) -> np.ndarray:
    """Uniform values in [-amp, amp): 53 high bits of SplitMix64."""
    z = splitmix64_at(seed, counters)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return amp * (2.0 * u - 1.0)


def bubble_fields(nx, ny, ncomp, xi, bubbles, seed=0, noise=0.0, periodic_y=False):
    """Initial order parameters of discs (Sec. 4.2, Eq. 42).

    Component c of every disc (cx, cy, R, c) gets 0.5 - 0.5 tanh((r - R)/(xi/2))
    (periodic distance along periodic axes) plus uniform noise in [-noise, noise]
    drawn at counter (c - 1) * nx * ny + node; component 1 is the rest.
    Returns the transported fields, shape (ncomp - 1, ny, nx): C1 (and C2).
    """
    n = nx * ny
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    comp_field = {2: np.zeros((ny, nx)), 3: np.zeros((ny, nx))}
    used = set()
    for cx, cy, R, c in bubbles:
        c = int(c)
        if c not in (2, 3) or (ncomp == 2 and c != 3):
            raise ValueError("disc component must be 3 (two components) or 2/3 (three)")
        used.add(c)
        dx = np.abs(x - cx)
        dx = np.where(dx > 0.5 * nx, nx - dx, dx)
        dy = np.abs(y - cy)
        if periodic_y:
            dy = np.where(dy > 0.5 * ny, ny - dy, dy)
        r = np.sqrt(dx * dx + dy * dy)
        comp_field[c] = comp_field[c] + (0.5 - 0.5 * np.tanh((r - R) / (0.5 * xi)))
    if noise != 0.0:
        k = np.arange(n, dtype=np.uint64)
        for c in sorted(used):
            counters = np.uint64((c - 1) * n) + k
            comp_field[c] = comp_field[c] + uniform_noise(seed, counters, noise).reshape(ny, nx)
    C1 = 1.0 - comp_field[2] - comp_field[3]
    if ncomp == 2:
        return C1[None].copy()
    return np.stack([C1, comp_field[2]])


def round_to_fp32(a) -> np.ndarray:
    """Values rounded to the nearest float32, returned as float64."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


# ----------------------------------------------------------------- workloads

def rising_bubble_params(nx, ny, *, density_ratio=1000.0, n=0.7, k=1.667e-2, sigma=1e-3,
                         eotvos=None, gravity=None, radius=None, xi=4.0, D0=4.0 / 300.0,
                         mobility=0, tau_gas=0.5, tau_min=0.01, tau_max=3.0, powerlaw=1):
    """Two-component rising bubble: liquid = component 1 (power law), gas =
    component 3, walls at top and bottom, periodic sides.  Gravity is given
    directly or through the Eotvos number Eo = drho g d^2 / sigma with d = 2R."""
    rho_g = 1.0 / density_ratio
    if gravity is None:
        d = 2.0 * radius
        gravity = eotvos * sigma / ((1.0 - rho_g) * d * d)
    return dict(nx=nx, ny=ny, ncomp=2, periodic_y=0, rho=(1.0, 1.0, rho_g),
                tau=(0.5, 0.5, tau_gas), powerlaw=powerlaw, pl_n=n, pl_k=k,
                tau_min=tau_min, tau_max=tau_max, sigma12=sigma, sigma13=sigma, sigma23=sigma,
                Lambda=0.0, xi=xi, D0=D0, mobility=mobility, gravity=gravity, force_x=0.0,
                fd_scheme=0, gas_comp=3)


def small_case(mobility=0, density_ratio=100.0):
    """64 x 128 rising bubble, R = 10 at (32, 32), Eo = 10, n = 0.7.

    Density ratio 100 and D0 = xi/300: the printed scheme diverges at density
    ratio 1000 for this small bubble, and D0 = 0.02 lies past the scheme's
    linear stability bound at xi = 4 (both measured with the oracle)."""
    p = rising_bubble_params(64, 128, density_ratio=density_ratio, radius=10.0, eotvos=10.0,
                             mobility=mobility)
    return p, [(32.0, 32.0, 10.0, 3)]


def sweep_case(nx, density_ratio=1000.0, mobility=0):
    """Bandwidth-sweep rising bubble on nx x 2nx, R = nx / 8 at (nx/2, 0.6 * 2nx / 2)."""
    ny = 2 * nx
    R = nx / 8.0
    d = 2.0 * R
    g = 0.01 ** 2 / 50.0  # sqrt(g d) = 0.01 for the paper's d = 50
    sigma = (1.0 - 1.0 / density_ratio) * g * d * d / 10.0  # Eo = 10
    p = rising_bubble_params(nx, ny, density_ratio=density_ratio, sigma=sigma, gravity=g,
                             mobility=mobility)
    return p, [(nx / 2.0, 0.3 * ny, R, 3)]


def paper_case(n=0.6, eotvos=10.0, density_ratio=1000.0, mobility=1, k=None):
    """200 x 400, d = 50 (L/4) at (L/2, 0.6 L) as in Sec. 4.2-4.3."""
    L = 200
    R = 25.0
    d = 2 * R
    g = 2e-6
    sigma = (1.0 - 1.0 / density_ratio) * g * d * d / eotvos
    if k is None:
        k = 5e-4
    p = rising_bubble_params(L, 2 * L, density_ratio=density_ratio, n=n, k=k, sigma=sigma,
                             gravity=g, mobility=mobility)
    return p, [(L / 2.0, 0.6 * L, R, 3)]


# Table 5 of Sec. 4.3: (n, k, g, sigma) of the six rising-bubble cases (density
# ratio 800, tau of the gas 0.5, d = L / 4 on L x 2L with L = 200).
TABLE5 = {1: (0.5, 1e-4, 5e-7, 2.61e-6), 2: (0.5, 1e-4, 5e-7, 2.61e-5), 3: (0.5, 2e-4, 5e-7, 5e-4),
          4: (0.6, 5e-4, 2e-7, 2.61e-5), 5: (0.63, 5e-4, 2e-7, 2.61e-5), 6: (0.8, 1e-2, 5e-7, 2.61e-5)}


def table5_case(case, density_ratio=800.0, mobility=0, L=200):
    """Case `case` of Table 5 (Sec. 4.3): L x 2L, bubble d = L / 4 at (L/2, 0.6 L)
    (Eq. 42), the printed n, k, g and sigma, gas relaxation time 0.5, at the
    given density ratio (the paper's is 800)."""
    n, k, g, sigma = TABLE5[case]
    p = rising_bubble_params(L, 2 * L, density_ratio=density_ratio, n=n, k=k, sigma=sigma, gravity=g,
                             mobility=mobility)
    return p, [(L / 2.0, 0.6 * L, L / 8.0, 3)]


def paper_grid_cases(density_ratio=1000.0, mobility=0, fd_scheme=0, ns=(0.5, 0.6, 0.8, 1.0),
                     eotvos=(1.0, 10.0, 50.0), log10_mo=(-3.0, -1.0, 1.0), L=200):
    """The rising-bubble grid of Sec. 4.3 at the paper's size: L x 2L, d = L/4
    at (L/2, 0.6 L), g from sqrt(g d) = 0.01, sigma from Eo, the power-law
    consistency k from Mo = g drho / (rho_l^2 sigma^3) [k (U/d)^(n-1)]^4 with
    U = sqrt(g d), gas relaxation time 0.5 (viscosity ratio k / eta_gas up to
    about 1000).  Returns [(params, discs, meta)]."""
    out = []
    R = L / 8.0
    d = 2.0 * R
    g = 0.01 ** 2 / d
    U = math.sqrt(g * d)
    rho_g = 1.0 / density_ratio
    drho = 1.0 - rho_g
    for n in ns:
        for Eo in eotvos:
            for lm in log10_mo:
                sigma = drho * g * d * d / Eo
                k = (10.0 ** lm * sigma ** 3 / (g * drho)) ** 0.25 / (U / d) ** (n - 1.0)
                p = rising_bubble_params(L, 2 * L, density_ratio=density_ratio, n=n, k=k, sigma=sigma,
                                         gravity=g, mobility=mobility)
                p["fd_scheme"] = fd_scheme
                out.append((p, [(L / 2.0, 0.6 * L, R, 3)], dict(n=n, Eo=Eo, log10_Mo=lm, density_ratio=density_ratio,
                                                               viscosity_ratio=k / (rho_g * p["tau"][2] / 3.0))))
    return out


def three_comp_case(nx=256, mobility=0, seed=0, max_draws=100000):
    """Three components, fully periodic: matrix 1 (power law n = 0.6), two droplets
    of component 2 (R = 20, 12 at nx = 256, scaled with nx) and a bubble of 3
    (R = 6, scaled) at seeded non-overlapping centres; no gravity."""
    xi = 4.0
    p = dict(nx=nx, ny=nx, ncomp=3, periodic_y=1, rho=(1.0, 1.0, 0.01), tau=(0.5, 0.5, 0.25),
             powerlaw=1, pl_n=0.6, pl_k=1e-2, tau_min=0.01, tau_max=3.0, sigma12=1e-3,
             sigma13=1e-3, sigma23=1e-3, Lambda=0.0, xi=xi, D0=xi / 300.0, mobility=mobility,
             gravity=0.0, force_x=0.0, fd_scheme=0, gas_comp=3)
    scale = nx / 256.0
    radii = [(max(20.0 * scale, 4.0), 2), (max(12.0 * scale, 4.0), 2), (max(6.0 * scale, 3.0), 3)]
    gap = 2 * xi * max(scale, 0.25)
    centres = []
    for draw in range(max_draws):
        if len(centres) == len(radii):
            break
        z = splitmix64_at(seed, [2 * draw, 2 * draw + 1])
        cx, cy = (z >> np.uint64(11)).astype(np.float64) * (nx / 9007199254740992.0)
        R, c = radii[len(centres)]
        ok = True
        for (ox, oy, oR, _) in centres:
            dx = min(abs(cx - ox), nx - abs(cx - ox))
            dy = min(abs(cy - oy), nx - abs(cy - oy))
            if math.hypot(dx, dy) < R + oR + gap:
                ok = False
        if ok:
            centres.append((float(cx), float(cy), R, c))
    if len(centres) < len(radii):
        raise ValueError("could not place the discs without overlap")
    return p, centres


def layered_channel_case(n, k, force, tau_outer=0.8, H=25, nx=2, xi=4.0, sigma=5e-4, tau_min=0.02, tau_max=20.0):
    """Two-phase layered channel of Sec. 3.3: walls at y = -0.5 and y = 2H - 0.5
    (half-way bounce-back), periodic in x, a uniform body force along x, equal
    densities, and the fluid at |y - H + 0.5| < H/2 different from the fluid
    outside.  The paper puts the power-law fluid (its component 3) in the
    middle and a Newtonian one outside; here the power-law fluid is component 1
    (the component whose relaxation time the power law sets) and the outer
    Newtonian fluid component 3 with tau_outer, the same flow with the labels
    swapped.  Returns (params, C) with the tanh profile of Eq. 42 across the
    two flat interfaces."""
    ny = 2 * H
    y = np.arange(ny) + 0.5 - H
    C1 = 0.5 - 0.5 * np.tanh((np.abs(y) - 0.5 * H) / (0.5 * xi))
    p = dict(nx=nx, ny=ny, ncomp=2, rho=(1.0, 1.0, 1.0), tau=(tau_outer, tau_outer, tau_outer), powerlaw=1,
             pl_n=n, pl_k=k, tau_min=tau_min, tau_max=tau_max, force_x=force, sigma12=sigma, sigma13=sigma,
             sigma23=sigma, xi=xi, D0=xi / 300.0)
    return p, np.repeat(C1[None, :, None], nx, axis=2)


def open_channel_case(n, ny=20, nx=40, u_in=0.04, tau_wall=0.8, tau_min=0.02, tau_max=20.0):
    """Single-phase power-law channel of Sec. 3.2 between walls at y = -0.5 and
    y = ny - 0.5, velocity inlet at x = 0 and convective outlet at x = nx - 1,
    filled with component 1 (the power-law component; the paper fills it with
    its component 3, the same fluid under another label).  The consistency k
    gives tau = tau_wall at the wall shear rate of the fully developed profile
    with mean velocity u_in.  Returns (params, C, ux) with the channel at rest
    in pressure and moving at u_in."""
    H = ny / 2.0
    gw = u_in * (2 * n + 1) / n / H
    k = (tau_wall / 3.0) / gw ** (n - 1.0)
    p = dict(nx=nx, ny=ny, ncomp=2, periodic_y=0, rho=(1.0, 1.0, 1.0), tau=(tau_wall,) * 3, powerlaw=1,
             pl_n=n, pl_k=k, tau_min=tau_min, tau_max=tau_max, open_x=1, u_in=u_in, c_in=(1.0, 0.0))
    return p, np.ones((1, ny, nx)), np.full((ny, nx), u_in)


ENSEMBLE_GRIDS = ((100, 200), (150, 300), (200, 400), (300, 600))


def ensemble_cases(ncases=128, seed=0, grids=ENSEMBLE_GRIDS, density_ratio=100.0, mobility=0):
    """Seeded rising-bubble cases: grid drawn from ``grids``, R = nx / 8,
    n ~ U[0.4, 1.0], Eo ~ U[1, 100], log10 Mo ~ U[-3, 1] (Mo taken with the
    velocity scale sqrt(g d)), g from sqrt(g d) = 0.01.  Density ratio 100 by
    default: at 1000 the printed scheme diverges within 100 steps for the
    R = 12.5 bubbles of the smallest grid (measured with the oracle).  Constant
    mobility by default: with the variable mobility as printed, C undershoots
    grow and the 100 x 200 cases diverge within 2000 steps (oracle)."""
    cases = []
    for c in range(ncases):
        z = splitmix64_at(seed + 7919 * c, np.arange(4, dtype=np.uint64))
        u = (z >> np.uint64(11)).astype(np.float64) / 9007199254740992.0
        nx, ny = grids[int(u[0] * len(grids)) % len(grids)]
        n = 0.4 + 0.6 * u[1]
        Eo = 1.0 + 99.0 * u[2]
        log_mo = -3.0 + 4.0 * u[3]
        R = nx / 8.0
        d = 2.0 * R
        g = 0.01 ** 2 / d
        rho_g = 1.0 / density_ratio
        drho = 1.0 - rho_g
        sigma = drho * g * d * d / Eo
        U = math.sqrt(g * d)
        # Mo = g drho / (rho_l^2 sigma^3) [k (U/d)^(n-1)]^4  ->  k
        k = (10.0 ** log_mo * sigma ** 3 / (g * drho)) ** 0.25 / (U / d) ** (n - 1.0)
        p = rising_bubble_params(nx, ny, density_ratio=density_ratio, n=n, k=k, sigma=sigma,
                                 gravity=g, mobility=mobility)
        cases.append((p, [(nx / 2.0, 0.3 * ny, R, 3)],
                      dict(n=n, Eo=Eo, log10_Mo=log_mo, density_ratio=density_ratio)))
    return cases


# ------------------------------------------------------------------ surrogate

MLP_SIZES = (5, 128, 128, 128, 2)


def mlp_init(members=1, seed=0):
    """Initial weights of the surrogate members, flat per member in the layout
    W_1 (out x in, row-major), b_1, W_2, b_2, ...: W uniform in
    [-sqrt(6/(in+out)), +sqrt(6/(in+out))] (Glorot and Bengio 2010) from
    SplitMix64, biases zero.  Returns (members, P) float64."""
    flat = []
    for m in range(members):
        parts = []
        ctr = 0
        for l in range(len(MLP_SIZES) - 1):
            fan_in, fan_out = MLP_SIZES[l], MLP_SIZES[l + 1]
            a = math.sqrt(6.0 / (fan_in + fan_out))
            cnt = fan_in * fan_out
            u = uniform_noise(seed * 1000003 + m, np.arange(ctr, ctr + cnt, dtype=np.uint64), 1.0)
            ctr += cnt
            parts.append(a * u)
            parts.append(np.zeros(fan_out))
        flat.append(np.concatenate(parts))
    return np.stack(flat)


def mlp_unflatten(w):
    """Flat member vector -> list of (W, b) in the network's layout."""
    out, o = [], 0
    for l in range(len(MLP_SIZES) - 1):
        i, j = MLP_SIZES[l], MLP_SIZES[l + 1]
        W = np.asarray(w[o:o + i * j]).reshape(j, i)
        o += i * j
        b = np.asarray(w[o:o + j])
        o += j
        out.append((W, b))
    return out


def mlp_flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])
