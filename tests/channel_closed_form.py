"""Closed-form velocity of the two-phase layered power-law channel (Sec. 3.3).

Steady, fully developed flow between walls at |y| = H driven by a body force F
along x: the shear stress balances the force, tau_xy = F |y|, in both fluids.
With k |du/dy|^n = F |y| the outer fluid (|y| > Y_i, index n_o, consistency
k_o) has u = n_o/(n_o+1) (F/k_o)^(1/n_o) (H^((n_o+1)/n_o) - |y|^((n_o+1)/n_o)),
and the inner fluid adds to the interface value u(Y_i) its own profile
n_i/(n_i+1) (F/k_i)^(1/n_i) (Y_i^((n_i+1)/n_i) - |y|^((n_i+1)/n_i)).
The paper's printed formula uses Y_i in place of H in the outer branch, which
gives negative velocities near the walls; this is the force-balance form.
"""
import numpy as np


def branch(n, k, F, a, y):
    e = (n + 1.0) / n
    return n / (n + 1.0) * (F / k) ** (1.0 / n) * (a ** e - np.abs(y) ** e)


def layered_profile(y, H, Yi, F, n_in, k_in, n_out, k_out):
    outer = branch(n_out, k_out, F, H, np.minimum(np.abs(y), H))
    inner = branch(n_out, k_out, F, H, Yi) + branch(n_in, k_in, F, Yi, y)
    return np.where(np.abs(y) < Yi, inner, outer)


def design(n, tau_inner_at_interface, tau_outer, H, umax):
    """Force F and inner consistency k such that the inner fluid has relaxation
    time tau_inner_at_interface at |y| = H/2 (eta = tau / 3 at rho = 1) and the
    centreline velocity is umax."""
    Yi = 0.5 * H
    k_out = tau_outer / 3.0
    eta_i = tau_inner_at_interface / 3.0
    F = 1e-6
    for _ in range(60):
        # eta(Yi) = k gd^(n-1) with gd = F Yi / eta(Yi)
        k = eta_i ** n / (F * Yi) ** (n - 1.0)
        u0 = layered_profile(np.array([0.0]), H, Yi, F, n, k, 1.0, k_out)[0]
        F *= (umax / u0) ** 0.5
    k = eta_i ** n / (F * Yi) ** (n - 1.0)
    return F, k, k_out


def stress_balance_profile(y, eta, F, H):
    """Velocity that balances the body force for a given viscosity profile:
    eta(y) du/dy = -F y, u(+-H) = 0, so u(y) = int_|y|^H F s / eta(s) ds
    (trapezoid between the node centres y, eta constant over the last half
    node to the wall).  Independent of how eta came about, so it checks the
    momentum balance across a diffuse interface whatever the mixture law."""
    half = len(y) // 2
    ys, es = y[half:], eta[half:]
    g = F * ys / es
    u = np.zeros(len(ys))
    u[-1] = F * (H ** 2 - ys[-1] ** 2) / (2.0 * es[-1])
    for j in range(len(ys) - 2, -1, -1):
        u[j] = u[j + 1] + 0.5 * (g[j] + g[j + 1]) * (ys[j + 1] - ys[j])
    return np.concatenate([u[::-1], u])
