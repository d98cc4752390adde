"""Independent vectorised NumPy restatement of one LB time step (test helper).

Written from the paper's equations (arXiv 2207.09431, Sec. 2.1-2.3, Eq. 1-33)
and the readings listed in the oracle's header, in a different arrangement from
the C oracle: whole-array operations, ghost rows built with ``np.pad``,
streaming by ``np.roll`` with the bounce-back fixed afterwards.  It is used
only on tiny grids to brute-force check the oracle.
"""
from __future__ import annotations

import numpy as np

E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
Wt = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
OPPOSITE = [0, 3, 4, 1, 2, 7, 8, 5, 6]
cs2 = 1.0 / 3.0


def _pad(X, periodic_y, r=2):
    Xp = np.pad(X, ((0, 0), (r, r)), mode="wrap")
    return np.pad(Xp, ((r, r), (0, 0)), mode="wrap" if periodic_y else "symmetric")


def _shift(Xp, dx, dy, ny, nx, r=2):
    """Values X(x + dx, y + dy) for every node, from a padded array."""
    return Xp[r + dy:r + dy + ny, r + dx:r + dx + nx]


def _grad(X, py):
    ny, nx = X.shape
    Xp = _pad(X, py)
    gx = sum(Wt[a] * E[a, 0] * _shift(Xp, E[a, 0], E[a, 1], ny, nx) for a in range(9)) / cs2
    gy = sum(Wt[a] * E[a, 1] * _shift(Xp, E[a, 0], E[a, 1], ny, nx) for a in range(9)) / cs2
    return gx, gy


def _lap(X, py):
    ny, nx = X.shape
    Xp = _pad(X, py)
    return 2.0 / cs2 * sum(Wt[a] * (_shift(Xp, E[a, 0], E[a, 1], ny, nx) - X) for a in range(9))


def _dir(X, a, py, scheme):
    ny, nx = X.shape
    Xp = _pad(X, py)
    ex, ey = E[a]
    fwd = _shift(Xp, ex, ey, ny, nx)
    bwd = _shift(Xp, -ex, -ey, ny, nx)
    if scheme == 0:
        return 0.5 * (fwd - bwd)
    fwd2 = _shift(Xp, 2 * ex, 2 * ey, ny, nx)
    return 0.25 * (-fwd2 + 5 * fwd - 3 * X - bwd)


def _gamma(ux, uy):
    out = []
    for a in range(9):
        eu = E[a, 0] * ux + E[a, 1] * uy
        out.append(Wt[a] * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * (ux ** 2 + uy ** 2)))
    return np.array(out)


def _clip_weights(C):
    c = np.clip(C, 0.0, 1.0)
    return c / c.sum(axis=0)


def macros(prm, g, h):
    """Fields of the current populations: C (3, ny, nx), rho, mu (3, ...), u, p."""
    nh = prm["ncomp"] - 1
    py = bool(prm["periodic_y"])
    ny, nx = g.shape[1:]
    C = np.zeros((3, ny, nx))
    C[0] = h[0].sum(axis=0)
    if nh == 2:
        C[1] = h[1].sum(axis=0)
    C[2] = 1.0 - C[0] - C[1]
    return _fields_from_C(prm, C, g=g)


def _fields_from_C(prm, C, g=None, p=None, ux=None, uy=None):
    py = bool(prm["periodic_y"])
    s12, s13, s23, Lam = prm["sigma12"], prm["sigma13"], prm["sigma23"], prm["Lambda"]
    Sig = np.array([s12 + s13 - s23, s12 + s23 - s13, s13 + s23 - s12])
    SigT = 3.0 / np.sum(1.0 / Sig)
    rho_i = np.array(prm["rho"])
    cw = _clip_weights(C)
    rho = np.tensordot(rho_i, cw, axes=1)
    C1, C2, C3 = C
    mix = Sig[0] * C1 + Sig[1] * C2 + Sig[2] * C3
    # partial derivatives of E0 (Eq. 3)
    dE = np.array([
        2 * s12 * C1 * C2 ** 2 + 2 * s13 * C1 * C3 ** 2 + C2 * C3 * (mix + Sig[0] * C1)
        + 2 * Lam * C1 * C2 ** 2 * C3 ** 2,
        2 * s12 * C1 ** 2 * C2 + 2 * s23 * C2 * C3 ** 2 + C1 * C3 * (mix + Sig[1] * C2)
        + 2 * Lam * C1 ** 2 * C2 * C3 ** 2,
        2 * s13 * C1 ** 2 * C3 + 2 * s23 * C2 ** 2 * C3 + C1 * C2 * (mix + Sig[2] * C3)
        + 2 * Lam * C1 ** 2 * C2 ** 2 * C3,
    ])
    mu = np.zeros_like(C)
    for i in range(3):
        others = [j for j in range(3) if j != i]
        bulk = sum((dE[i] - dE[j]) / Sig[j] for j in others)
        mu[i] = 4 * SigT / prm["xi"] * bulk - 0.75 * prm["xi"] * Sig[i] * _lap(C[i], py)
    gC = [np.array(_grad(C[i], py)) for i in range(3)]
    grho = np.array(_grad(rho, py))
    Fs = sum(mu[i] * gC[i] for i in range(3))
    Fb = np.array([np.full_like(rho, prm["force_x"]), -rho * prm["gravity"]])
    if g is not None:
        mom = np.tensordot(E.T.astype(float), g, axes=1)
        u = (mom / cs2 + 0.5 * (Fs + Fb)) / rho
        p = g.sum(axis=0) + 0.5 * cs2 * (u * grho).sum(axis=0)
    else:
        u = np.array([ux, uy])
    return dict(C=C, cw=cw, rho=rho, mu=mu, gC=gC, grho=grho, Fs=Fs, Fb=Fb, u=u, p=p, Sig=Sig)


def _forcings(prm, F):
    py = bool(prm["periodic_y"])
    scheme = prm["fd_scheme"]
    nh = prm["ncomp"] - 1
    u = F["u"]
    G = _gamma(u[0], u[1])
    gp = np.array(_grad(F["p"], py))
    Phig = np.zeros_like(G)
    Phih = np.zeros((nh,) + G.shape)
    for a in range(9):
        eu_minus = lambda dX, grad: dX - (u * grad).sum(axis=0)  # noqa: E731
        dC = [_dir(F["C"][j], a, py, scheme) for j in range(3)]
        eFs = sum(F["mu"][j] * dC[j] for j in range(3)) - (u * F["Fs"]).sum(axis=0)
        eFb = ((E[a][:, None, None] - u) * F["Fb"]).sum(axis=0)
        erho = eu_minus(_dir(F["rho"], a, py, scheme), F["grho"])
        Phig[a] = erho * cs2 * (G[a] - Wt[a]) + (eFs + eFb) * G[a]
        ep = eu_minus(_dir(F["p"], a, py, scheme), gp)
        for i in range(nh):
            eC = eu_minus(dC[i], F["gC"][i])
            Phih[i, a] = (eC - F["C"][i] / (F["rho"] * cs2) * (ep - eFs - eFb)) * G[a]
    geq = np.array([Wt[a] * F["p"] + F["rho"] * cs2 * (G[a] - Wt[a]) for a in range(9)]) - 0.5 * Phig
    heq = np.array([F["C"][i] * G for i in range(nh)]) - 0.5 * Phih
    return G, Phig, Phih, geq, heq


def _tau_of(prm, cw, rho, shear):
    if prm["powerlaw"]:
        with np.errstate(divide="ignore"):
            eta = prm["pl_k"] * shear ** (prm["pl_n"] - 1.0)
        tpl = np.clip(eta / (rho * cs2), prm["tau_min"], prm["tau_max"])
    else:
        tpl = np.full_like(rho, prm["tau"][0])
    return cw[0] * tpl + cw[1] * prm["tau"][1] + cw[2] * prm["tau"][2]


def init_state(prm, Cin):
    """Populations of the modified equilibria at u = 0, p = 0 (reading R11)."""
    ny, nx = Cin.shape[1:]
    C = np.zeros((3, ny, nx))
    C[0] = Cin[0]
    if prm["ncomp"] == 3:
        C[1] = Cin[1]
    C[2] = 1 - C[0] - C[1]
    z = np.zeros((ny, nx))
    F = _fields_from_C(prm, C, p=z.copy(), ux=z.copy(), uy=z.copy())
    _, _, _, geq, heq = _forcings(prm, F)
    tau = _tau_of(prm, F["cw"], F["rho"], np.zeros_like(F["rho"]))
    return geq.copy(), heq.copy(), tau


def step(prm, g, h, tau):
    """One time step; returns new (g, h, tau)."""
    py = bool(prm["periodic_y"])
    nh = prm["ncomp"] - 1
    ny, nx = g.shape[1:]
    F = macros(prm, g, h)
    G, Phig, Phih, geq, heq = _forcings(prm, F)
    # strain rate (Eq. 25-29 with reading R23)
    fneq = (1 / cs2) * (2 * tau / (2 * tau + 1)) * (g - geq)
    Pxx = np.tensordot(E[:, 0] ** 2 * 1.0, fneq, axes=1)
    Pyy = np.tensordot(E[:, 1] ** 2 * 1.0, fneq, axes=1)
    Pxy = np.tensordot(E[:, 0] * E[:, 1] * 1.0, fneq, axes=1)
    Dm = -np.array([Pxx, Pyy, Pxy]) / (2 * tau * F["rho"] * cs2)
    shear = np.sqrt(2 * (Dm[0] ** 2 + Dm[1] ** 2 + 2 * Dm[2] ** 2))
    tau_new = _tau_of(prm, F["cw"], F["rho"], shear)
    # collision
    gpost = g - (g - geq) / (tau_new + 0.5) + Phig
    src = np.zeros((nh, ny, nx))
    for i in range(nh):
        D = prm["D0"] / F["Sig"][i]
        lapmu = _lap(F["mu"][i], py)
        if prm["mobility"] == 1:
            # mobility of C clipped to [0, 1]; its derivative where C is inside
            gmu = np.array(_grad(F["mu"][i], py))
            Ci = F["C"][i]
            c = np.clip(Ci, 0.0, 1.0)
            inside = (Ci >= 0.0) & (Ci <= 1.0)
            src[i] = D * c * (1 - c) * lapmu + np.where(inside, D * (1 - 2 * Ci) * (F["gC"][i] * gmu).sum(axis=0),
                                                        0.0)
        else:
            src[i] = D * lapmu
    hpost = np.array([h[i] - (h[i] - heq[i]) / 1.0 + Phih[i] + 0.5 * src[i] * G for i in range(nh)])
    # streaming (push by roll), then bounce-back at the walls
    gn = np.empty_like(g)
    hn = np.empty_like(h)
    for a in range(9):
        ex, ey = E[a]
        gn[a] = np.roll(np.roll(gpost[a], ey, axis=0), ex, axis=1)
        for i in range(nh):
            hn[i, a] = np.roll(np.roll(hpost[i, a], ey, axis=0), ex, axis=1)
        if not py:
            rows = [0] if ey == 1 else ([ny - 1] if ey == -1 else [])
            for r in rows:
                gn[a, r] = gpost[OPPOSITE[a], r]
                for i in range(nh):
                    hn[i, a, r] = hpost[i, OPPOSITE[a], r]
    for i in range(nh):
        hn[i] += 0.5 * src[i] * G
    return gn, hn, tau_new
