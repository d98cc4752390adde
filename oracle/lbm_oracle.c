/*
 * FP64 CPU oracle of the coupled power-law / Cahn-Hilliard lattice Boltzmann
 * step (arXiv 2207.09431, Sec. 2).  TEST INFRASTRUCTURE ONLY: the tests, the
 * smoke check and the benchmark's CPU-baseline leg load it; the product path
 * never does.  It shares no code, header or table with the CUDA library.
 *
 * Style: plain nested loops over nodes, one whole-field pass per quantity,
 * every intermediate field stored in its own array, two population buffers.
 * Nothing is fused or reordered beyond what the equations state.
 *
 * Lattice units dx = dt = c = 1, cs^2 = 1/3 (Sec. 2.2, below Eq. 11).
 *
 * Components.  Three phase fields C1, C2, C3 with C1 + C2 + C3 = 1 (Eq. 1).
 * Component 1 is the (power-law) matrix liquid.  With ncomp == 2 only C1 is
 * transported and C2 == 0 identically (the paper itself zeroes one component
 * for its two-phase cases, Sec. 3.2 / 3.3), so C3 = 1 - C1.  With ncomp == 3,
 * C1 and C2 are transported (Eq. 17-18 are written for i = 1, 2) and
 * C3 = 1 - C1 - C2.
 *
 * Readings where the paper is silent or garbled (each one is applied here and
 * in the CUDA path alike):
 *   R1  mixture laws (Sec. 2.2 calls rho "the density of mixture" without a
 *       law): rho = sum_i c_i rho_i and tau = sum_i c_i tau_i with the weights
 *       c_i = clip(C_i, 0, 1) / sum_j clip(C_j, 0, 1).  The clip matters: the
 *       Cahn-Hilliard bulk values of a curved interface shift by about
 *       xi / (24 R), so C_i dips below 0 inside a bubble, and the unclipped
 *       linear law gives a negative density once that dip exceeds
 *       rho_gas / rho_liquid.
 *   R2  stencils: isotropic gradient 3 sum_a w_a e_a X(x+e_a), isotropic
 *       Laplacian 6 sum_a w_a (X(x+e_a) - X(x)); the (e_a - u).grad X terms
 *       use the directional derivative along e_a (central by default, the
 *       mixed central/biased form when fd_scheme == 1) minus u . isotropic.
 *   R3  p = sum g + (1/2) u . grad(rho) cs^2: Eq. 24 drops the 1/2; taking the
 *       zeroth moment of Eq. 16 gives sum geq = p - (1/2) cs^2 u.grad(rho).
 *   R4  tau_PL = eta / (rho cs^2) with the local mixture rho, clamped to
 *       [tau_min, tau_max] (the truncation of Eq. 33 written on tau); node tau
 *       = sum_i C_i tau_i with tau_1 := tau_PL; the strain rate uses the
 *       previous step's node tau (Sec. 2.3, text after Eq. 32).
 *   R7  the sum inside Eq. 18 runs over a separate index j (same force for
 *       every i).
 *   R8  the variable mobility of Eq. 6 is (D0/Sigma_i) c_i (1 - c_i) with
 *       c_i = clip(C_i, 0, 1): with C_i itself the mobility turns negative
 *       (backward diffusion) wherever C_i leaves [0, 1], which the
 *       Cahn-Hilliard bulk shift of a curved interface does inside every
 *       bubble (C_i ~ -xi/(24 R)); every paper-size case then diverges within
 *       1000 steps.  The variable-mobility term of Eq. 18 is the derivative
 *       of that mobility: the scalar (D0/Sigma_i)(1 - 2 C_i) grad C_i .
 *       grad mu_i where 0 <= C_i <= 1, else 0; it is absent for the constant
 *       mobility.
 *   R9  the destination-side terms of Eq. 18 are added at the node where each
 *       population actually arrives, bounced ones included.
 *   R10 half-way walls at y = -1/2 and y = ny - 1/2; stencils read ghost rows
 *       that mirror the fluid rows (zero normal derivative).
 *   R11 initial populations are the modified equilibria (Eq. 16 and Eq. 20)
 *       of the given C, p, u; initial tau uses a zero strain rate.
 *   R23 Eq. 25 divides by 2 (tau + 1/2) rho cs^2, which is the factor for the
 *       barred populations; Eq. 29 already converts them to f - f^eq with
 *       2 tau / (2 tau + 1).  Applying both under-reads the strain rate by
 *       tau / (tau + 1/2), so D = -Pi / (2 tau rho cs^2) with Pi from Eq. 29.
 *   R27 open x boundaries (the channel of Sec. 3.2 names a velocity inlet and a
 *       convective outlet without their discrete form): stencils read ghost
 *       columns that mirror the fluid columns; the populations entering at
 *       x = 0 come from a ghost column x = -1 whose post-collision g is the
 *       equilibrium at the inlet velocity plus the non-equilibrium part of the
 *       post-collision g of column 0 (non-equilibrium extrapolation,
 *       equilibria w p + rho cs^2 (Gamma - w) without forcing), and whose h is
 *       the equilibrium C_in Gamma at the inlet velocity for the given inflow
 *       composition C_in; the populations entering at x = nx - 1 follow the
 *       convective condition f(t+1) = (f(t) + U f_(nx-2)(t+1)) / (1 + U)
 *       with U the node's x velocity clamped to [0, 1], and then share, by
 *       weight, the shift that brings the node's zeroth moment of g to zero
 *       (a pressure reference: without it the inflow and the extrapolated
 *       outflow do not balance and the pressure level drifts).  Wall rows keep
 *       their bounce-back.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Internal precision.  FP64 is the oracle; the same source compiled with
 * -DORACLE_REAL=float measures the FP32 rounding floor of the scheme (test
 * yardstick only).  Parameters and every API array stay double. */
#ifndef ORACLE_REAL
#define ORACLE_REAL double
#endif

/* Whole-field passes treat every node independently (each node's own sums
 * keep their order), so a build with -fopenmp may share a pass's nodes among
 * threads without changing a single result; without -fopenmp the pragma is
 * ignored.  Only the timed CPU baseline uses that build. */
#define ORC_NODE_LOOP _Pragma("omp parallel for schedule(static)")
typedef ORACLE_REAL real;

typedef struct {
  int nx, ny, ncomp, periodic_y;
  double rho[3];   /* component densities */
  double tau[3];   /* Newtonian relaxation times tau_i = nu_i / cs^2 (Eq. 14) */
  int powerlaw;    /* 1: component 1 follows the truncated power law (Eq. 31, 33) */
  double pl_n, pl_k, tau_min, tau_max;
  double sigma12, sigma13, sigma23, Lambda; /* Eq. 3 */
  double xi;       /* interface width (Eq. 2) */
  double D0;       /* mobility scale (Eq. 6) */
  int mobility;    /* 0 constant, 1 variable (Eq. 6) */
  double gravity;  /* F_b = -rho g j (Eq. 12) */
  double force_x;  /* uniform body-force density along x (drives the channel tests of Sec. 3.2-3.3) */
  int fd_scheme;   /* 0 central, 1 mixed directional differences */
  int open_x;      /* 0 periodic in x; 1 velocity inlet at x = 0, convective outlet at x = nx - 1 (R27) */
  double u_in;     /* inlet velocity along x */
  double c_in[2];  /* composition C_1, C_2 of the inflow */
} orc_params;

/* D2Q9 (Eq. 10, 11): 0 rest, 1-4 = E N W S, 5-8 = NE NW SW SE. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const real W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const real CS2 = 1.0 / 3.0;

typedef struct {
  orc_params p;
  int nh;          /* number of transported order parameters (ncomp - 1) */
  size_t n;        /* nodes */
  long long step;
  real Sig[3], SigT;  /* capillary coefficients Sigma_i and Sigma_T (Sec. 2.1) */
  /* state */
  real *g, *h, *tau;          /* g[9][n], h[nh][9][n], tau[n] (previous-step tau) */
  real *gpost, *hpost;        /* post-collision buffers */
  /* intermediate whole fields, recomputed every step */
  real *C[3], *rho, *lapC[3], *mu[3], *gCx[3], *gCy[3], *grx, *gry;
  real *Fsx, *Fsy, *Fbx, *Fby, *ux, *uy, *pr;
  real *gpx, *gpy, *gmux[3], *gmuy[3], *lapmu[3];
  real *tau_new, *shear, *S[2], *V[2];
  /* per-direction whole fields [9][n]: directional derivatives of rho, C_j, p;
   * forcing terms and modified equilibria of g and h */
  real *drho, *dC[3], *dp, *Phig, *Phih[2], *geqb, *heqb[2];
  /* node index of x + e_a and x + 2 e_a under the ghost rule of reading R10 */
  size_t *nb1, *nb2;
  /* populations of the outlet column before streaming (open x, R27) */
  real *gold, *hold;
} orc_state;

/* ---------------------------------------------------------------- helpers */

static size_t idx(const orc_state *s, int x, int y) { return (size_t)y * s->p.nx + x; }

/* Node index holding the value seen at (x, y): periodic x (or mirror ghost
 * columns for open x, R27), and either periodic y or the mirror ghost rows of
 * reading R10. */
static size_t wrap_index(const orc_state *s, int x, int y) {
  int nx = s->p.nx, ny = s->p.ny;
  if (s->p.open_x) {
    while (x < 0 || x >= nx) {
      if (x < 0) x = -1 - x;
      if (x >= nx) x = 2 * nx - 1 - x;
    }
  } else {
    x = ((x % nx) + nx) % nx;
  }
  if (s->p.periodic_y) {
    y = ((y % ny) + ny) % ny;
  } else {
    while (y < 0 || y >= ny) {
      if (y < 0) y = -1 - y;
      if (y >= ny) y = 2 * ny - 1 - y;
    }
  }
  return idx(s, x, y);
}

/* Value of field f at node k shifted by d * e_a (d = 1 or 2). */
static real at(const orc_state *s, const real *f, size_t k, int a, int d) {
  return f[(d == 1 ? s->nb1 : s->nb2)[(size_t)a * s->n + k]];
}

/* Isotropic gradient (reading R2). */
static void grad_iso(const orc_state *s, const real *f, real *gx, real *gy) {
  ORC_NODE_LOOP
  for (size_t k = 0; k < s->n; ++k) {
    real sx = 0.0, sy = 0.0;
    for (int a = 0; a < 9; ++a) {
      real v = at(s, f, k, a, 1);
      sx += W[a] * EX[a] * v;
      sy += W[a] * EY[a] * v;
    }
    gx[k] = sx / CS2;
    gy[k] = sy / CS2;
  }
}

/* Isotropic Laplacian (reading R2). */
static void lap_iso(const orc_state *s, const real *f, real *out) {
  ORC_NODE_LOOP
  for (size_t k = 0; k < s->n; ++k) {
    real c = f[k], acc = 0.0;
    for (int a = 0; a < 9; ++a) acc += W[a] * (at(s, f, k, a, 1) - c);
    out[k] = 2.0 * acc / CS2;
  }
}

/* Directional derivative e_a . grad X at node (x, y) (reading R2). */
static real dir_deriv(const orc_state *s, const real *f, size_t k, int a) {
  real xp = at(s, f, k, a, 1);
  real xm = at(s, f, k, OPP[a], 1);
  if (s->p.fd_scheme == 0) return 0.5 * (xp - xm);
  /* mixed: average of the central and the second-order biased difference */
  real xpp = at(s, f, k, a, 2);
  real x0 = f[k];
  real central = 0.5 * (xp - xm);
  real biased = 0.5 * (-xpp + 4.0 * xp - 3.0 * x0);
  return 0.5 * (central + biased);
}

/* Gamma_a(u) = f_a^eq / rho (Eq. 9). */
static real Gamma(int a, real ux, real uy) {
  real eu = EX[a] * ux + EY[a] * uy;
  real uu = ux * ux + uy * uy;
  return W[a] * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Partial derivatives of the bulk free energy E0 (Eq. 3) with respect to
 * C1, C2, C3 taken as independent variables. */
static void dE0(const orc_state *s, real C1, real C2, real C3, real d[3]) {
  const real s12 = s->p.sigma12, s13 = s->p.sigma13, s23 = s->p.sigma23, L = s->p.Lambda;
  const real S1 = s->Sig[0], S2 = s->Sig[1], S3 = s->Sig[2];
  real mix = S1 * C1 + S2 * C2 + S3 * C3;
  d[0] = 2.0 * s12 * C1 * C2 * C2 + 2.0 * s13 * C1 * C3 * C3 + C2 * C3 * mix + C1 * C2 * C3 * S1 +
         2.0 * L * C1 * C2 * C2 * C3 * C3;
  d[1] = 2.0 * s12 * C1 * C1 * C2 + 2.0 * s23 * C2 * C3 * C3 + C1 * C3 * mix + C1 * C2 * C3 * S2 +
         2.0 * L * C1 * C1 * C2 * C3 * C3;
  d[2] = 2.0 * s13 * C1 * C1 * C3 + 2.0 * s23 * C2 * C2 * C3 + C1 * C2 * mix + C1 * C2 * C3 * S3 +
         2.0 * L * C1 * C1 * C2 * C2 * C3;
}

/* Power-law relaxation time of component 1 at strain rate gd and local
 * mixture density rho: Eq. 31 and Eq. 32, truncated as in Eq. 33 (reading R4). */
static real tau_powerlaw(const orc_state *s, real gd, real rho) {
  real eta = s->p.pl_k * pow(gd, s->p.pl_n - 1.0);
  real t = eta / (rho * CS2);
  if (!(t <= s->p.tau_max)) t = s->p.tau_max; /* also catches +inf at gd == 0, n < 1 */
  if (t < s->p.tau_min) t = s->p.tau_min;
  return t;
}

/* Mixture weights of reading R1. */
static void mixture_weights(real C1, real C2, real C3, real c[3]) {
  real v[3] = {C1, C2, C3}, sum = 0.0;
  for (int i = 0; i < 3; ++i) {
    c[i] = v[i] < 0.0 ? 0.0 : (v[i] > 1.0 ? 1.0 : v[i]);
    sum += c[i];
  }
  for (int i = 0; i < 3; ++i) c[i] /= sum;
}

static real rho_mixture(const orc_state *s, real C1, real C2, real C3) {
  real c[3];
  mixture_weights(C1, C2, C3, c);
  return c[0] * s->p.rho[0] + c[1] * s->p.rho[1] + c[2] * s->p.rho[2];
}

static real tau_mixture(const orc_state *s, size_t k, real tau1) {
  real c[3];
  mixture_weights(s->C[0][k], s->C[1][k], s->C[2][k], c);
  return c[0] * tau1 + c[1] * s->p.tau[1] + c[2] * s->p.tau[2];
}

/* ------------------------------------------------------------ macroscopic */

/* Moments and chemical potentials of the current populations:
 * C_i (Eq. 22 and Eq. 1), rho (R1), mu_i (Eq. 5), grad C_i, grad rho,
 * u (Eq. 23) and p (Eq. 24 with R3). */
static void compute_macros(orc_state *s) {
  const size_t n = s->n;
  ORC_NODE_LOOP
  for (size_t k = 0; k < n; ++k) {
    real c[2] = {0.0, 0.0};
    for (int i = 0; i < s->nh; ++i)
      for (int a = 0; a < 9; ++a) c[i] += s->h[((size_t)i * 9 + a) * n + k];
    s->C[0][k] = c[0];
    s->C[1][k] = (s->nh == 2) ? c[1] : 0.0;
    s->C[2][k] = 1.0 - s->C[0][k] - s->C[1][k];
    s->rho[k] = rho_mixture(s, s->C[0][k], s->C[1][k], s->C[2][k]);
  }
  for (int i = 0; i < 3; ++i) lap_iso(s, s->C[i], s->lapC[i]);
  ORC_NODE_LOOP
  for (size_t k = 0; k < n; ++k) {
    real d[3];
    dE0(s, s->C[0][k], s->C[1][k], s->C[2][k], d);
    for (int i = 0; i < 3; ++i) {
      real bulk = 0.0;
      for (int j = 0; j < 3; ++j)
        if (j != i) bulk += (d[i] - d[j]) / s->Sig[j];
      s->mu[i][k] = 4.0 * s->SigT / s->p.xi * bulk - 0.75 * s->p.xi * s->Sig[i] * s->lapC[i][k];
    }
  }
  for (int i = 0; i < 3; ++i) grad_iso(s, s->C[i], s->gCx[i], s->gCy[i]);
  grad_iso(s, s->rho, s->grx, s->gry);
  ORC_NODE_LOOP
  for (size_t k = 0; k < n; ++k) {
    real fx = 0.0, fy = 0.0;
    for (int j = 0; j < 3; ++j) {
      fx += s->mu[j][k] * s->gCx[j][k];
      fy += s->mu[j][k] * s->gCy[j][k];
    }
    s->Fsx[k] = fx;
    s->Fsy[k] = fy;
    s->Fbx[k] = s->p.force_x;
    s->Fby[k] = -s->rho[k] * s->p.gravity;
    real mx = 0.0, my = 0.0, m0 = 0.0;
    for (int a = 0; a < 9; ++a) {
      real ga = s->g[(size_t)a * n + k];
      m0 += ga;
      mx += EX[a] * ga;
      my += EY[a] * ga;
    }
    s->ux[k] = (mx / CS2 + 0.5 * (fx + s->Fbx[k])) / s->rho[k];
    s->uy[k] = (my / CS2 + 0.5 * (fy + s->Fby[k])) / s->rho[k];
    s->pr[k] = m0 + 0.5 * CS2 * (s->ux[k] * s->grx[k] + s->uy[k] * s->gry[k]);
  }
}

/* Forcing term of Eq. 14 for direction a at node (x, y):
 * (e_a - u).[grad(rho) cs^2 (Gamma_a - Gamma_a(0)) + (sum_j mu_j grad C_j + F_b) Gamma_a]. */
static real forcing_g(const orc_state *s, size_t k, int a) {
  const size_t n = s->n;
  real ux = s->ux[k], uy = s->uy[k];
  real G = Gamma(a, ux, uy);
  real e_rho = s->drho[(size_t)a * n + k] - (ux * s->grx[k] + uy * s->gry[k]);
  real e_Fs = -(ux * s->Fsx[k] + uy * s->Fsy[k]);
  for (int j = 0; j < 3; ++j) e_Fs += s->mu[j][k] * s->dC[j][(size_t)a * n + k];
  real e_Fb = (EX[a] - ux) * s->Fbx[k] + (EY[a] - uy) * s->Fby[k];
  return e_rho * CS2 * (G - W[a]) + (e_Fs + e_Fb) * G;
}

/* Forcing term of Eq. 18 for order parameter i, direction a at (x, y):
 * (e_a - u).[grad C_i - C_i/(rho cs^2) (grad p - sum_j mu_j grad C_j - F_b)] Gamma_a. */
static real forcing_h(const orc_state *s, int i, size_t k, int a) {
  const size_t n = s->n;
  real ux = s->ux[k], uy = s->uy[k];
  real G = Gamma(a, ux, uy);
  real e_C = s->dC[i][(size_t)a * n + k] - (ux * s->gCx[i][k] + uy * s->gCy[i][k]);
  real e_p = s->dp[(size_t)a * n + k] - (ux * s->gpx[k] + uy * s->gpy[k]);
  real e_Fs = -(ux * s->Fsx[k] + uy * s->Fsy[k]);
  for (int j = 0; j < 3; ++j) e_Fs += s->mu[j][k] * s->dC[j][(size_t)a * n + k];
  real e_Fb = (EX[a] - ux) * s->Fbx[k] + (EY[a] - uy) * s->Fby[k];
  return (e_C - s->C[i][k] / (s->rho[k] * CS2) * (e_p - e_Fs - e_Fb)) * G;
}

/* Directional derivatives along every e_a of rho, C_1..3 and p (reading R2). */
static void directional_fields(orc_state *s) {
  const size_t n = s->n;
  for (int a = 0; a < 9; ++a)
    ORC_NODE_LOOP
    for (size_t k = 0; k < n; ++k) {
      size_t ak = (size_t)a * n + k;
      s->drho[ak] = dir_deriv(s, s->rho, k, a);
      for (int j = 0; j < 3; ++j) s->dC[j][ak] = dir_deriv(s, s->C[j], k, a);
      s->dp[ak] = dir_deriv(s, s->pr, k, a);
    }
}

/* Forcing terms of Eq. 14 and Eq. 18 and the modified equilibria
 *   geq_bar = g^eq - (1/2) forcing,  g^eq = f^eq cs^2 + (p - rho cs^2) Gamma_a(0)
 *   (Eq. 13, 16), and heq_bar = C_i Gamma_a - (1/2) forcing (Eq. 20). */
static void forcing_and_equilibria(orc_state *s) {
  const size_t n = s->n;
  for (int a = 0; a < 9; ++a)
    ORC_NODE_LOOP
    for (size_t k = 0; k < n; ++k) {
      size_t ak = (size_t)a * n + k;
      real G = Gamma(a, s->ux[k], s->uy[k]);
      s->Phig[ak] = forcing_g(s, k, a);
      real feq = s->rho[k] * G;
      real geq = feq * CS2 + (s->pr[k] - s->rho[k] * CS2) * W[a];
      s->geqb[ak] = geq - 0.5 * s->Phig[ak];
      for (int i = 0; i < s->nh; ++i) {
        s->Phih[i][ak] = forcing_h(s, i, k, a);
        s->heqb[i][ak] = s->C[i][k] * G - 0.5 * s->Phih[i][ak];
      }
    }
}

/* ------------------------------------------------------------------ API */

orc_state *orc_create(const orc_params *prm) {
  if (!prm || prm->nx < 1 || prm->ny < 2 || (prm->ncomp != 2 && prm->ncomp != 3)) return NULL;
  if (prm->fd_scheme != 0 && prm->fd_scheme != 1) return NULL;
  if (!prm->periodic_y && prm->fd_scheme == 1 && prm->ny < 3) return NULL;
  if (prm->open_x && prm->nx < 4) return NULL;
  orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
  if (!s) return NULL;
  s->p = *prm;
  s->nh = prm->ncomp - 1;
  s->n = (size_t)prm->nx * prm->ny;
  /* Sigma_i = sigma_ij + sigma_ik - sigma_jk and 3/Sigma_T = sum 1/Sigma_i (Sec. 2.1) */
  s->Sig[0] = prm->sigma12 + prm->sigma13 - prm->sigma23;
  s->Sig[1] = prm->sigma12 + prm->sigma23 - prm->sigma13;
  s->Sig[2] = prm->sigma13 + prm->sigma23 - prm->sigma12;
  if (!(s->Sig[0] > 0 && s->Sig[1] > 0 && s->Sig[2] > 0) || !(prm->xi > 0)) {
    free(s);
    return NULL;
  }
  s->SigT = 3.0 / (1.0 / s->Sig[0] + 1.0 / s->Sig[1] + 1.0 / s->Sig[2]);
  size_t n = s->n;
  s->g = calloc(9 * n, sizeof(real));
  s->gpost = calloc(9 * n, sizeof(real));
  s->h = calloc((size_t)s->nh * 9 * n, sizeof(real));
  s->hpost = calloc((size_t)s->nh * 9 * n, sizeof(real));
  s->tau = calloc(n, sizeof(real));
  real **fields[] = {&s->rho, &s->grx, &s->gry, &s->Fsx, &s->Fsy, &s->Fbx, &s->Fby, &s->ux,
                       &s->uy, &s->pr, &s->gpx, &s->gpy, &s->tau_new, &s->shear};
  for (size_t f = 0; f < sizeof(fields) / sizeof(fields[0]); ++f) *fields[f] = calloc(n, sizeof(real));
  for (int i = 0; i < 3; ++i) {
    s->C[i] = calloc(n, sizeof(real));
    s->lapC[i] = calloc(n, sizeof(real));
    s->mu[i] = calloc(n, sizeof(real));
    s->gCx[i] = calloc(n, sizeof(real));
    s->gCy[i] = calloc(n, sizeof(real));
    s->gmux[i] = calloc(n, sizeof(real));
    s->gmuy[i] = calloc(n, sizeof(real));
    s->lapmu[i] = calloc(n, sizeof(real));
  }
  for (int i = 0; i < 2; ++i) {
    s->S[i] = calloc(n, sizeof(real));
    s->V[i] = calloc(n, sizeof(real));
    s->Phih[i] = calloc(9 * n, sizeof(real));
    s->heqb[i] = calloc(9 * n, sizeof(real));
  }
  s->nb1 = calloc(9 * n, sizeof(size_t));
  s->nb2 = calloc(9 * n, sizeof(size_t));
  for (int a = 0; a < 9; ++a)
    for (int y = 0; y < prm->ny; ++y)
      for (int x = 0; x < prm->nx; ++x) {
        s->nb1[(size_t)a * n + idx(s, x, y)] = wrap_index(s, x + EX[a], y + EY[a]);
        s->nb2[(size_t)a * n + idx(s, x, y)] = wrap_index(s, x + 2 * EX[a], y + 2 * EY[a]);
      }
  s->drho = calloc(9 * n, sizeof(real));
  s->dp = calloc(9 * n, sizeof(real));
  for (int j = 0; j < 3; ++j) s->dC[j] = calloc(9 * n, sizeof(real));
  s->Phig = calloc(9 * n, sizeof(real));
  s->geqb = calloc(9 * n, sizeof(real));
  s->gold = calloc(9 * (size_t)prm->ny, sizeof(real));
  s->hold = calloc((size_t)s->nh * 9 * prm->ny, sizeof(real));
  return s;
}

void orc_destroy(orc_state *s) {
  if (!s) return;
  free(s->g); free(s->gpost); free(s->h); free(s->hpost); free(s->tau);
  real *fields[] = {s->rho, s->grx, s->gry, s->Fsx, s->Fsy, s->Fbx, s->Fby, s->ux,
                      s->uy,  s->pr,  s->gpx, s->gpy, s->tau_new, s->shear};
  for (size_t f = 0; f < sizeof(fields) / sizeof(fields[0]); ++f) free(fields[f]);
  for (int i = 0; i < 3; ++i) {
    free(s->C[i]); free(s->lapC[i]); free(s->mu[i]); free(s->gCx[i]); free(s->gCy[i]);
    free(s->gmux[i]); free(s->gmuy[i]); free(s->lapmu[i]);
  }
  for (int i = 0; i < 2; ++i) { free(s->S[i]); free(s->V[i]); free(s->Phih[i]); free(s->heqb[i]); }
  free(s->drho); free(s->dp); free(s->Phig); free(s->geqb); free(s->nb1); free(s->nb2);
  free(s->gold); free(s->hold);
  for (int j = 0; j < 3; ++j) free(s->dC[j]);
  free(s);
}

/* Initial state from given fields (reading R11).  C holds nh fields of n
 * values (C1, then C2 when ncomp == 3); p, ux, uy may be NULL for zero. */
int orc_set_fields(orc_state *s, const double *C, const double *p, const double *ux, const double *uy) {
  const size_t n = s->n;
  /* Build the macroscopic fields directly from the inputs. */
  for (size_t k = 0; k < n; ++k) {
    s->C[0][k] = C[k];
    s->C[1][k] = (s->nh == 2) ? C[n + k] : 0.0;
    s->C[2][k] = 1.0 - s->C[0][k] - s->C[1][k];
    s->rho[k] = rho_mixture(s, s->C[0][k], s->C[1][k], s->C[2][k]);
    s->pr[k] = p ? p[k] : 0.0;
    s->ux[k] = ux ? ux[k] : 0.0;
    s->uy[k] = uy ? uy[k] : 0.0;
  }
  for (int i = 0; i < 3; ++i) lap_iso(s, s->C[i], s->lapC[i]);
  for (size_t k = 0; k < n; ++k) {
    real d[3];
    dE0(s, s->C[0][k], s->C[1][k], s->C[2][k], d);
    for (int i = 0; i < 3; ++i) {
      real bulk = 0.0;
      for (int j = 0; j < 3; ++j)
        if (j != i) bulk += (d[i] - d[j]) / s->Sig[j];
      s->mu[i][k] = 4.0 * s->SigT / s->p.xi * bulk - 0.75 * s->p.xi * s->Sig[i] * s->lapC[i][k];
    }
  }
  for (int i = 0; i < 3; ++i) grad_iso(s, s->C[i], s->gCx[i], s->gCy[i]);
  grad_iso(s, s->rho, s->grx, s->gry);
  grad_iso(s, s->pr, s->gpx, s->gpy);
  for (size_t k = 0; k < n; ++k) {
    real fx = 0.0, fy = 0.0;
    for (int j = 0; j < 3; ++j) {
      fx += s->mu[j][k] * s->gCx[j][k];
      fy += s->mu[j][k] * s->gCy[j][k];
    }
    s->Fsx[k] = fx;
    s->Fsy[k] = fy;
    s->Fbx[k] = s->p.force_x;
    s->Fby[k] = -s->rho[k] * s->p.gravity;
  }
  directional_fields(s);
  forcing_and_equilibria(s);
  for (size_t k = 0; k < n; ++k) {
    for (int a = 0; a < 9; ++a) {
      s->g[(size_t)a * n + k] = s->geqb[(size_t)a * n + k];
      for (int i = 0; i < s->nh; ++i) s->h[((size_t)i * 9 + a) * n + k] = s->heqb[i][(size_t)a * n + k];
    }
    real tau1 = s->p.powerlaw ? tau_powerlaw(s, 0.0, s->rho[k]) : s->p.tau[0];
    s->tau[k] = tau_mixture(s, k, tau1);
  }
  s->step = 0;
  return 0;
}

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) evaluated at counter i:
 * mix(seed + (i + 1) * golden_gamma). */
static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Bubbles and droplets (Sec. 4.2, Eq. 42): component c gets
 * 0.5 - 0.5 tanh((r - R) / (0.5 xi)) for every disc of that component, with
 * the distance taken periodically along periodic axes, plus uniform noise in
 * [-a, a] from SplitMix64 at counter (c - 1) * n + node; the matrix component 1
 * takes the rest (Eq. 1).  bubbles = nb rows of (cx, cy, R, comp). */
int orc_init_bubbles(orc_state *s, const double *bubbles, int nb, unsigned long long seed, double noise) {
  const size_t n = s->n;
  const int nx = s->p.nx, ny = s->p.ny;
  double *Cc[3];
  int used[3] = {0, 0, 0};
  for (int c = 0; c < 3; ++c) Cc[c] = calloc(n, sizeof(double));
  for (int b = 0; b < nb; ++b) {
    int comp = (int)bubbles[4 * b + 3];
    if (comp < 2 || comp > 3 || (s->nh == 1 && comp != 3)) {
      for (int c = 0; c < 3; ++c) free(Cc[c]);
      return -1;
    }
    used[comp - 1] = 1;
    double cx = bubbles[4 * b], cy = bubbles[4 * b + 1], R = bubbles[4 * b + 2];
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        double dx = fabs(x - cx), dy = fabs(y - cy);
        if (dx > 0.5 * nx) dx = nx - dx;
        if (s->p.periodic_y && dy > 0.5 * ny) dy = ny - dy;
        double r = sqrt(dx * dx + dy * dy);
        Cc[comp - 1][idx(s, x, y)] += 0.5 - 0.5 * tanh((r - R) / (0.5 * s->p.xi));
      }
  }
  for (int c = 1; c < 3; ++c) {
    if (!used[c] || noise == 0.0) continue;
    for (size_t k = 0; k < n; ++k) {
      uint64_t z = splitmix64_at(seed, (uint64_t)c * n + k);
      double u01 = (double)(z >> 11) * (1.0 / 9007199254740992.0);
      Cc[c][k] += noise * (2.0 * u01 - 1.0);
    }
  }
  double *Cin = calloc((size_t)s->nh * n, sizeof(double));
  for (size_t k = 0; k < n; ++k) {
    Cin[k] = 1.0 - Cc[1][k] - Cc[2][k];
    if (s->nh == 2) Cin[n + k] = Cc[1][k];
  }
  int rc = orc_set_fields(s, Cin, NULL, NULL, NULL);
  free(Cin);
  for (int c = 0; c < 3; ++c) free(Cc[c]);
  return rc;
}

/* Populations entering through the open x boundaries (reading R27), after the
 * periodic pull of the streaming loop has written placeholders there.  Wall
 * rows keep the bounce-back of that loop. */
static real geq_plain(int a, real p, real rho, real ux, real uy) {
  return W[a] * p + rho * CS2 * (Gamma(a, ux, uy) - W[a]);
}

static void open_boundaries(orc_state *s) {
  const size_t n = s->n;
  const int nx = s->p.nx, ny = s->p.ny;
  const real uin = s->p.u_in;
  for (int y = 0; y < ny; ++y) {
    /* inlet: directions with e_x = +1 leave the ghost column x = -1 */
    size_t k = idx(s, 0, y);
    for (int a = 0; a < 9; ++a) {
      if (EX[a] != 1) continue;
      int sy = y - EY[a];
      if (!s->p.periodic_y && (sy < 0 || sy >= ny)) continue;
      sy = ((sy % ny) + ny) % ny;
      size_t k0 = idx(s, 0, sy);
      real gpost0 = s->gpost[(size_t)a * n + k0];
      s->g[(size_t)a * n + k] = geq_plain(a, s->pr[k0], s->rho[k0], uin, 0.0) +
                                (gpost0 - geq_plain(a, s->pr[k0], s->rho[k0], s->ux[k0], s->uy[k0]));
      real G = Gamma(a, s->ux[k], s->uy[k]);
      for (int i = 0; i < s->nh; ++i)
        s->h[((size_t)i * 9 + a) * n + k] = s->p.c_in[i] * Gamma(a, uin, 0.0) + 0.5 * (s->S[i][k] + s->V[i][k]) * G;
    }
    /* outlet: directions with e_x = -1 would leave the ghost column x = nx */
    k = idx(s, nx - 1, y);
    size_t kin = idx(s, nx - 2, y);
    real U = s->ux[k];
    U = U < 0.0 ? 0.0 : (U > 1.0 ? 1.0 : U);
    real wsum = 0.0;
    int set[9] = {0};
    for (int a = 0; a < 9; ++a) {
      if (EX[a] != -1) continue;
      int sy = y - EY[a];
      if (!s->p.periodic_y && (sy < 0 || sy >= ny)) continue;
      set[a] = 1;
      wsum += W[a];
      s->g[(size_t)a * n + k] = (s->gold[(size_t)a * ny + y] + U * s->g[(size_t)a * n + kin]) / (1.0 + U);
      for (int i = 0; i < s->nh; ++i) {
        size_t ia = (size_t)i * 9 + a;
        s->h[ia * n + k] = (s->hold[ia * ny + y] + U * s->h[ia * n + kin]) / (1.0 + U);
      }
    }
    /* pressure anchor: the entering populations share, by weight, the shift
     * that brings the node's zeroth moment of g to zero */
    if (wsum > 0.0) {
      real p0 = 0.0;
      for (int a = 0; a < 9; ++a) p0 += s->g[(size_t)a * n + k];
      for (int a = 0; a < 9; ++a)
        if (set[a]) s->g[(size_t)a * n + k] -= p0 * W[a] / wsum;
    }
  }
}

/* One time step: Sec. 2.2-2.3 in the order moments -> mu -> gradients -> u, p
 * -> tau update -> collision of g and h -> streaming with bounce-back and the
 * destination-side terms of Eq. 18. */
static void one_step(orc_state *s) {
  const size_t n = s->n;
  const int nx = s->p.nx, ny = s->p.ny;
  compute_macros(s);
  grad_iso(s, s->pr, s->gpx, s->gpy);
  for (int i = 0; i < s->nh; ++i) {
    grad_iso(s, s->mu[i], s->gmux[i], s->gmuy[i]);
    lap_iso(s, s->mu[i], s->lapmu[i]);
  }
  directional_fields(s);
  forcing_and_equilibria(s);
  /* Strain rate from the non-equilibrium part of g with the previous step's tau
   * (Eq. 25, 26, 29; reading R23) and the new relaxation time (Eq. 31-33,
   * reading R4).  f^neq follows Eq. 29; Eq. 25's denominator 2 (tau + 1/2)
   * rho cs^2 belongs to the barred populations, so with the un-barred f^neq of
   * Eq. 29 it is 2 tau rho cs^2 (the two forms give the same D). */
  ORC_NODE_LOOP
  for (size_t k = 0; k < n; ++k) {
    real tp = s->tau[k];
    real Pxx = 0.0, Pyy = 0.0, Pxy = 0.0;
    for (int a = 0; a < 9; ++a) {
      real fneq = (1.0 / CS2) * (2.0 * tp / (2.0 * tp + 1.0)) *
                    (s->g[(size_t)a * n + k] - s->geqb[(size_t)a * n + k]);
      Pxx += fneq * EX[a] * EX[a];
      Pyy += fneq * EY[a] * EY[a];
      Pxy += fneq * EX[a] * EY[a];
    }
    real den = 2.0 * tp * s->rho[k] * CS2;
    real Dxx = -Pxx / den, Dyy = -Pyy / den, Dxy = -Pxy / den;
    real gd = sqrt(2.0 * (Dxx * Dxx + Dyy * Dyy + 2.0 * Dxy * Dxy));
    s->shear[k] = gd;
    real tau1 = s->p.powerlaw ? tau_powerlaw(s, gd, s->rho[k]) : s->p.tau[0];
    s->tau_new[k] = tau_mixture(s, k, tau1);
  }
  /* Diffusion sources of Eq. 18: S_i = D_i lap(mu_i) (Eq. 6) and, for the
   * variable mobility, V_i of Eq. 21 (reading R8). */
  for (int i = 0; i < s->nh; ++i)
    ORC_NODE_LOOP
    for (size_t k = 0; k < n; ++k) {
      real Ci = s->C[i][k];
      real D = s->p.D0 / s->Sig[i];
      /* reading R8: the mobility of Eq. 6 with C_i clipped to [0, 1], and V_i
       * the derivative of that mobility, zero where C_i lies outside */
      real ci = Ci < 0.0 ? 0.0 : (Ci > 1.0 ? 1.0 : Ci);
      int inside = Ci >= 0.0 && Ci <= 1.0;
      if (s->p.mobility == 1) D *= ci * (1.0 - ci);
      s->S[i][k] = D * s->lapmu[i][k];
      s->V[i][k] = (s->p.mobility == 1 && inside)
                       ? s->p.D0 / s->Sig[i] * (1.0 - 2.0 * Ci) *
                             (s->gCx[i][k] * s->gmux[i][k] + s->gCy[i][k] * s->gmuy[i][k])
                       : 0.0;
    }
  /* Collision (Eq. 14 and Eq. 18 with tau_h = 0.5, source-side terms). */
  const real tau_h = 0.5;
  for (int a = 0; a < 9; ++a)
    ORC_NODE_LOOP
    for (size_t k = 0; k < n; ++k) {
      size_t ak = (size_t)a * n + k;
      real ga = s->g[ak];
      s->gpost[ak] = ga - (ga - s->geqb[ak]) / (s->tau_new[k] + 0.5) + s->Phig[ak];
      real G = Gamma(a, s->ux[k], s->uy[k]);
      for (int i = 0; i < s->nh; ++i) {
        size_t iak = (size_t)i * 9 * n + ak;
        real ha = s->h[iak];
        s->hpost[iak] = ha - (ha - s->heqb[i][ak]) / (tau_h + 0.5) + s->Phih[i][ak] +
                        0.5 * (s->S[i][k] + s->V[i][k]) * G;
      }
    }
  if (s->p.open_x)
    for (int y = 0; y < ny; ++y)
      for (int a = 0; a < 9; ++a) {
        size_t k = idx(s, nx - 1, y);
        s->gold[(size_t)a * ny + y] = s->g[(size_t)a * n + k];
        for (int i = 0; i < s->nh; ++i)
          s->hold[((size_t)i * 9 + a) * ny + y] = s->h[((size_t)i * 9 + a) * n + k];
      }
  /* Streaming: population a arriving at y left y - e_a; across a wall it is
   * the population leaving y in the opposite direction (half-way bounce-back),
   * then the destination-side terms of Eq. 18 at the arrival node (R9). */
  ORC_NODE_LOOP
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = idx(s, x, y);
      for (int a = 0; a < 9; ++a) {
        int sx = ((x - EX[a]) % nx + nx) % nx;
        int sy = y - EY[a];
        size_t src;
        int aa;
        if (s->p.periodic_y) {
          sy = ((sy % ny) + ny) % ny;
          src = idx(s, sx, sy);
          aa = a;
        } else if (sy < 0 || sy >= ny) {
          src = k;
          aa = OPP[a];
        } else {
          src = idx(s, sx, sy);
          aa = a;
        }
        s->g[(size_t)a * n + k] = s->gpost[(size_t)aa * n + src];
        real G = Gamma(a, s->ux[k], s->uy[k]);
        for (int i = 0; i < s->nh; ++i)
          s->h[((size_t)i * 9 + a) * n + k] =
              s->hpost[((size_t)i * 9 + aa) * n + src] + 0.5 * (s->S[i][k] + s->V[i][k]) * G;
      }
    }
  if (s->p.open_x) open_boundaries(s);
  memcpy(s->tau, s->tau_new, n * sizeof(real));
  s->step += 1;
}

int orc_step(orc_state *s, long long nsteps) {
  for (long long t = 0; t < nsteps; ++t) one_step(s);
  return 0;
}

long long orc_get_step(const orc_state *s) { return s->step; }

static void copy_out(double *out, const real *src, size_t n) {
  for (size_t k = 0; k < n; ++k) out[k] = (double)src[k];
}

/* Field ids (macroscopic fields are those of the current populations). */
enum {
  ORC_C1 = 0, ORC_C2 = 1, ORC_C3 = 2, ORC_RHO = 3, ORC_P = 4, ORC_UX = 5, ORC_UY = 6,
  ORC_TAU = 7, ORC_MU1 = 8, ORC_MU2 = 9, ORC_MU3 = 10, ORC_G = 11, ORC_H = 12,
  ORC_SHEAR = 13, ORC_S = 14, ORC_V = 15
};

/* Copies a field to out.  Returns the number of values, or -1. */
long long orc_get_field(orc_state *s, int id, double *out) {
  const size_t n = s->n;
  switch (id) {
    case ORC_G: copy_out(out, s->g, 9 * n); return (long long)(9 * n);
    case ORC_H: copy_out(out, s->h, (size_t)s->nh * 9 * n); return (long long)(s->nh * 9 * n);
    case ORC_TAU: copy_out(out, s->tau, n); return (long long)n;
    case ORC_SHEAR: copy_out(out, s->shear, n); return (long long)n;
    case ORC_S:
      for (int i = 0; i < s->nh; ++i) copy_out(out + (size_t)i * n, s->S[i], n);
      return (long long)(s->nh * n);
    case ORC_V:
      for (int i = 0; i < s->nh; ++i) copy_out(out + (size_t)i * n, s->V[i], n);
      return (long long)(s->nh * n);
    default: break;
  }
  compute_macros(s);
  const real *src = NULL;
  switch (id) {
    case ORC_C1: src = s->C[0]; break;
    case ORC_C2: src = s->C[1]; break;
    case ORC_C3: src = s->C[2]; break;
    case ORC_RHO: src = s->rho; break;
    case ORC_P: src = s->pr; break;
    case ORC_UX: src = s->ux; break;
    case ORC_UY: src = s->uy; break;
    case ORC_MU1: src = s->mu[0]; break;
    case ORC_MU2: src = s->mu[1]; break;
    case ORC_MU3: src = s->mu[2]; break;
    default: return -1;
  }
  copy_out(out, src, n);
  return (long long)n;
}

/* Raw observable sums of the current state (Sec. 3.1 thresholded masses,
 * Sec. 4.2 Eq. 43-44 averages, bubble extents for the aspect ratio of Eq. 41):
 *  out[0..2]  M_i = sum C_i
 *  out[3..5]  sum C_i over nodes with C_i > 0.5
 *  out[6..10] sum C_g, sum C_g x, sum C_g y, sum C_g ux, sum C_g uy
 *  out[11..14] xmin, xmax, ymin, ymax of nodes with C_g > 0.5 (-1 if none) */
void orc_observables(orc_state *s, int gas_comp, double *out) {
  compute_macros(s);
  for (int i = 0; i < 15; ++i) out[i] = 0.0;
  double xmin = -1, xmax = -1, ymin = -1, ymax = -1;
  const real *Cg = s->C[gas_comp - 1];
  for (int y = 0; y < s->p.ny; ++y)
    for (int x = 0; x < s->p.nx; ++x) {
      size_t k = idx(s, x, y);
      for (int i = 0; i < 3; ++i) {
        out[i] += s->C[i][k];
        if (s->C[i][k] > 0.5) out[3 + i] += s->C[i][k];
      }
      double c = Cg[k];
      out[6] += c;
      out[7] += c * x;
      out[8] += c * y;
      out[9] += c * s->ux[k];
      out[10] += c * s->uy[k];
      if (c > 0.5) {
        if (xmin < 0 || x < xmin) xmin = x;
        if (xmax < 0 || x > xmax) xmax = x;
        if (ymin < 0 || y < ymin) ymin = y;
        if (ymax < 0 || y > ymax) ymax = y;
      }
    }
  out[11] = xmin; out[12] = xmax; out[13] = ymin; out[14] = ymax;
}
