// Multi-pass form of the coupled D2Q9 step (arXiv 2207.09431, Sec. 2.2-2.3):
//   k_moments  C_i = sum_a h_a^i                         (Eq. 22)
//   k_fields   rho, mu (Eq. 5), u (Eq. 23), p (Eq. 24/R3), new tau (Eq. 25-33)
//   k_sources  S_i + V_i = D_i lap(mu_i) + variable-mobility term (Eq. 6, 21)
//   k_collide  collision of g (Eq. 14) and h (Eq. 18), pushed to the
//              neighbours with half-way bounce-back and the destination-side
//              source term (R9)
// The intermediate fields live in scratch planes carved from the caller's
// arena.  One thread per node; all arithmetic FP32.
#include "lbm_device.cuh"
#include "lbm_kernels.h"

namespace lbm {

namespace {

// Order parameter j (0..2) at node (x, y) of the scratch planes (C3 derived).
struct CReader {
  const float *C;
  long long plane;
  int nh;
  __device__ __forceinline__ void at(long long k, float out[3]) const {
    out[0] = C[k];
    out[1] = (nh == 2) ? C[plane + k] : 0.0f;
    out[2] = 1.0f - out[0] - out[1];
  }
};

__device__ __forceinline__ long long node_index(const DevParams &P, int x, int y) {
  return (long long)y * P.pitch + x;
}

// Column seen at x: periodic, or (open x) the mirror ghost columns beyond the
// inlet and outlet, for offsets of at most two columns.
__device__ __forceinline__ int column_of(const DevParams &P, int x) {
  if (!P.open_x) return wrap_x(x, P.nx);
  if (x < 0) x = -1 - x;
  if (x >= P.nx) x = 2 * P.nx - 1 - x;
  return x;
}

__device__ __forceinline__ long long shifted(const DevParams &P, int x, int y, int dx, int dy) {
  return node_index(P, column_of(P, x + dx), wrap_y(y + dy, P.ny, P.periodic_y));
}

// Directional derivative e_a . grad X from samples X(x - e), X(x), X(x + e),
// X(x + 2e) (R2; mixed = mean of central and second-order biased forms).
// The final scaling is a separate rounding (__fmul_rn), never fused into the
// caller's next addition, whether or not this is inlined.
__device__ __forceinline__ float dir_deriv(int scheme, float xm, float x0, float xp, float xpp) {
  if (scheme == 0) return __fmul_rn(0.5f, xp - xm);
  return __fmul_rn(0.25f, -xpp + 5.0f * xp - 3.0f * x0 - xm);
}

// Everything the forcing terms need at one node.
struct NodeCtx {
  float C[3], rho, ux, uy, p, mu[3];
  float gC[3][2], grho[2], gp[2], Fs[2], Fb[2];
  float dC[3][9], drho[9], dp[9];
};

// Gathers C (radius 1 or 2), rho (from C), p (radius 1 or 2) around (x, y).
// Inlined, so that NodeCtx stays in registers.
__device__ __forceinline__ void gather_gradients(const DevParams &P, const CReader &cr, const float *pf, int x, int y,
                                 NodeCtx &n) {
  const long long k0 = node_index(P, x, y);
  float Cn[9][3], rn[9], pn[9];
  for (int a = 0; a < 9; ++a) {
    long long k = shifted(P, x, y, ex(a), ey(a));
    cr.at(k, Cn[a]);
    rn[a] = rho_of(P, Cn[a][0], Cn[a][1], Cn[a][2]);
    pn[a] = pf[k];
  }
  (void)k0;
  for (int j = 0; j < 3; ++j) {
    n.C[j] = Cn[0][j];
    float sx = 0.f, sy = 0.f;
    for (int a = 0; a < 9; ++a) {
      sx += wt(a) * ex(a) * Cn[a][j];
      sy += wt(a) * ey(a) * Cn[a][j];
    }
    n.gC[j][0] = 3.0f * sx;
    n.gC[j][1] = 3.0f * sy;
  }
  n.rho = rn[0];
  n.p = pn[0];
  {
    float sx = 0.f, sy = 0.f, qx = 0.f, qy = 0.f;
    for (int a = 0; a < 9; ++a) {
      sx += wt(a) * ex(a) * rn[a];
      sy += wt(a) * ey(a) * rn[a];
      qx += wt(a) * ex(a) * pn[a];
      qy += wt(a) * ey(a) * pn[a];
    }
    n.grho[0] = 3.0f * sx;
    n.grho[1] = 3.0f * sy;
    n.gp[0] = 3.0f * qx;
    n.gp[1] = 3.0f * qy;
  }
  for (int a = 0; a < 9; ++a) {
    const int o = opp(a);
    float C2e[3] = {0.f, 0.f, 0.f}, r2e = 0.f, p2e = 0.f;
    if (P.fd_scheme == 1) {
      long long k2 = shifted(P, x, y, 2 * ex(a), 2 * ey(a));
      cr.at(k2, C2e);
      r2e = rho_of(P, C2e[0], C2e[1], C2e[2]);
      p2e = pf[k2];
    }
    for (int j = 0; j < 3; ++j) n.dC[j][a] = dir_deriv(P.fd_scheme, Cn[o][j], Cn[0][j], Cn[a][j], C2e[j]);
    n.drho[a] = dir_deriv(P.fd_scheme, rn[o], rn[0], rn[a], r2e);
    n.dp[a] = dir_deriv(P.fd_scheme, pn[o], pn[0], pn[a], p2e);
  }
}

// Forcing of Eq. 14 for direction a.
__device__ __forceinline__ float phi_g(const NodeCtx &n, int a, float G) {
  float e_rho = n.drho[a] - (n.ux * n.grho[0] + n.uy * n.grho[1]);
  float e_Fs = n.mu[0] * n.dC[0][a] + n.mu[1] * n.dC[1][a] + n.mu[2] * n.dC[2][a] -
               (n.ux * n.Fs[0] + n.uy * n.Fs[1]);
  float e_Fb = (ex(a) - n.ux) * n.Fb[0] + (ey(a) - n.uy) * n.Fb[1];
  return e_rho * kCs2 * (G - wt(a)) + (e_Fs + e_Fb) * G;
}

// Forcing of Eq. 18 for order parameter i, direction a.
__device__ __forceinline__ float phi_h(const NodeCtx &n, int i, int a, float G) {
  float e_C = n.dC[i][a] - (n.ux * n.gC[i][0] + n.uy * n.gC[i][1]);
  float e_p = n.dp[a] - (n.ux * n.gp[0] + n.uy * n.gp[1]);
  float e_Fs = n.mu[0] * n.dC[0][a] + n.mu[1] * n.dC[1][a] + n.mu[2] * n.dC[2][a] -
               (n.ux * n.Fs[0] + n.uy * n.Fs[1]);
  float e_Fb = (ex(a) - n.ux) * n.Fb[0] + (ey(a) - n.uy) * n.Fb[1];
  return (e_C - n.C[i] / (n.rho * kCs2) * (e_p - e_Fs - e_Fb)) * G;
}

__device__ __forceinline__ bool node_of_thread(const DevParams &P, int &x, int &y) {
  x = blockIdx.x * blockDim.x + threadIdx.x;
  y = blockIdx.y * blockDim.y + threadIdx.y;
  return x < P.nx && y < P.ny;
}

}  // namespace

__global__ void k_moments(DevParams P, const float *__restrict__ h, float *__restrict__ C) {
  int x, y;
  if (!node_of_thread(P, x, y)) return;
  const long long k = node_index(P, x, y);
  for (int i = 0; i < P.nh; ++i) {
    float s = 0.f;
    for (int a = 0; a < 9; ++a) s += h[pop_index(k, i * 9 + a, 9 * P.nh)];
    C[(long long)i * P.plane + k] = s;
  }
}

// The fields of node (x, y) from the order parameters around it and its g
// (Eq. 5, 22-24): C and rho at the node and its neighbours, grad C, lap C,
// grad rho, mu_1..3, the forces, the moments of g and u.  Shared by k_fields
// and the observables, so that both see the same velocity.
template <int NH>
__device__ __forceinline__ void fields_core(const DevParams &P, const float *__restrict__ Cf,
                                            const float *__restrict__ g, int x, int y, long long k, NodeCtx &n,
                                            float (&Cn)[9][3], float (&rn)[9], float (&ga)[9], float &m0) {
  CReader cr{Cf, P.plane, NH};
  for (int a = 0; a < 9; ++a) {
    long long kk = shifted(P, x, y, ex(a), ey(a));
    cr.at(kk, Cn[a]);
    rn[a] = rho_of(P, Cn[a][0], Cn[a][1], Cn[a][2]);
  }
  float lapC[3];
  for (int j = 0; j < 3; ++j) {
    n.C[j] = Cn[0][j];
    float sx = 0.f, sy = 0.f, lp = 0.f;
    for (int a = 0; a < 9; ++a) {
      sx += wt(a) * ex(a) * Cn[a][j];
      sy += wt(a) * ey(a) * Cn[a][j];
      lp += wt(a) * (Cn[a][j] - Cn[0][j]);
    }
    n.gC[j][0] = 3.0f * sx;
    n.gC[j][1] = 3.0f * sy;
    lapC[j] = 6.0f * lp;
  }
  n.rho = rn[0];
  {
    float sx = 0.f, sy = 0.f;
    for (int a = 0; a < 9; ++a) {
      sx += wt(a) * ex(a) * rn[a];
      sy += wt(a) * ey(a) * rn[a];
    }
    n.grho[0] = 3.0f * sx;
    n.grho[1] = 3.0f * sy;
  }
  chem_potentials(P, n.C, lapC, n.mu);
  n.Fs[0] = n.mu[0] * n.gC[0][0] + n.mu[1] * n.gC[1][0] + n.mu[2] * n.gC[2][0];
  n.Fs[1] = n.mu[0] * n.gC[0][1] + n.mu[1] * n.gC[1][1] + n.mu[2] * n.gC[2][1];
  n.Fb[0] = P.force_x;
  n.Fb[1] = -n.rho * P.gravity;
  m0 = 0.f;
  float mx = 0.f, my = 0.f;
  for (int a = 0; a < 9; ++a) {
    ga[a] = g[pop_index(k, a, 9)];
    m0 += ga[a];
    mx += ex(a) * ga[a];
    my += ey(a) * ga[a];
  }
  n.ux = (3.0f * mx + 0.5f * (n.Fs[0] + n.Fb[0])) / n.rho;
  n.uy = (3.0f * my + 0.5f * (n.Fs[1] + n.Fb[1])) / n.rho;
}

// rho, mu_1..3, u, p and (if write_tau) the new relaxation time and strain rate.
template <int NH>
__global__ void k_fields(DevParams P, const float *__restrict__ Cf, const float *__restrict__ g,
                         const float *__restrict__ tau_prev, float *__restrict__ mu, float *__restrict__ pf,
                         float *__restrict__ uxf, float *__restrict__ uyf, float *__restrict__ tau_new,
                         float *__restrict__ shear, unsigned *err, int write_tau) {
  int x, y;
  if (!node_of_thread(P, x, y)) return;
  const long long k = node_index(P, x, y);
  CReader cr{Cf, P.plane, NH};
  float Cn[9][3], rn[9], ga[9], m0;
  NodeCtx n;
  fields_core<NH>(P, Cf, g, x, y, k, n, Cn, rn, ga, m0);
  n.p = m0 + 0.5f * kCs2 * (n.ux * n.grho[0] + n.uy * n.grho[1]);
  for (int j = 0; j < 3; ++j) mu[(long long)j * P.plane + k] = n.mu[j];
  pf[k] = n.p;
  uxf[k] = n.ux;
  uyf[k] = n.uy;
  if (!write_tau) return;
  // directional derivatives of rho and C (the g forcing has no p derivative)
  for (int a = 0; a < 9; ++a) {
    const int o = opp(a);
    float C2e[3] = {0.f, 0.f, 0.f}, r2e = 0.f;
    if (P.fd_scheme == 1) {
      cr.at(shifted(P, x, y, 2 * ex(a), 2 * ey(a)), C2e);
      r2e = rho_of(P, C2e[0], C2e[1], C2e[2]);
    }
    for (int j = 0; j < 3; ++j) n.dC[j][a] = dir_deriv(P.fd_scheme, Cn[o][j], Cn[0][j], Cn[a][j], C2e[j]);
    n.drho[a] = dir_deriv(P.fd_scheme, rn[o], rn[0], rn[a], r2e);
  }
  // strain rate from the non-equilibrium part with the previous tau (R23)
  const float tp = tau_prev[k];
  const float fac = 3.0f * (2.0f * tp / (2.0f * tp + 1.0f));
  float Pxx = 0.f, Pyy = 0.f, Pxy = 0.f;
  for (int a = 0; a < 9; ++a) {
    float G = gamma_a(a, n.ux, n.uy);
    float geq = wt(a) * n.p + n.rho * kCs2 * (G - wt(a)) - 0.5f * phi_g(n, a, G);
    float fneq = fac * (ga[a] - geq);
    Pxx += fneq * (float)(ex(a) * ex(a));
    Pyy += fneq * (float)(ey(a) * ey(a));
    Pxy += fneq * (float)(ex(a) * ey(a));
  }
  const float den = 2.0f * tp * n.rho * kCs2;
  const float Dxx = -Pxx / den, Dyy = -Pyy / den, Dxy = -Pxy / den;
  const float gd = sqrtf(2.0f * (Dxx * Dxx + Dyy * Dyy + 2.0f * Dxy * Dxy));
  const float tau1 = P.powerlaw ? tau_powerlaw(P, gd, 1.0f / n.rho) : P.tau[0];
  const float tn = tau_mix(P, n.C[0], n.C[1], n.C[2], tau1);
  tau_new[k] = tn;
  shear[k] = gd;
  if (!(isfinite(n.rho) && isfinite(n.p) && isfinite(n.ux) && isfinite(n.uy) && isfinite(tn))) atomicOr(err, 1u);
}

// S_i + V_i (Eq. 6, 18, 21; R8) for every transported order parameter.
__global__ void k_sources(DevParams P, const float *__restrict__ Cf, const float *__restrict__ mu,
                          float *__restrict__ SV) {
  int x, y;
  if (!node_of_thread(P, x, y)) return;
  const long long k = node_index(P, x, y);
  for (int i = 0; i < P.nh; ++i) {
    const float *Ci = Cf + (long long)i * P.plane;
    const float *mi = mu + (long long)i * P.plane;
    float gcx = 0.f, gcy = 0.f, gmx = 0.f, gmy = 0.f, lm = 0.f;
    const float m0 = mi[k];
    for (int a = 0; a < 9; ++a) {
      long long kk = shifted(P, x, y, ex(a), ey(a));
      float cv = Ci[kk], mv = mi[kk];
      gcx += wt(a) * ex(a) * cv;
      gcy += wt(a) * ey(a) * cv;
      gmx += wt(a) * ex(a) * mv;
      gmy += wt(a) * ey(a) * mv;
      lm += wt(a) * (mv - m0);
    }
    const float lapmu = 6.0f * lm;
    const float C = Ci[k];
    const float D0s = P.d0_sig[i];
    float s;
    if (P.mobility == 1) {
      // mobility with C clipped to [0, 1] and its derivative (reading R8)
      const float cc = fminf(fmaxf(C, 0.0f), 1.0f);
      const float dv = (C >= 0.0f && C <= 1.0f)
                           ? D0s * (1.0f - 2.0f * C) * (3.0f * gcx * 3.0f * gmx + 3.0f * gcy * 3.0f * gmy)
                           : 0.0f;
      s = D0s * cc * (1.0f - cc) * lapmu + dv;
    } else {
      s = D0s * lapmu;
    }
    SV[(long long)i * P.plane + k] = s;
  }
}

// Collision of g (Eq. 14) and h (Eq. 18, tau_h = 1/2) at each node, pushed to
// x + e_a; populations that would cross a wall return to x in the opposite
// direction.  With tau_h = 1/2 the BGK step of Eq. 18 replaces h by its
// modified equilibrium, so h itself is not read: h* = C Gamma + Phi/2 + SV Gamma/2.
template <int NH>
__global__ void k_collide(DevParams P, const float *__restrict__ g, const float *__restrict__ Cf,
                          const float *__restrict__ mu, const float *__restrict__ pf, const float *__restrict__ uxf,
                          const float *__restrict__ uyf, const float *__restrict__ tau_new,
                          const float *__restrict__ SV, float *__restrict__ g_out, float *__restrict__ h_out) {
  int x, y;
  if (!node_of_thread(P, x, y)) return;
  const long long k = node_index(P, x, y);
  CReader cr{Cf, P.plane, NH};
  NodeCtx n;
  gather_gradients(P, cr, pf, x, y, n);
  n.ux = uxf[k];
  n.uy = uyf[k];
  for (int j = 0; j < 3; ++j) n.mu[j] = mu[(long long)j * P.plane + k];
  n.Fs[0] = n.mu[0] * n.gC[0][0] + n.mu[1] * n.gC[1][0] + n.mu[2] * n.gC[2][0];
  n.Fs[1] = n.mu[0] * n.gC[0][1] + n.mu[1] * n.gC[1][1] + n.mu[2] * n.gC[2][1];
  n.Fb[0] = P.force_x;
  n.Fb[1] = -n.rho * P.gravity;
  const float omega = 1.0f / (tau_new[k] + 0.5f);
  float sv[2] = {0.f, 0.f};
#pragma unroll
  for (int i = 0; i < 2; ++i)
    if (i < NH) sv[i] = SV[(long long)i * P.plane + k];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const float G = gamma_a(a, n.ux, n.uy);
    const float pg = phi_g(n, a, G);
    const float geq = wt(a) * n.p + n.rho * kCs2 * (G - wt(a)) - 0.5f * pg;
    const float gv = g[pop_index(k, a, 9)];
    const float gstar = gv - omega * (gv - geq) + pg;
    // destination
    int dx = x + ex(a), dy = y + ey(a);
    int da = a;
    long long kd;
    if (!P.periodic_y && (dy < 0 || dy >= P.ny)) {
      kd = k;
      da = opp(a);
    } else if (P.open_x && (dx < 0 || dx >= P.nx)) {
      continue;  // leaves through the inlet or outlet; k_open_x sets what enters
    } else {
      kd = node_index(P, wrap_x(dx, P.nx), P.periodic_y ? wrap_y(dy, P.ny, 1) : dy);
    }
    g_out[pop_index(kd, da, 9)] = gstar;
    const float Gd = gamma_a(da, uxf[kd], uyf[kd]);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      if (i >= NH) break;
      const float ph = phi_h(n, i, a, G);
      const float hstar = n.C[i] * G + 0.5f * ph + 0.5f * sv[i] * G;
      h_out[pop_index(kd, i * 9 + da, 9 * NH)] = hstar + 0.5f * SV[(long long)i * P.plane + kd] * Gd;
    }
  }
}

// Populations entering through the open x boundaries, after k_collide (one
// thread per row).  Inlet (x = 0, e_x = +1): g from a ghost column x = -1 whose
// post-collision g is the equilibrium w p + rho cs^2 (Gamma - w) at (u_in, 0)
// plus the non-equilibrium part of column 0's post-collision g (which k_collide
// stored at column 1), h the equilibrium c_in Gamma(u_in) plus the node's
// destination-side term.  Outlet (x = nx - 1, e_x = -1): the convective
// condition f(t+1) = (f(t) + U f_(nx-2)(t+1)) / (1 + U), U the node's x velocity
// clamped to [0, 1], then the shift (shared by weight among the entering g)
// that sets the node's pressure sum_a g_a to 0.  Wall rows keep bounce-back.
__global__ void k_open_x(DevParams P, const float *__restrict__ g_old, const float *__restrict__ h_old,
                         const float *__restrict__ Cf, const float *__restrict__ pf, const float *__restrict__ uxf,
                         const float *__restrict__ uyf, const float *__restrict__ SV, float *__restrict__ g_out,
                         float *__restrict__ h_out) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= P.ny) return;
  const long long pl = P.plane;
  CReader cr{Cf, P.plane, P.nh};
  // inlet
  {
    const long long k = node_index(P, 0, y), k1 = node_index(P, 1, y);
    for (int a = 0; a < 9; ++a) {
      if (ex(a) != 1) continue;
      int sy = y - ey(a);
      if (!P.periodic_y && (sy < 0 || sy >= P.ny)) continue;
      sy = wrap_y(sy, P.ny, P.periodic_y);
      const long long k0 = node_index(P, 0, sy);
      float c[3];
      cr.at(k0, c);
      const float rho = rho_of(P, c[0], c[1], c[2]);
      const float p = pf[k0];
      const float w = wt(a);
      const float eq_in = w * p + rho * kCs2 * (gamma_a(a, P.u_in, 0.0f) - w);
      const float eq_0 = w * p + rho * kCs2 * (gamma_a(a, uxf[k0], uyf[k0]) - w);
      g_out[pop_index(k, a, 9)] = eq_in + (g_out[pop_index(k1, a, 9)] - eq_0);
      const float G = gamma_a(a, uxf[k], uyf[k]);
      const float Gin = gamma_a(a, P.u_in, 0.0f);
      for (int i = 0; i < P.nh; ++i)
        h_out[pop_index(k, i * 9 + a, 9 * P.nh)] = P.c_in[i] * Gin + 0.5f * SV[(long long)i * pl + k] * G;
    }
  }
  // outlet
  {
    const long long k = node_index(P, P.nx - 1, y), kin = node_index(P, P.nx - 2, y);
    const float U = fminf(fmaxf(uxf[k], 0.0f), 1.0f);
    const float inv = 1.0f / (1.0f + U);
    float wsum = 0.f;
    bool set[9];
    for (int a = 0; a < 9; ++a) {
      set[a] = false;
      if (ex(a) != -1) continue;
      const int sy = y - ey(a);
      if (!P.periodic_y && (sy < 0 || sy >= P.ny)) continue;
      set[a] = true;
      wsum += wt(a);
      g_out[pop_index(k, a, 9)] = (g_old[pop_index(k, a, 9)] + U * g_out[pop_index(kin, a, 9)]) * inv;
      for (int i = 0; i < P.nh; ++i) {
        const int q = i * 9 + a, nq = 9 * P.nh;
        h_out[pop_index(k, q, nq)] = (h_old[pop_index(k, q, nq)] + U * h_out[pop_index(kin, q, nq)]) * inv;
      }
    }
    if (wsum > 0.f) {
      float p0 = 0.f;
      for (int a = 0; a < 9; ++a) p0 += g_out[pop_index(k, a, 9)];
      for (int a = 0; a < 9; ++a)
        if (set[a]) g_out[pop_index(k, a, 9)] -= p0 * wt(a) / wsum;
    }
  }
}

// Modified equilibria (Eq. 16, 20) of given C, p, u, and tau at zero strain
// rate (reading R11).  C, p, u are in the scratch planes.
template <int NH>
__global__ void k_init(DevParams P, const float *__restrict__ Cf, const float *__restrict__ pf,
                       const float *__restrict__ uxf, const float *__restrict__ uyf, float *__restrict__ g,
                       float *__restrict__ h, float *__restrict__ tau, int y0, int y1) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = y0 + blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= P.nx || y >= y1) return;
  const long long k = node_index(P, x, y);
  CReader cr{Cf, P.plane, NH};
  NodeCtx n;
  gather_gradients(P, cr, pf, x, y, n);
  float Cn[9][3], lapC[3];
  for (int a = 0; a < 9; ++a) cr.at(shifted(P, x, y, ex(a), ey(a)), Cn[a]);
  for (int j = 0; j < 3; ++j) {
    float lp = 0.f;
    for (int a = 0; a < 9; ++a) lp += wt(a) * (Cn[a][j] - Cn[0][j]);
    lapC[j] = 6.0f * lp;
  }
  chem_potentials(P, n.C, lapC, n.mu);
  n.ux = uxf[k];
  n.uy = uyf[k];
  n.Fs[0] = n.mu[0] * n.gC[0][0] + n.mu[1] * n.gC[1][0] + n.mu[2] * n.gC[2][0];
  n.Fs[1] = n.mu[0] * n.gC[0][1] + n.mu[1] * n.gC[1][1] + n.mu[2] * n.gC[2][1];
  n.Fb[0] = P.force_x;
  n.Fb[1] = -n.rho * P.gravity;
  for (int a = 0; a < 9; ++a) {
    const float G = gamma_a(a, n.ux, n.uy);
    g[pop_index(k, a, 9)] = wt(a) * n.p + n.rho * kCs2 * (G - wt(a)) - 0.5f * phi_g(n, a, G);
    if (h) {
#pragma unroll
      for (int i = 0; i < 2; ++i)
        if (i < NH) h[pop_index(k, i * 9 + a, 9 * NH)] = n.C[i] * G - 0.5f * phi_h(n, i, a, G);
    }
  }
  const float tau1 = P.powerlaw ? tau_powerlaw(P, 0.0f, 1.0f / n.rho) : P.tau[0];
  tau[k] = tau_mix(P, n.C[0], n.C[1], n.C[2], tau1);
}

// Observable sums (Sec. 3.1; Eq. 43-44 inputs) in FP64: acc[0..10] = M1..3,
// M1..3 above 0.5, A, sum C_g x, sum C_g y, sum C_g ux, sum C_g uy; ext[0..3] =
// xmin, -xmax, ymin, -ymax of C_g > 0.5.  Each thread walks rows (a block per
// row, grid-stride) accumulating its nodes, then warp shuffles, one
// shared-memory pass per block and one atomic per block and quantity.
constexpr int kObsThreads = 256;

// Dense FP64 host-layout planes (ny x nx each) into pitched FP32 planes, one
// thread per column of the pitch (the padding columns get 0); FP64 -> FP32
// rounds to nearest, as a host conversion does.
__global__ void k_planes_from_f64(DevParams P, const double *__restrict__ src, float *__restrict__ dst,
                                  int nplanes, int y0) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = y0 + blockIdx.y;
  if (x >= P.pitch) return;
  for (int q = 0; q < nplanes; ++q)
    dst[(long long)q * P.plane + (long long)y * P.pitch + x] =
        x < P.nx ? (float)src[((long long)q * P.ny + y) * P.nx + x] : 0.0f;
}

// A running FP32 sum with Neumaier's compensation: c collects the rounding
// error of every addition (and, in add_prod, the exact error of the product,
// from fmaf), so s + c, taken in FP64, is the exact sum of a short run of
// terms up to a relative error of order n 2^-48.  Explicit _rn intrinsics keep
// the compiler from fusing a product into the next addition.
struct CompSum {
  float s, c;
  __device__ __forceinline__ void add(float v) {
    const float t = __fadd_rn(s, v);
    c = __fadd_rn(c, fabsf(s) >= fabsf(v) ? __fadd_rn(__fsub_rn(s, t), v) : __fadd_rn(__fsub_rn(v, t), s));
    s = t;
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    add(p);
    c = __fadd_rn(c, __fmaf_rn(a, b, -p));
  }
};

// Nodes a thread sums in FP32 (compensated) before it adds the run to its
// FP64 totals: GB300's FP64 pipe runs at a small fraction of its FP32 rate, so
// one FP64 addition per node and quantity bound the kernel.
constexpr int kObsRun = 16;

// The observable sums straight from the state: C from the C planes, u
// computed at each node as k_fields computes it (fields_core), without
// writing the macro fields.
template <int NH>
__global__ void __launch_bounds__(kObsThreads) k_obs_direct(DevParams P, const float *__restrict__ Cf,
                                                            const float *__restrict__ g, int gas_comp,
                                                            double *acc, int *ext) {
  double v[11];
  CompSum r[11];
  for (int q = 0; q < 11; ++q) {
    v[q] = 0.0;
    r[q] = {0.f, 0.f};
  }
  int run = 0;
  auto flush = [&]() {
    for (int q = 0; q < 11; ++q) {
      v[q] += (double)r[q].s + (double)r[q].c;
      r[q] = {0.f, 0.f};
    }
    run = 0;
  };
  int e[4] = {0x7fffffff, 0x7fffffff, 0x7fffffff, 0x7fffffff};
  for (int y = blockIdx.x; y < P.ny; y += gridDim.x) {
    for (int x = threadIdx.x; x < P.nx; x += blockDim.x) {
      const long long k = node_index(P, x, y);
      NodeCtx n;
      float Cn[9][3], rn[9], ga[9], m0;
      fields_core<NH>(P, Cf, g, x, y, k, n, Cn, rn, ga, m0);
      for (int i = 0; i < 3; ++i) {
        r[i].add(n.C[i]);
        r[3 + i].add(n.C[i] > 0.5f ? n.C[i] : 0.0f);
      }
      // C of the gas component, selected without indexing (keeps n in registers)
      const float cg = gas_comp == 1 ? n.C[0] : (gas_comp == 2 ? n.C[1] : n.C[2]);
      r[6].add(cg);
      r[7].add_prod(cg, (float)x);  // x, y < 2^24: exact in FP32
      r[8].add_prod(cg, (float)y);
      r[9].add_prod(cg, n.ux);
      r[10].add_prod(cg, n.uy);
      if (++run == kObsRun) flush();
      if (cg > 0.5f) {
        e[0] = min(e[0], x);
        e[1] = min(e[1], -x);
        e[2] = min(e[2], y);
        e[3] = min(e[3], -y);
      }
    }
  }
  flush();
  for (int off = 16; off > 0; off >>= 1) {
    for (int q = 0; q < 11; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
    for (int q = 0; q < 4; ++q) e[q] = min(e[q], __shfl_down_sync(0xffffffffu, e[q], off));
  }
  __shared__ double sv[kObsThreads / 32][11];
  __shared__ int se[kObsThreads / 32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    for (int q = 0; q < 11; ++q) sv[warp][q] = v[q];
    for (int q = 0; q < 4; ++q) se[warp][q] = e[q];
  }
  __syncthreads();
  if (threadIdx.x < 11) {
    double t = 0.0;
    for (int w = 0; w < kObsThreads / 32; ++w) t += sv[w][threadIdx.x];
    atomicAdd(&acc[threadIdx.x], t);
  } else if (threadIdx.x >= 32 && threadIdx.x < 36) {
    const int q = threadIdx.x - 32;
    int m = 0x7fffffff;
    for (int w = 0; w < kObsThreads / 32; ++w) m = min(m, se[w][q]);
    if (m != 0x7fffffff) atomicMin(&ext[q], m);
  }
}

static dim3 node_grid(const DevParams &P, dim3 blk) {
  return dim3((P.nx + blk.x - 1) / blk.x, (P.ny + blk.y - 1) / blk.y);
}

void launch_split_step(const DevParams &P, const StepBuffers &B, cudaStream_t s, cudaEvent_t *ev) {
  const dim3 blk(32, 8);
  const dim3 grd = node_grid(P, blk);
  if (ev) cudaEventRecord(ev[0], s);
  k_moments<<<grd, blk, 0, s>>>(P, B.h_in, B.C);
  if (ev) cudaEventRecord(ev[1], s);
  if (P.nh == 1)
    k_fields<1><<<grd, blk, 0, s>>>(P, B.C, B.g_in, B.tau_in, B.mu, B.p, B.ux, B.uy, B.tau_out, B.shear, B.err, 1);
  else
    k_fields<2><<<grd, blk, 0, s>>>(P, B.C, B.g_in, B.tau_in, B.mu, B.p, B.ux, B.uy, B.tau_out, B.shear, B.err, 1);
  if (ev) cudaEventRecord(ev[2], s);
  k_sources<<<grd, blk, 0, s>>>(P, B.C, B.mu, B.SV);
  if (ev) cudaEventRecord(ev[3], s);
  if (P.nh == 1)
    k_collide<1><<<grd, blk, 0, s>>>(P, B.g_in, B.C, B.mu, B.p, B.ux, B.uy, B.tau_out, B.SV, B.g_out, B.h_out);
  else
    k_collide<2><<<grd, blk, 0, s>>>(P, B.g_in, B.C, B.mu, B.p, B.ux, B.uy, B.tau_out, B.SV, B.g_out, B.h_out);
  if (P.open_x)
    k_open_x<<<(P.ny + 127) / 128, 128, 0, s>>>(P, B.g_in, B.h_in, B.C, B.p, B.ux, B.uy, B.SV, B.g_out, B.h_out);
  if (ev) cudaEventRecord(ev[4], s);
}

void launch_macros(const DevParams &P, const StepBuffers &B, cudaStream_t s) {
  const dim3 blk(32, 8);
  const dim3 grd = node_grid(P, blk);
  if (B.h_in) k_moments<<<grd, blk, 0, s>>>(P, B.h_in, B.C);  // null: the state holds C
  if (P.nh == 1)
    k_fields<1><<<grd, blk, 0, s>>>(P, B.C, B.g_in, B.tau_in, B.mu, B.p, B.ux, B.uy, nullptr, nullptr, B.err, 0);
  else
    k_fields<2><<<grd, blk, 0, s>>>(P, B.C, B.g_in, B.tau_in, B.mu, B.p, B.ux, B.uy, nullptr, nullptr, B.err, 0);
}

// Rows [y0, y1) of nplanes dense FP64 planes into the pitched FP32 planes.
cudaError_t launch_planes_from_f64_rows(const DevParams &P, const double *src, float *dst, int nplanes, int y0,
                                        int y1, cudaStream_t s) {
  if (y1 <= y0) return cudaSuccess;
  k_planes_from_f64<<<dim3((P.pitch + 127) / 128, y1 - y0), 128, 0, s>>>(P, src, dst, nplanes, y0);
  return cudaGetLastError();
}

cudaError_t launch_planes_from_f64(const DevParams &P, const double *src, float *dst, int nplanes, cudaStream_t s) {
  return launch_planes_from_f64_rows(P, src, dst, nplanes, 0, P.ny, s);
}

// Initial equilibria of rows [y0, y1) (they read C and p two rows beyond).
void launch_init_rows(const DevParams &P, const StepBuffers &B, int y0, int y1, cudaStream_t s) {
  const dim3 blk(32, 8);
  const dim3 grd((P.nx + blk.x - 1) / blk.x, (y1 - y0 + blk.y - 1) / blk.y);
  if (y1 <= y0) return;
  if (P.nh == 1)
    k_init<1><<<grd, blk, 0, s>>>(P, B.C, B.p, B.ux, B.uy, B.g_out, B.h_out, B.tau_out, y0, y1);
  else
    k_init<2><<<grd, blk, 0, s>>>(P, B.C, B.p, B.ux, B.uy, B.g_out, B.h_out, B.tau_out, y0, y1);
}

void launch_init(const DevParams &P, const StepBuffers &B, cudaStream_t s) { launch_init_rows(P, B, 0, P.ny, s); }

void launch_moments(const DevParams &P, const float *h, float *C, cudaStream_t s) {
  const dim3 blk(32, 8);
  k_moments<<<node_grid(P, blk), blk, 0, s>>>(P, h, C);
}

void launch_observables_direct(const DevParams &P, const float *C, const float *g, int gas_comp, double *acc,
                               int *ext, cudaStream_t s) {
  const int blocks = P.ny < 1216 ? P.ny : 1216;  // 8 per SM on 152 SMs, at most one per row
  if (P.nh == 1)
    k_obs_direct<1><<<blocks, kObsThreads, 0, s>>>(P, C, g, gas_comp, acc, ext);
  else
    k_obs_direct<2><<<blocks, kObsThreads, 0, s>>>(P, C, g, gas_comp, acc, ext);
}


}  // namespace lbm
