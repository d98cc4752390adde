// Per-node arithmetic of the fused step (arXiv 2207.09431, Sec. 2.2-2.3),
// shared by every kernel that computes it (tile and row-sweep forms), so that
// all launch configurations produce the same values.  The callers gather the
// neighbour values from their own shared-memory layouts; index a of a
// neighbour array is the D2Q9 direction (value at x + e_a, a = 0 the node).
#pragma once

#include <cuda_fp16.h>

#include "lbm_device.cuh"
#include "lbm_kernels.h"

namespace lbm {

// Periodic index for offsets of at most one period (the common case) with a
// modulo fallback for lattices smaller than a tile.
__device__ __forceinline__ int wrap_periodic(int v, int n) {
  if (v < 0) v += n;
  if (v >= n) v -= n;
  if (v < 0 || v >= n) v = ((v % n) + n) % n;
  return v;
}

// Row read for row gy: periodic, or mirrored about the half-way walls (R10);
// rows far outside (only in unused slots of a ragged tile) are clamped.
__device__ __forceinline__ int row_read(int gy, int ny, int periodic) {
  if (periodic) return wrap_periodic(gy, ny);
  if (gy < 0) gy = -1 - gy;
  if (gy >= ny) gy = 2 * ny - 1 - gy;
  return gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);
}

// Mixture density and C of a node of the 3-ring (Eq. 1, 22; reading R1).
template <int NH>
__device__ __forceinline__ float node_rho(const DevParams &P, const float (&c)[NH]) {
  const float C2 = NH == 2 ? c[NH - 1] : 0.0f;
  return rho_of(P, c[0], C2, 1.0f - c[0] - C2);
}

// Fields of a node of the 2-ring: moments of g, isotropic gradients of C and
// rho, chemical potentials (Eq. 5), velocity (Eq. 23) and pressure (Eq. 24,
// reading R3).
struct NodeFields {
  float mu[3], gCx[3], gCy[3];
  float rx, ry, ux, uy, p;
};

template <int NH>
__device__ __forceinline__ void node_fields(const DevParams &P, const float (&g)[9], const float (&cn)[NH][9],
                                            const float (&rn)[9], NodeFields &f) {
  float m0 = 0.f, mx = 0.f, my = 0.f;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    m0 += g[a];
    mx += ex(a) * g[a];
    my += ey(a) * g[a];
  }
  float C[3], lap[3];
  float rx = 0.f, ry = 0.f;
  float cc[3][9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    cc[0][a] = cn[0][a];
    cc[1][a] = NH == 2 ? cn[NH - 1][a] : 0.f;
    cc[2][a] = 1.0f - cc[0][a] - cc[1][a];
    rx += wt(a) * ex(a) * rn[a];
    ry += wt(a) * ey(a) * rn[a];
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    float sx = 0.f, sy = 0.f, lp = 0.f;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      sx += wt(a) * ex(a) * cc[j][a];
      sy += wt(a) * ey(a) * cc[j][a];
      lp += wt(a) * (cc[j][a] - cc[j][0]);
    }
    C[j] = cc[j][0];
    f.gCx[j] = 3.0f * sx;
    f.gCy[j] = 3.0f * sy;
    lap[j] = 6.0f * lp;
  }
  // C_3 = 1 - C_1 - C_2 (Eq. 1): its stencils are minus the sum of the others'
  C[2] = cc[2][0];
  f.gCx[2] = -(f.gCx[0] + f.gCx[1]);
  f.gCy[2] = -(f.gCy[0] + f.gCy[1]);
  lap[2] = -(lap[0] + lap[1]);
  rx *= 3.0f;
  ry *= 3.0f;
  chem_potentials(P, C, lap, f.mu);
  const float Fsx = f.mu[0] * f.gCx[0] + f.mu[1] * f.gCx[1] + f.mu[2] * f.gCx[2];
  const float Fsy = f.mu[0] * f.gCy[0] + f.mu[1] * f.gCy[1] + f.mu[2] * f.gCy[2];
  const float rho = rn[0];
  const float irho = __fdividef(1.0f, rho);
  f.ux = (3.0f * mx + 0.5f * (Fsx + P.force_x)) * irho;
  f.uy = (3.0f * my + 0.5f * (Fsy - rho * P.gravity)) * irho;
  f.p = m0 + 0.5f * kCs2 * (f.ux * rx + f.uy * ry);
  f.rx = rx;
  f.ry = ry;
}

// Collision of a node of the 1-ring: diffusion sources (Eq. 6, 21, reading
// R8), h* of every direction (Eq. 18, tau_h = 1/2), strain rate from the
// non-equilibrium part with the previous tau (Eq. 25-29, reading R23), the new
// tau (Eq. 31-33, R4) and g* of every direction (Eq. 14).
struct NodeCenter {
  float ux, uy, p, rho, grx, gry;
  float dmu[2], gCx[2], gCy[2];
};

template <int NH>
__device__ __forceinline__ void node_collide(const DevParams &P, const NodeCenter &c, const float (&pn)[9],
                                             const float (&rn)[9], const float (&cn)[NH][9],
                                             const float (&mun)[NH][9], float (&g)[9], float tau_prev,
                                             float (&hs)[NH][9], float (&sv)[NH], float &tn, float &gd2) {
  const float ux = c.ux, uy = c.uy, p = c.p, rho = c.rho;
  const float irho = __fdividef(1.0f, rho);
  float px = 0.f, py = 0.f, mgx[NH], mgy[NH], mlap[NH];
#pragma unroll
  for (int i = 0; i < NH; ++i) mgx[i] = mgy[i] = mlap[i] = 0.f;
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    px += wt(a) * ex(a) * pn[a];
    py += wt(a) * ey(a) * pn[a];
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      const float m = mun[i][a];
      mgx[i] += wt(a) * ex(a) * m;
      mgy[i] += wt(a) * ey(a) * m;
      mlap[i] += wt(a) * (m - mun[i][0]);
    }
  }
  px *= 3.0f;
  py *= 3.0f;
  float Fsx = 0.f, Fsy = 0.f, Cc[NH], kap[NH], udC[NH];
#pragma unroll
  for (int i = 0; i < NH; ++i) {
    const float gcx = c.gCx[i], gcy = c.gCy[i];
    Fsx += c.dmu[i] * gcx;
    Fsy += c.dmu[i] * gcy;
    Cc[i] = cn[i][0];
    const float D0s = P.d0_sig[i];
    const float lapmu = 6.0f * mlap[i];
    if (P.mobility == 1)
      sv[i] = D0s * Cc[i] * (1.0f - Cc[i]) * lapmu +
              D0s * (1.0f - 2.0f * Cc[i]) * 3.0f * (gcx * mgx[i] + gcy * mgy[i]);
    else
      sv[i] = D0s * lapmu;
    kap[i] = 3.0f * Cc[i] * irho;  // C_i / (rho cs^2)
    udC[i] = ux * gcx + uy * gcy;
  }
  const float Fby = -rho * P.gravity;
  const float udr = ux * c.grx + uy * c.gry;
  const float udFs = ux * Fsx + uy * Fsy;
  const float udFb = ux * P.force_x + uy * Fby;
  const float udp = ux * px + uy * py;
  const float uu = ux * ux + uy * uy;
  const float rcs2 = rho * kCs2;
  // central directional derivatives along e_a (x + e_a and x - e_a); those
  // of opposite directions are negatives of each other
  float drv[9], dpv[9], dCv[NH][9];
  drv[0] = dpv[0] = 0.f;
#pragma unroll
  for (int i = 0; i < NH; ++i) dCv[i][0] = 0.f;
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    if (a == 1 || a == 2 || a == 5 || a == 6) {
      drv[a] = 0.5f * (rn[a] - rn[opp(a)]);
      dpv[a] = 0.5f * (pn[a] - pn[opp(a)]);
      drv[opp(a)] = -drv[a];
      dpv[opp(a)] = -dpv[a];
#pragma unroll
      for (int i = 0; i < NH; ++i) {
        dCv[i][a] = 0.5f * (cn[i][a] - cn[i][opp(a)]);
        dCv[i][opp(a)] = -dCv[i][a];
      }
    }
  }
  // Per direction a, with Gamma_a = w_a T_a, T_a = 1 - 1.5 u.u + 4.5 (e.u)^2 + 3 e.u:
  //   E_a   = (e_a - u).(F_s + F_b) = sum_i (mu_i - mu_3) d_a C_i + e_a.F_b - u.F
  //   ph_a  = (d_a rho - u.grad rho) cs^2 (Gamma_a - w_a) + E_a Gamma_a        (Eq. 14-16)
  //   geq_a = w_a p + rho cs^2 (Gamma_a - w_a) - ph_a / 2
  //   h*_a  = C_i Gamma_a + [d_a C_i - u.grad C_i
  //            - C_i/(rho cs^2) (d_a p - u.grad p - E_a)] Gamma_a / 2 + S_i Gamma_a / 2   (Eq. 18-20)
  // e.u, e.F_b and the directional derivatives change sign between opposite
  // directions, (e.u)^2 does not: those are formed once per pair.
  const float S0 = 1.0f - 1.5f * uu;
  const float uF = udFs + udFb;
  const float udr3 = udr * kCs2;
  float euv[9], Bv[9], Xv[9];
  euv[0] = 0.f;
  Bv[0] = S0;
  Xv[0] = 0.f;
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    if (a == 1 || a == 2 || a == 5 || a == 6) {
      const float eu = ex(a) * ux + ey(a) * uy;
      const float Bp = fmaf(4.5f * eu, eu, S0);
      float X = ex(a) * P.force_x + ey(a) * Fby;
#pragma unroll
      for (int i = 0; i < NH; ++i) X = fmaf(c.dmu[i], dCv[i][a], X);
      euv[a] = eu;
      euv[opp(a)] = -eu;
      Bv[a] = Bv[opp(a)] = Bp;
      Xv[a] = X;
      Xv[opp(a)] = -X;
    }
  }
  float eqf[9];
  float Pxx = 0.f, Pyy = 0.f, Pxy = 0.f;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const float exa = (float)ex(a), eya = (float)ey(a), w = wt(a);
    const float G = w * fmaf(3.0f, euv[a], Bv[a]);
    const float Gw = G - w;
    const float E = Xv[a] - uF;
    const float ph = fmaf(fmaf(drv[a], kCs2, -udr3), Gw, E * G);
    const float geq = fmaf(-0.5f, ph, fmaf(rcs2, Gw, w * p));
    const float fneq = g[a] - geq;
    g[a] = fneq;
    eqf[a] = geq + ph;
    Pxx += fneq * exa * exa;
    Pyy += fneq * eya * eya;
    Pxy += fneq * exa * eya;
    const float ep = (dpv[a] - udp) - E;
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      // C_i Gamma kept as its own term: the small corrections are not rounded
      // into a value of the size of C_i first
      const float phh = (dCv[i][a] - udC[i] - kap[i] * ep) * G;
      hs[i][a] = Cc[i] * G + 0.5f * phh + 0.5f * sv[i] * G;
    }
  }
  // (1/cs^2) (2 tau / (2 tau + 1)) / (2 tau rho cs^2) = 9 / ((2 tau + 1) rho)
  const float fac = __fdividef(9.0f * irho, 2.0f * tau_prev + 1.0f);
  const float Dxx = -fac * Pxx, Dyy = -fac * Pyy, Dxy = -fac * Pxy;
  // squared strain rate 2 D:D; the power law takes it without a square root
  gd2 = 2.0f * (Dxx * Dxx + Dyy * Dyy + 2.0f * Dxy * Dxy);
  const float C3 = 1.0f - Cc[0] - (NH == 2 ? Cc[NH - 1] : 0.f);
  const float tau1 = P.powerlaw ? tau_powerlaw_sq(P, gd2, irho) : P.tau[0];
  tn = tau_mix(P, Cc[0], NH == 2 ? Cc[NH - 1] : 0.f, C3, tau1);
  const float om = __fdividef(1.0f, tn + 0.5f);
#pragma unroll
  for (int a = 0; a < 9; ++a) g[a] = (1.0f - om) * g[a] + eqf[a];
}

// FP16 deviation codec of the FP16 storage form: g_a is kept as
// half((g_a - w_a P) scale) with P = sum_a g_a in FP32.  One rounding order for
// every encoder and decoder, so that a decode-encode round trip is exact.
__device__ __forceinline__ float g16_decode(float Pref, __half d, int a, float inv_scale) {
  return __fmaf_rn(wt(a), Pref, __half2float(d) * inv_scale);
}
__device__ __forceinline__ __half g16_encode(float g, float Pref, int a, float scale) {
  return __float2half_rn(__fmaf_rn(-wt(a), Pref, g) * scale);
}
__device__ __forceinline__ float g16_reference(const float (&g)[9]) {
  float Pn = 0.f;
#pragma unroll
  for (int a = 0; a < 9; ++a) Pn += g[a];
  return Pn;
}

// State forms (see the fused kernels): 0 populations g, h; 1 g and C;
// 2 FP16 g deviations with an FP32 reference plane, and C.

// C_i of node k (Eq. 22, or the stored C_i).
template <int NH, int FORM>
__device__ __forceinline__ void load_order_parameters(const FusedBuffers &B, long long plane, long long k,
                                                      float (&c)[NH]) {
#pragma unroll
  for (int i = 0; i < NH; ++i) {
    float acc;
    if constexpr (FORM == 0) {
      acc = 0.f;
#pragma unroll
      for (int a = 0; a < 9; ++a) acc += B.h_in[((long long)i * 9 + a) * plane + k];
    } else {
      acc = B.h_in[(long long)i * plane + k];
    }
    c[i] = acc;
  }
}

// The nine g of node k (decoded in the FP16 form).
template <int FORM>
__device__ __forceinline__ void load_populations(const DevParams &P, const FusedBuffers &B, long long plane,
                                                 long long k, float (&g)[9]) {
  if constexpr (FORM == 2) {
    const float Pref = B.g_in[(9 * plane) / 2 + k];
    const __half *gh = reinterpret_cast<const __half *>(B.g_in);
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = g16_decode(Pref, gh[(long long)a * plane + k], a, P.g16_inv_scale);
  } else {
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = B.g_in[(long long)a * plane + k];
  }
}

// New tau of an owned node, optional diagnostics (strain rate from its square
// gd2), and the finiteness check.
template <int NH>
__device__ __forceinline__ void store_diagnostics(const FusedBuffers &B, long long plane, long long k, float tn,
                                                  float gd2, const float (&sv)[NH], const NodeCenter &c) {
  B.tau_out[k] = tn;
  if (B.shear) B.shear[k] = sqrtf(gd2);
  if (B.SV) {
#pragma unroll
    for (int i = 0; i < NH; ++i) B.SV[(long long)i * plane + k] = sv[i];
  }
  if (!(isfinite(tn) && isfinite(c.p) && isfinite(c.ux) && isfinite(c.uy))) atomicOr(B.err, 1u);
}

// Stores the arrived populations of node ky: gy[a] = g*_b of the source,
// hy[i][a] = h*_b of the source (b = a, or opp(a) after bounce-back), sv the
// node's diffusion sources; destination-side term S_i Gamma_a / 2 (R9), which
// sums to S_i / 2 in the C forms.
template <int NH, int FORM>
__device__ __forceinline__ void store_node(const DevParams &P, const FusedBuffers &B, long long plane, long long ky,
                                           const float (&gy)[9], const float (&hy)[NH][9], const float (&sv)[NH],
                                           float ux, float uy) {
  if constexpr (FORM == 2) {
    const float Pn = g16_reference(gy);
    B.g_out[(9 * plane) / 2 + ky] = Pn;
    __half *gh = reinterpret_cast<__half *>(B.g_out);
#pragma unroll
    for (int a = 0; a < 9; ++a) gh[(long long)a * plane + ky] = g16_encode(gy[a], Pn, a, P.g16_scale);
  } else {
#pragma unroll
    for (int a = 0; a < 9; ++a) B.g_out[(long long)a * plane + ky] = gy[a];
  }
  if constexpr (FORM == 0) {
    // Gamma_a = w_a (1 - 1.5 u.u + 4.5 (e.u)^2 + 3 e.u): the even part is shared
    // by opposite directions
    const float S0 = 1.0f - 1.5f * (ux * ux + uy * uy);
    float G[9];
    G[0] = wt(0) * S0;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      if (a == 1 || a == 2 || a == 5 || a == 6) {
        const float eu = ex(a) * ux + ey(a) * uy;
        const float Bp = fmaf(4.5f * eu, eu, S0);
        G[a] = wt(a) * fmaf(3.0f, eu, Bp);
        G[opp(a)] = wt(a) * fmaf(-3.0f, eu, Bp);
      }
    }
    float hsv[NH];
#pragma unroll
    for (int i = 0; i < NH; ++i) hsv[i] = 0.5f * sv[i];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
#pragma unroll
      for (int i = 0; i < NH; ++i) B.h_out[((long long)i * 9 + a) * plane + ky] = fmaf(hsv[i], G[a], hy[i][a]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int a = 0; a < 9; ++a) acc += hy[i][a];
      B.h_out[(long long)i * plane + ky] = acc + 0.5f * sv[i];
    }
  }
}

}  // namespace lbm
