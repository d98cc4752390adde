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
  if constexpr (NH == 1) return rho_of2(P, c[0]);
  else return rho_of(P, c[0], c[1], 1.0f - c[0] - c[1]);
}

// Stencil helpers.  The four direction pairs (a, opp(a)) with a = 1, 2, 5, 6:
// pair k has direction pair_dir(k).  Sums over e_a are written out so that no
// product with a zero component of e_a is formed.
__device__ __host__ constexpr int pair_dir(int k) { return k < 2 ? k + 1 : k + 3; }

// D[k] = v(x + e_a) - v(x - e_a), a = pair_dir(k): twice the central
// directional derivative along e_a.
__device__ __forceinline__ void pair_diff(const float (&v)[9], float (&D)[4]) {
  D[0] = v[1] - v[3];
  D[1] = v[2] - v[4];
  D[2] = v[5] - v[7];
  D[3] = v[6] - v[8];
}

// Isotropic gradient 3 sum_a w_a e_a v_a from the pair differences
// (e_5 = (1, 1), e_6 = (-1, 1)).
__device__ __forceinline__ void iso_grad(const float (&D)[4], float &gx, float &gy) {
  gx = fmaf(3.0f * LBM_W2, D[2] - D[3], (3.0f * LBM_W1) * D[0]);
  gy = fmaf(3.0f * LBM_W2, D[2] + D[3], (3.0f * LBM_W1) * D[1]);
}

// Isotropic Laplacian 6 sum_a w_a (v_a - v_0), from the differences to the
// centre (exact for neighbouring values close to it).
__device__ __forceinline__ float iso_lap(const float (&v)[9]) {
  const float v0 = v[0];
  const float sa = ((v[1] - v0) + (v[3] - v0)) + ((v[2] - v0) + (v[4] - v0));
  const float sd = ((v[5] - v0) + (v[7] - v0)) + ((v[6] - v0) + (v[8] - v0));
  return fmaf(6.0f * LBM_W2, sd, (6.0f * LBM_W1) * sa);
}

// Packed FP32 forms (two lanes per instruction on sm_100-family SMs) of the
// stencils above, for two fields stored side by side: each lane performs the
// scalar helpers' operations in their order, so the values are theirs.
__device__ __forceinline__ float2 bcast2(float v) { return make_float2(v, v); }
// a - b with one rounding (the product by -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bcast2(-1.0f), a); }

// pair differences, isotropic gradient and isotropic Laplacian of both lanes
__device__ __forceinline__ void stencil2(const float2 (&v)[9], float2 (&D)[4], float2 &gx, float2 &gy,
                                         float2 &lap) {
  D[0] = sub2(v[1], v[3]);
  D[1] = sub2(v[2], v[4]);
  D[2] = sub2(v[5], v[7]);
  D[3] = sub2(v[6], v[8]);
  gx = __ffma2_rn(bcast2(3.0f * LBM_W2), sub2(D[2], D[3]), __fmul2_rn(bcast2(3.0f * LBM_W1), D[0]));
  gy = __ffma2_rn(bcast2(3.0f * LBM_W2), __fadd2_rn(D[2], D[3]), __fmul2_rn(bcast2(3.0f * LBM_W1), D[1]));
  const float2 v0 = v[0];
  const float2 sa = __fadd2_rn(__fadd2_rn(sub2(v[1], v0), sub2(v[3], v0)), __fadd2_rn(sub2(v[2], v0), sub2(v[4], v0)));
  const float2 sd = __fadd2_rn(__fadd2_rn(sub2(v[5], v0), sub2(v[7], v0)), __fadd2_rn(sub2(v[6], v0), sub2(v[8], v0)));
  lap = __ffma2_rn(bcast2(6.0f * LBM_W2), sd, __fmul2_rn(bcast2(6.0f * LBM_W1), sa));
}

// e_a . (vx, vy) for a != 0.
__device__ __forceinline__ float edot(int a, float vx, float vy) {
  const float sx = ex(a) > 0 ? vx : -vx, sy = ey(a) > 0 ? vy : -vy;
  return ex(a) == 0 ? sy : (ey(a) == 0 ? sx : sx + sy);
}

// Gamma_a(u) = w_a (1 - 1.5 u.u + 4.5 (e_a.u)^2 + 3 e_a.u) (Eq. 9) of every
// direction: the even part is shared by opposite directions.
__device__ __forceinline__ void gamma_all(float ux, float uy, float (&G)[9]) {
  const float S0 = 1.0f - 1.5f * (ux * ux + uy * uy);
  G[0] = LBM_W0 * S0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int a = pair_dir(k);
    const float w = wt(a), eu = edot(a, ux, uy);
    const float wB = fmaf((4.5f * w) * eu, eu, w * S0);
    G[a] = fmaf(3.0f * w, eu, wB);
    G[opp(a)] = fmaf(-3.0f * w, eu, wB);
  }
}

// Fields of a node of the 2-ring: moments of g, isotropic gradients of C and
// rho, chemical potentials (Eq. 5), velocity (Eq. 23) and pressure (Eq. 24,
// reading R3).
struct NodeFields {
  float mu[3], gCx[3], gCy[3];
  float rx, ry, ux, uy, p, rho, irho;
  float C[2], Dr[4], DC[2][4];  // C_i, and the pair differences of rho and C_i
};

template <int NH>
__device__ __forceinline__ void node_fields(const DevParams &P, const float (&g)[9], const float (&cn)[NH][9],
                                            const float (&rn)[9], NodeFields &f) {
  float Dg[4];
  pair_diff(g, Dg);
  const float m0 = (((g[1] + g[3]) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]))) + g[0];
  const float mx = Dg[0] + (Dg[2] - Dg[3]);
  const float my = Dg[1] + (Dg[2] + Dg[3]);
  pair_diff(rn, f.Dr);
  float rx, ry;
  iso_grad(f.Dr, rx, ry);
  float C[3], lap[3];
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    pair_diff(cn[j], f.DC[j]);
    iso_grad(f.DC[j], f.gCx[j], f.gCy[j]);
    lap[j] = iso_lap(cn[j]);
    C[j] = f.C[j] = cn[j][0];
  }
  float Fsx, Fsy;
  if constexpr (NH == 1) {
    // C_3 = 1 - C_1 (Eq. 1): its stencils are minus those of C_1
    C[2] = 1.0f - C[0];
    f.gCx[2] = -f.gCx[0];
    f.gCy[2] = -f.gCy[0];
    lap[2] = -lap[0];
    f.gCx[1] = f.gCy[1] = f.mu[1] = 0.0f;
    chem_potentials2(P, C[0], C[2], lap[0], lap[2], f.mu[0], f.mu[2]);
    Fsx = f.mu[0] * f.gCx[0] + f.mu[2] * f.gCx[2];
    Fsy = f.mu[0] * f.gCy[0] + f.mu[2] * f.gCy[2];
  } else {
    // C_3 = 1 - C_1 - C_2 (Eq. 1): its stencils are minus the sum of the others'
    C[2] = 1.0f - C[0] - C[1];
    f.gCx[2] = -(f.gCx[0] + f.gCx[1]);
    f.gCy[2] = -(f.gCy[0] + f.gCy[1]);
    lap[2] = -(lap[0] + lap[1]);
    chem_potentials(P, C, lap, f.mu);
    Fsx = f.mu[0] * f.gCx[0] + f.mu[1] * f.gCx[1] + f.mu[2] * f.gCx[2];
    Fsy = f.mu[0] * f.gCy[0] + f.mu[1] * f.gCy[1] + f.mu[2] * f.gCy[2];
  }
  const float rho = rn[0];
  const float irho = __fdividef(1.0f, rho);
  f.rho = rho;
  f.irho = irho;
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
// The node's own values come from the field stage (NodeFields of the same
// node): rho and 1 / rho, C_i, and the pair differences of rho and C_i.
struct NodeCenter {
  float ux, uy, p, rho, irho, grx, gry;
  float dmu[2], gCx[2], gCy[2];
  float C[2], Dr[4], DC[2][4];
};

template <int NH>
__device__ __forceinline__ void node_collide(const DevParams &P, const NodeCenter &c, const float (&pn)[9],
                                             const float (&mun)[NH][9], float (&g)[9], float tau_prev,
                                             float (&hs)[NH][9], float (&sv)[NH], float &tn, float &gd2) {
  const float ux = c.ux, uy = c.uy, p = c.p, rho = c.rho;
  const float irho = c.irho;
  // Differences across the node along the direction pairs: the central
  // directional derivative d_a v = (v(x + e_a) - v(x - e_a)) / 2 is half of
  // one, and d_opp(a) v = -d_a v.
  float Dp[4], px, py, mgxs[NH], mgys[NH], lapmus[NH];
  if constexpr (NH == 1) {
    // mu_1 and p side by side
    float2 v[9], D[4], gx, gy, lp;
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = make_float2(mun[0][a], pn[a]);
    stencil2(v, D, gx, gy, lp);
#pragma unroll
    for (int k = 0; k < 4; ++k) Dp[k] = D[k].y;
    px = gx.y;
    py = gy.y;
    mgxs[0] = gx.x;
    mgys[0] = gy.x;
    lapmus[0] = lp.x;
  } else {
    pair_diff(pn, Dp);
    iso_grad(Dp, px, py);
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      float Dm[4];
      pair_diff(mun[i], Dm);
      iso_grad(Dm, mgxs[i], mgys[i]);
      lapmus[i] = iso_lap(mun[i]);
    }
  }
  const float (&Dr)[4] = c.Dr;
  float Fsx, Fsy, Cc[NH], kh[NH], hb[NH], hdmu[NH];
#pragma unroll
  for (int i = 0; i < NH; ++i) {
    const float mgx = mgxs[i], mgy = mgys[i], lapmu = lapmus[i];
    const float gcx = c.gCx[i], gcy = c.gCy[i];
    Fsx = i == 0 ? c.dmu[0] * gcx : fmaf(c.dmu[i], gcx, Fsx);
    Fsy = i == 0 ? c.dmu[0] * gcy : fmaf(c.dmu[i], gcy, Fsy);
    Cc[i] = c.C[i];
    const float D0s = P.d0_sig[i];
    if (P.mobility == 1) {
      // mobility with C clipped to [0, 1] and its derivative (reading R8)
      const float cc = fminf(fmaxf(Cc[i], 0.0f), 1.0f);
      const float dv = (Cc[i] >= 0.0f && Cc[i] <= 1.0f) ? D0s * (1.0f - 2.0f * Cc[i]) * (gcx * mgx + gcy * mgy)
                                                       : 0.0f;
      sv[i] = D0s * cc * (1.0f - cc) * lapmu + dv;
    } else {
      sv[i] = D0s * lapmu;
    }
    kh[i] = 1.5f * Cc[i] * irho;                     // C_i / (rho cs^2) / 2
    hb[i] = 0.5f * (sv[i] - (ux * gcx + uy * gcy));  // (S_i - u.grad C_i) / 2
    hdmu[i] = 0.5f * c.dmu[i];
  }
  const float Fby = -rho * P.gravity;
  const float udr3 = (ux * c.grx + uy * c.gry) * kCs2;
  const float uF = (ux * Fsx + uy * Fsy) + (ux * P.force_x + uy * Fby);
  const float udp = ux * px + uy * py;
  const float S0 = 1.0f - 1.5f * (ux * ux + uy * uy);
  const float rcs2 = rho * kCs2;
  const float c0 = uF - udp;
  // Per direction a, with Gamma_a = w_a (1 - 1.5 u.u + 4.5 (e.u)^2 + 3 e.u):
  //   X_a   = sum_i (mu_i - mu_3) d_a C_i + e_a.F_b,   E_a = X_a - u.(F_s + F_b)
  //   t_a   = (d_a rho - u.grad rho) cs^2
  //   ph_a  = t_a (Gamma_a - w_a) + E_a Gamma_a                               (Eq. 14-16)
  //   geq_a = w_a p + rho cs^2 (Gamma_a - w_a) - ph_a / 2
  //   ep_a  = d_a p - u.grad p - E_a = (d_a p - X_a) + (u.F - u.grad p)
  //   h*_a  = C_i Gamma_a + Gamma_a [(d_a C_i - u.grad C_i + S_i) / 2
  //            - C_i / (rho cs^2) ep_a / 2]                                      (Eq. 18-20)
  // X_a, d_a and e.u change sign between opposite directions, (e.u)^2 does
  // not: each is formed once per pair.  C_i Gamma_a is kept as its own term so
  // that the small corrections are not rounded into a value of the size of C_i.
  // A direction and its opposite are evaluated as one pair on the packed FP32
  // pipe (lane x: a, lane y: opp(a)), each lane the same operation sequence
  // as the scalar form, so the values do not depend on the packing.
  const float G0 = LBM_W0 * S0, Gw0 = G0 - LBM_W0;
  const float ph0 = fmaf(-udr3, Gw0, -uF * G0);
  const float geq0 = fmaf(-0.5f, ph0, fmaf(rcs2, Gw0, LBM_W0 * p));
  const float fn0 = g[0] - geq0, eq0 = geq0 + ph0;
#pragma unroll
  for (int i = 0; i < NH; ++i) hs[i][0] = fmaf(Cc[i], G0, G0 * fmaf(-kh[i], c0, hb[i]));
  float2 fn2[4], eq2[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int a = pair_dir(k), b = opp(a);
    const float w = wt(a), eu = edot(a, ux, uy);
    const float wB = fmaf((4.5f * w) * eu, eu, w * S0);
    float X = edot(a, P.force_x, Fby);
#pragma unroll
    for (int i = 0; i < NH; ++i) X = fmaf(hdmu[i], c.DC[i][k], X);
    const float o = fmaf(0.5f, Dp[k], -X);
    const float2 G = __ffma2_rn(make_float2(3.0f * w, -3.0f * w), bcast2(eu), bcast2(wB));
    const float2 E = __fadd2_rn(make_float2(X, -X), bcast2(-uF));
    const float2 t = __ffma2_rn(make_float2(0.5f * kCs2, -0.5f * kCs2), bcast2(Dr[k]),
                                bcast2(-udr3));
    const float2 ep = __fadd2_rn(make_float2(o, -o), bcast2(c0));
    const float2 Gw = __fadd2_rn(G, bcast2(-w));
    const float2 ph = __ffma2_rn(t, Gw, __fmul2_rn(E, G));
    const float wp = w * p;
    const float2 geq = __ffma2_rn(bcast2(-0.5f), ph,
                                  __ffma2_rn(bcast2(rcs2), Gw, bcast2(wp)));
    fn2[k] = __ffma2_rn(geq, bcast2(-1.0f), make_float2(g[a], g[b]));  // g - geq, exact negation
    eq2[k] = __fadd2_rn(geq, ph);
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      const float2 hq = __ffma2_rn(make_float2(0.25f, -0.25f), bcast2(c.DC[i][k]),
                                   bcast2(hb[i]));
      const float2 r = __ffma2_rn(bcast2(Cc[i]), G,
                                  __fmul2_rn(G, __ffma2_rn(bcast2(-kh[i]), ep, hq)));
      hs[i][a] = r.x;
      hs[i][b] = r.y;
    }
  }
  // second moments of the non-equilibrium part (pairs 5-7 and 6-8 enter all three)
  const float s57 = fn2[2].x + fn2[2].y, s68 = fn2[3].x + fn2[3].y, sd = s57 + s68;
  const float Pxx = (fn2[0].x + fn2[0].y) + sd, Pyy = (fn2[1].x + fn2[1].y) + sd, Pxy = s57 - s68;
  // (1/cs^2) (2 tau / (2 tau + 1)) / (2 tau rho cs^2) = 9 / ((2 tau + 1) rho)
  const float fac = __fdividef(9.0f * irho, 2.0f * tau_prev + 1.0f);
  const float Dxx = -fac * Pxx, Dyy = -fac * Pyy, Dxy = -fac * Pxy;
  // squared strain rate 2 D:D; the power law takes it without a square root
  gd2 = 2.0f * (Dxx * Dxx + Dyy * Dyy + 2.0f * Dxy * Dxy);
  const float tau1 = P.powerlaw ? tau_powerlaw_sq(P, gd2, irho) : P.tau[0];
  if constexpr (NH == 1) tn = tau_mix2(P, Cc[0], tau1);
  else tn = tau_mix(P, Cc[0], Cc[1], 1.0f - Cc[0] - Cc[1], tau1);
  const float om = __fdividef(1.0f, tn + 0.5f), om1 = 1.0f - om;
  g[0] = fmaf(om1, fn0, eq0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 r = __ffma2_rn(make_float2(om1, om1), fn2[k], eq2[k]);
    g[pair_dir(k)] = r.x;
    g[opp(pair_dir(k))] = r.y;
  }
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
      const float *hp = B.h_in + pop_index(k, i * 9, 9 * NH);
      acc = 0.f;
#pragma unroll
      for (int a = 0; a < 9; ++a) acc += hp[a * 32];
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
    const __half *gh = reinterpret_cast<const __half *>(B.g_in) + pop_index(k, 0, 9);
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = g16_decode(Pref, gh[a * 32], a, P.g16_inv_scale);
  } else {
    const float *gp = B.g_in + pop_index(k, 0, 9);
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = gp[a * 32];
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
    __half *gh = reinterpret_cast<__half *>(B.g_out) + pop_index(ky, 0, 9);
#pragma unroll
    for (int a = 0; a < 9; ++a) gh[a * 32] = g16_encode(gy[a], Pn, a, P.g16_scale);
  } else {
    float *go = B.g_out + pop_index(ky, 0, 9);
#pragma unroll
    for (int a = 0; a < 9; ++a) go[a * 32] = gy[a];
  }
  if constexpr (FORM == 0) {
    float G[9];
    gamma_all(ux, uy, G);
    float hsv[NH];
#pragma unroll
    for (int i = 0; i < NH; ++i) hsv[i] = 0.5f * sv[i];
    float *ho = B.h_out + pop_index(ky, 0, 9 * NH);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
#pragma unroll
      for (int i = 0; i < NH; ++i) ho[(i * 9 + a) * 32] = fmaf(hsv[i], G[a], hy[i][a]);
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
