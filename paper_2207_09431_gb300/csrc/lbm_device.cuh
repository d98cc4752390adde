// Device-side definitions of the coupled power-law / Cahn-Hilliard D2Q9 step
// (arXiv 2207.09431, Sec. 2).  FP32 arithmetic throughout.
//
// Readings of the paper applied here (the same ones the CPU oracle applies):
//  R1  mixture laws rho = sum c_i rho_i, tau = sum c_i tau_i with weights
//      c_i = clip(C_i, 0, 1) / sum_j clip(C_j, 0, 1) (Sec. 2.2 names no law);
//  R2  isotropic gradient 3 sum w e X(x+e), Laplacian 6 sum w (X(x+e) - X(x));
//      (e_a - u).grad X = directional derivative along e_a - u . isotropic;
//  R3  p = sum g + (1/2) cs^2 u . grad rho (Eq. 24 with the half restored);
//  R4  tau_PL = eta / (rho cs^2) clamped to [tau_min, tau_max], node tau =
//      sum c_i tau_i with tau_1 = tau_PL, strain rate from the previous tau;
//  R8  variable mobility (D0/Sigma_i) c (1 - c), c = clip(C_i, 0, 1), and its
//      derivative term (D0/Sigma_i)(1 - 2 C_i) grad C_i . grad mu_i where
//      0 <= C_i <= 1 (else 0);
//  R9  destination-side source terms of Eq. 18 at the arrival node;
//  R10 half-way walls, ghost rows mirror the fluid rows;
//  R23 strain rate D = -Pi / (2 tau rho cs^2) with Pi from Eq. 29.
#pragma once

#include <cstdint>

#include "lbm_devparams.h"

namespace lbm {

// D2Q9 (Eq. 10-11): 0 rest, 1-4 E N W S, 5-8 NE NW SW SE.  Compile-time
// functions, so that unrolled loops see immediates.
//
// FP32 weights chosen so that w0 + 4 w1 + 4 w2 == 1 exactly: fl(4/9), fl(1/9)
// and fl(1/36) lowered by one ulp.  With the nearest floats the nine weights
// sum to 1 + 1.1e-8, and every node would gain that fraction of its order
// parameter per step (a systematic mass drift of 1e-5 in 1000 steps).
#define LBM_W0 0x1.c71c72p-2f
#define LBM_W1 0x1.c71c72p-4f
#define LBM_W2 0x1.c71c70p-6f
__host__ __device__ constexpr int ex(int a) { return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0); }
__host__ __device__ constexpr int ey(int a) { return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0); }
__host__ __device__ constexpr float wt(int a) { return a == 0 ? LBM_W0 : (a < 5 ? LBM_W1 : LBM_W2); }
__host__ __device__ constexpr int opp(int a) { return a == 0 ? 0 : (a < 5 ? (a + 1) % 4 + 1 : (a - 3) % 4 + 5); }
static_assert(opp(1) == 3 && opp(2) == 4 && opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "D2Q9");

constexpr float kCs2 = 1.0f / 3.0f;

// Periodic wrap along x for |dx| <= nx.
__device__ __forceinline__ int wrap_x(int x, int nx) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }

// y index of the value seen at row y (periodic, or the mirror ghost rows of R10)
// for |offset| <= ny.
__device__ __forceinline__ int wrap_y(int y, int ny, int periodic) {
  if (periodic) return y < 0 ? y + ny : (y >= ny ? y - ny : y);
  return y < 0 ? -1 - y : (y >= ny ? 2 * ny - 1 - y : y);
}

// Gamma_a(u) = f_a^eq / rho (Eq. 9).
__device__ __forceinline__ float gamma_a(int a, float ux, float uy) {
  float eu = ex(a) * ux + ey(a) * uy;
  float uu = ux * ux + uy * uy;
  return wt(a) * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * uu);
}

// Mixture weights of reading R1.
__device__ __forceinline__ void mixture_weights(float C1, float C2, float C3, float c[3]) {
  c[0] = fminf(fmaxf(C1, 0.0f), 1.0f);
  c[1] = fminf(fmaxf(C2, 0.0f), 1.0f);
  c[2] = fminf(fmaxf(C3, 0.0f), 1.0f);
  float inv = __fdividef(1.0f, c[0] + c[1] + c[2]);
  c[0] *= inv;
  c[1] *= inv;
  c[2] *= inv;
}

__device__ __forceinline__ float rho_of(const DevParams &P, float C1, float C2, float C3) {
  float c[3];
  mixture_weights(C1, C2, C3, c);
  return c[0] * P.rho[0] + c[1] * P.rho[1] + c[2] * P.rho[2];
}

// Chemical potentials mu_1..3 (Eq. 5) from C and its isotropic Laplacian.
__device__ __forceinline__ void chem_potentials(const DevParams &P, const float C[3], const float lapC[3],
                                                float mu[3]) {
  const float C1 = C[0], C2 = C[1], C3 = C[2];
  const float S1 = P.Sig[0], S2 = P.Sig[1], S3 = P.Sig[2];
  const float mix = S1 * C1 + S2 * C2 + S3 * C3;
  const float L = P.Lambda;
  // partial derivatives of E0 (Eq. 3)
  float d0 = 2.f * P.sig12 * C1 * C2 * C2 + 2.f * P.sig13 * C1 * C3 * C3 + C2 * C3 * (mix + S1 * C1) +
             2.f * L * C1 * C2 * C2 * C3 * C3;
  float d1 = 2.f * P.sig12 * C1 * C1 * C2 + 2.f * P.sig23 * C2 * C3 * C3 + C1 * C3 * (mix + S2 * C2) +
             2.f * L * C1 * C1 * C2 * C3 * C3;
  float d2 = 2.f * P.sig13 * C1 * C1 * C3 + 2.f * P.sig23 * C2 * C2 * C3 + C1 * C2 * (mix + S3 * C3) +
             2.f * L * C1 * C1 * C2 * C2 * C3;
  // (4 Sigma_T / xi) sum_{j != i} (d_i - d_j) / Sigma_j - (3/4) xi Sigma_i lap C_i
  mu[0] = P.mu_pre * ((d0 - d1) * P.inv_sig[1] + (d0 - d2) * P.inv_sig[2]) - P.grad_coef[0] * lapC[0];
  mu[1] = P.mu_pre * ((d1 - d0) * P.inv_sig[0] + (d1 - d2) * P.inv_sig[2]) - P.grad_coef[1] * lapC[1];
  mu[2] = P.mu_pre * ((d2 - d0) * P.inv_sig[0] + (d2 - d1) * P.inv_sig[1]) - P.grad_coef[2] * lapC[2];
}

// Two-component forms (C_2 = 0 identically, C_3 = 1 - C_1): the same values
// as rho_of, chem_potentials and tau_mix with C_2 = 0, without the terms that
// vanish with C_2 (products with a constant zero are kept by IEEE
// arithmetic).  The clipped weights of R1 then sum to one exactly
// (clip(C_1) + clip(1 - C_1) = 1 for every C_1), so their normalisation is
// the identity and is left out.
__device__ __forceinline__ float rho_of2(const DevParams &P, float C1) {
  const float c0 = fminf(fmaxf(C1, 0.0f), 1.0f), c2 = fminf(fmaxf(1.0f - C1, 0.0f), 1.0f);
  return c0 * P.rho[0] + c2 * P.rho[2];
}

// mu_1 and mu_3 of Eq. 5 with C_2 = 0: dE0/dC_1 = 2 Sigma_13 C_1 C_3^2,
// dE0/dC_2 = C_1 C_3 (Sigma_1 C_1 + Sigma_3 C_3), dE0/dC_3 = 2 Sigma_13 C_1^2 C_3.
__device__ __forceinline__ void chem_potentials2(const DevParams &P, float C1, float C3, float lap1, float lap3,
                                                 float &mu1, float &mu3) {
  const float mix = P.Sig[0] * C1 + P.Sig[2] * C3;
  const float c13 = C1 * C3, s = 2.f * P.sig13 * c13;
  const float d0 = s * C3, d1 = c13 * mix, d2 = s * C1;
  mu1 = P.mu_pre * ((d0 - d1) * P.inv_sig[1] + (d0 - d2) * P.inv_sig[2]) - P.grad_coef[0] * lap1;
  mu3 = P.mu_pre * ((d2 - d0) * P.inv_sig[0] + (d2 - d1) * P.inv_sig[1]) - P.grad_coef[2] * lap3;
}

// Power-law relaxation time at strain rate gd (Eq. 31-33, reading R4):
// tau = k gd^(n-1) / (rho cs^2), clamped; irho = 1 / rho.
__device__ __forceinline__ float tau_powerlaw(const DevParams &P, float gd, float irho) {
  float t;
  if (gd > 0.0f) {
    t = P.k3 * exp2f(P.n1 * __log2f(gd)) * irho;
  } else {  // zero strain rate: infinite (n < 1), zero (n > 1) or k (n = 1) viscosity
    t = P.n1 < 0.0f ? __int_as_float(0x7f800000) : (P.n1 > 0.0f ? 0.0f : P.k3 * irho);
  }
  t = (t <= P.tau_max) ? t : P.tau_max;  // also maps +inf to tau_max
  return fmaxf(t, P.tau_min);
}

// The same from the squared strain rate gd2 = gd^2 (no square root):
// gd^(n-1) = gd2^((n-1)/2).
__device__ __forceinline__ float tau_powerlaw_sq(const DevParams &P, float gd2, float irho) {
  float t;
  if (gd2 > 0.0f) {
    t = P.k3 * exp2f(P.n1h * __log2f(gd2)) * irho;
  } else {
    t = P.n1 < 0.0f ? __int_as_float(0x7f800000) : (P.n1 > 0.0f ? 0.0f : P.k3 * irho);
  }
  t = (t <= P.tau_max) ? t : P.tau_max;
  return fmaxf(t, P.tau_min);
}

__device__ __forceinline__ float tau_mix(const DevParams &P, float C1, float C2, float C3, float tau1) {
  float c[3];
  mixture_weights(C1, C2, C3, c);
  return c[0] * tau1 + c[1] * P.tau[1] + c[2] * P.tau[2];
}

__device__ __forceinline__ float tau_mix2(const DevParams &P, float C1, float tau1) {
  const float c0 = fminf(fmaxf(C1, 0.0f), 1.0f), c2 = fminf(fmaxf(1.0f - C1, 0.0f), 1.0f);
  return c0 * tau1 + c2 * P.tau[2];
}

}  // namespace lbm
