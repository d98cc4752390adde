// Fused form of the coupled D2Q9 step (arXiv 2207.09431, Sec. 2.2-2.3): one
// kernel per time step, pull scheme, one CTA per TX x TY tile of output nodes.
//
// A population arriving at node y in direction a left x = y - e_a, so the tile
// needs the collision of its one-node ring R1; that collision needs p and mu
// on the two-node ring R2 (gradients and directional derivatives), which in
// turn need C on the three-node ring R3 (Laplacian inside mu).  Stages:
//   0  C_i = sum_a h_a^i (Eq. 22), or C_i itself in the collapsed form, and the
//      mixture density on R3
//   1  g loaded once into shared memory; mu (Eq. 5), grad C, grad rho, u (Eq. 23)
//      and p (Eq. 24 with the half of reading R3) on R2
//   2  on R1: S_i + V_i (Eq. 6, 21), h* for all directions (Eq. 18, tau_h = 1/2),
//      the strain rate and new tau (Eq. 25-33) and then g* for all directions
//      (Eq. 14), written over g in shared memory
//   3  per output node and direction: gather the post-collision value of the
//      source node (half-way bounce-back at walls), add the destination-side
//      source term (R9), coalesced stores
// Global memory sees the populations and tau read once and written once; the
// halo rings are re-read through L2.  Ghost rows beyond a wall hold mirrored
// values (R10): loaded data is mirrored pointwise, stencil-derived mu and p are
// copied from the mirror slot.
#include <cuda_fp16.h>

#include "lbm_device.cuh"
#include "lbm_kernels.h"

namespace lbm {

namespace {

// Periodic index for offsets of at most one period (the common case) with a
// modulo fallback for lattices smaller than a tile.
__device__ __forceinline__ int wrap_periodic(int v, int n) {
  if (v < 0) v += n;
  if (v >= n) v -= n;
  if (v < 0 || v >= n) v = ((v % n) + n) % n;
  return v;
}

// Row read for row gy: periodic, or mirrored about the half-way walls; rows far
// outside (only in unused slots of a ragged tile) are clamped.
__device__ __forceinline__ int row_read(int gy, int ny, int periodic) {
  if (periodic) return wrap_periodic(gy, ny);
  if (gy < 0) gy = -1 - gy;
  if (gy >= ny) gy = 2 * ny - 1 - gy;
  return gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy);
}

template <int TX, int TY, int NH>
struct Smem {
  static constexpr int W3 = TX + 6, H3 = TY + 6, N3 = W3 * H3;
  static constexpr int W2 = TX + 4, H2 = TY + 4, N2 = W2 * H2;
  static constexpr int W1 = TX + 2, H1 = TY + 2, N1 = W1 * H1;
  // R3
  float C[NH][N3];
  float rho[N3];
  // R2: populations g (post-collision g* on R1 after stage 2), chemical
  // potentials mu_i and mu_i - mu_3, pressure, velocity, isotropic gradients
  float g[9][N2];
  float mu[NH][N2], dmu[NH][N2];
  float p[N2], ux[N2], uy[N2];
  float gCx[NH][N2], gCy[NH][N2], grx[N2], gry[N2];
  // R1: post-collision h*, g^eq + forcing (pass A -> pass B of stage 2) and
  // the diffusion sources
  float hs[NH][9][N1];
  float eqf[9][N1];
  float sv[NH][N1];
};

template <int TX>
__device__ __forceinline__ int i3(int lx, int ly) { return (ly + 3) * (TX + 6) + (lx + 3); }
template <int TX>
__device__ __forceinline__ int i2(int lx, int ly) { return (ly + 2) * (TX + 4) + (lx + 2); }
template <int TX>
__device__ __forceinline__ int i1(int lx, int ly) { return (ly + 1) * (TX + 2) + (lx + 1); }

// FP16 deviation codec of the FORM 2 state (below).  One rounding order for
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

}  // namespace

// FORM 0: the state holds the populations h^i (the method's state).
// FORM 1: the state holds C_i only.  With tau_h = 1/2 the collision of Eq. 18
// depends on h only through C_i = sum_a h_a^i, so C_i(t+1) = sum_a h_a^i(t+1)
// carries the same information (same results up to the order of the FP32
// sums) at 88 instead of 152 bytes per node-step.
// FORM 2: as FORM 1, and g is stored as FP16 deviations from a per-node
// reference: d_a = (g_a - w_a P) * scale with P = sum_a g_a kept in FP32 (the
// pressure-sized part stays in FP32, only the small deviations go to FP16),
// 60 bytes per node-step.  In memory: 9 half planes, then the FP32 P plane,
// inside the space of the 9 FP32 planes.
// NT threads per CTA (NT >= TX * TY); NT close to the size of R1 lets the
// heaviest stage run in one pass.
template <int TX, int TY, int NH, int FORM, int NT>
__device__ __forceinline__ void fused_tile(const DevParams &P, const FusedBuffers &B, int x0, int y0,
                                           Smem<TX, TY, NH> &s) {
  using S = Smem<TX, TY, NH>;
  const int tid = threadIdx.x;
  const long long plane = P.plane;
  const int nx = P.nx, ny = P.ny, per = P.periodic_y, pitch = P.pitch;

  // ---- stage 0: order parameters and density on R3
  for (int q = tid; q < S::N3; q += NT) {
    const int lx = q % S::W3 - 3, ly = q / S::W3 - 3;
    const long long k = (long long)row_read(y0 + ly, ny, per) * pitch + wrap_periodic(x0 + lx, nx);
    float c[3] = {0.f, 0.f, 0.f};
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
      s.C[i][q] = acc;
    }
    c[2] = 1.0f - c[0] - c[1];
    s.rho[q] = rho_of(P, c[0], c[1], c[2]);
  }
  __syncthreads();

  // ---- stage 1: g into shared memory; mu, gradients, u, p on R2 (real rows)
  for (int q = tid; q < S::N2; q += NT) {
    const int lx = q % S::W2 - 2, ly = q / S::W2 - 2;
    const int gy = y0 + ly;
    if (!per && (gy < 0 || gy >= ny)) continue;
    const long long k = (long long)(per ? wrap_periodic(gy, ny) : gy) * pitch + wrap_periodic(x0 + lx, nx);
    float m0 = 0.f, mx = 0.f, my = 0.f;
    float Pref = 0.f;
    if constexpr (FORM == 2) Pref = B.g_in[(9 * plane) / 2 + k];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      float ga;
      if constexpr (FORM == 2) {
        const __half *gh = reinterpret_cast<const __half *>(B.g_in);
        ga = g16_decode(Pref, gh[(long long)a * plane + k], a, P.g16_inv_scale);
      } else {
        ga = B.g_in[(long long)a * plane + k];
      }
      s.g[a][q] = ga;
      m0 += ga;
      mx += ex(a) * ga;
      my += ey(a) * ga;
    }
    float C[3], lap[3], gx[3], gyv[3], mu[3];
    float rx = 0.f, ry = 0.f;
    {
      const int c0 = i3<TX>(lx, ly);
      float cc[3][9];
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        const int j3 = c0 + ey(a) * S::W3 + ex(a);
        cc[0][a] = s.C[0][j3];
        cc[1][a] = NH == 2 ? s.C[NH - 1][j3] : 0.f;
        cc[2][a] = 1.0f - cc[0][a] - cc[1][a];
        const float r = s.rho[j3];
        rx += wt(a) * ex(a) * r;
        ry += wt(a) * ey(a) * r;
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        float sx = 0.f, sy = 0.f, lp = 0.f;
#pragma unroll
        for (int a = 1; a < 9; ++a) {
          sx += wt(a) * ex(a) * cc[j][a];
          sy += wt(a) * ey(a) * cc[j][a];
          lp += wt(a) * (cc[j][a] - cc[j][0]);
        }
        C[j] = cc[j][0];
        gx[j] = 3.0f * sx;
        gyv[j] = 3.0f * sy;
        lap[j] = 6.0f * lp;
      }
    }
    rx *= 3.0f;
    ry *= 3.0f;
    chem_potentials(P, C, lap, mu);
    const float Fsx = mu[0] * gx[0] + mu[1] * gx[1] + mu[2] * gx[2];
    const float Fsy = mu[0] * gyv[0] + mu[1] * gyv[1] + mu[2] * gyv[2];
    const float rho = s.rho[i3<TX>(lx, ly)];
    const float irho = 1.0f / rho;
    const float ux = (3.0f * mx + 0.5f * (Fsx + P.force_x)) * irho;
    const float uy = (3.0f * my + 0.5f * (Fsy - rho * P.gravity)) * irho;
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      s.mu[i][q] = mu[i];
      s.dmu[i][q] = mu[i] - mu[2];
      s.gCx[i][q] = gx[i];
      s.gCy[i][q] = gyv[i];
    }
    s.p[q] = m0 + 0.5f * kCs2 * (ux * rx + uy * ry);
    s.ux[q] = ux;
    s.uy[q] = uy;
    s.grx[q] = rx;
    s.gry[q] = ry;
  }
  __syncthreads();
  if (!per && (y0 < 2 || y0 + TY + 2 > ny)) {
    // ghost rows of R2: copy the stencil-derived mu and p of the mirror row
    for (int q = tid; q < S::N2; q += NT) {
      const int lx = q % S::W2 - 2, ly = q / S::W2 - 2;
      const int gy = y0 + ly;
      if (gy >= 0 && gy < ny) continue;
      const int my = (gy < 0 ? -1 - gy : 2 * ny - 1 - gy) - y0;
      if (my < -2 || my >= TY + 2) continue;
      const int src = i2<TX>(lx, my);
#pragma unroll
      for (int i = 0; i < NH; ++i) s.mu[i][q] = s.mu[i][src];
      s.p[q] = s.p[src];
    }
    __syncthreads();
  }

  // ---- stage 2: full collision on R1 (real rows)
  for (int q = tid; q < S::N1; q += NT) {
    const int lx = q % S::W1 - 1, ly = q / S::W1 - 1;
    const int gy = y0 + ly;
    if (!per && (gy < 0 || gy >= ny)) continue;
    const long long k = (long long)(per ? wrap_periodic(gy, ny) : gy) * pitch + wrap_periodic(x0 + lx, nx);
    const int c2 = i2<TX>(lx, ly);
    const int c3 = i3<TX>(lx, ly);
    const float ux = s.ux[c2], uy = s.uy[c2], p = s.p[c2], rho = s.rho[c3];
    const float irho = 1.0f / rho;
    // neighbour values, loaded once: p (2-ring), rho and C (3-ring)
    float pn[9], rn[9], cn[NH][9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const int j2 = c2 + ey(a) * S::W2 + ex(a), j3 = c3 + ey(a) * S::W3 + ex(a);
      pn[a] = s.p[j2];
      rn[a] = s.rho[j3];
#pragma unroll
      for (int i = 0; i < NH; ++i) cn[i][a] = s.C[i][j3];
    }
    // gradients of p and mu on R2
    float px = 0.f, py = 0.f, mgx[NH], mgy[NH], mlap[NH];
#pragma unroll
    for (int i = 0; i < NH; ++i) mgx[i] = mgy[i] = mlap[i] = 0.f;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      const int j2 = c2 + ey(a) * S::W2 + ex(a);
      const float pv = pn[a];
      px += wt(a) * ex(a) * pv;
      py += wt(a) * ey(a) * pv;
#pragma unroll
      for (int i = 0; i < NH; ++i) {
        const float m = s.mu[i][j2];
        mgx[i] += wt(a) * ex(a) * m;
        mgy[i] += wt(a) * ey(a) * m;
        mlap[i] += wt(a) * (m - s.mu[i][c2]);
      }
    }
    px *= 3.0f;
    py *= 3.0f;
    float Fsx = 0.f, Fsy = 0.f, Cc[NH], sv[NH], kap[NH], udC[NH], dmu[NH];
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      dmu[i] = s.dmu[i][c2];
      const float gcx = s.gCx[i][c2], gcy = s.gCy[i][c2];
      Fsx += dmu[i] * gcx;
      Fsy += dmu[i] * gcy;
      Cc[i] = s.C[i][c3];
      const float D0s = P.d0_sig[i];
      const float lapmu = 6.0f * mlap[i];
      if (P.mobility == 1)
        sv[i] = D0s * Cc[i] * (1.0f - Cc[i]) * lapmu +
                D0s * (1.0f - 2.0f * Cc[i]) * 3.0f * (gcx * mgx[i] + gcy * mgy[i]);
      else
        sv[i] = D0s * lapmu;
      kap[i] = 3.0f * Cc[i] * irho;  // C_i / (rho cs^2)
      udC[i] = ux * gcx + uy * gcy;
      s.sv[i][q] = sv[i];
    }
    const float Fby = -rho * P.gravity;
    const float udr = ux * s.grx[c2] + uy * s.gry[c2];
    const float udFs = ux * Fsx + uy * Fsy;
    const float udFb = ux * P.force_x + uy * Fby;
    const float udp = ux * px + uy * py;
    const float uu = ux * ux + uy * uy;
    const float rcs2 = rho * kCs2;
    // pass A: equilibria and forcing of every direction, h*, momentum flux;
    // g - g^eq is written over g and g^eq + forcing kept for pass B
    float Pxx = 0.f, Pyy = 0.f, Pxy = 0.f;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const float exa = (float)ex(a), eya = (float)ey(a), w = wt(a);
      const float eu = exa * ux + eya * uy;
      const float G = w * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * uu);
      // directional derivatives from the neighbour registers (x + e_a, x - e_a)
      const float dr = 0.5f * (rn[a] - rn[opp(a)]);
      const float dp = 0.5f * (pn[a] - pn[opp(a)]);
      float dC[NH];
      float eFs = -udFs;
#pragma unroll
      for (int i = 0; i < NH; ++i) {
        dC[i] = 0.5f * (cn[i][a] - cn[i][opp(a)]);
        eFs += dmu[i] * dC[i];
      }
      const float eFb = exa * P.force_x + eya * Fby - udFb;
      const float ph = (dr - udr) * kCs2 * (G - w) + (eFs + eFb) * G;
      const float geq = w * p + rcs2 * (G - w) - 0.5f * ph;
      const float fneq = s.g[a][c2] - geq;
      s.g[a][c2] = fneq;
      s.eqf[a][q] = geq + ph;
      Pxx += fneq * exa * exa;
      Pyy += fneq * eya * eya;
      Pxy += fneq * exa * eya;
      const float ep = dp - udp - eFs - eFb;
#pragma unroll
      for (int i = 0; i < NH; ++i) {
        const float phh = (dC[i] - udC[i] - kap[i] * ep) * G;
        s.hs[i][a][q] = Cc[i] * G + 0.5f * phh + 0.5f * sv[i] * G;
      }
    }
    // strain rate with the previous tau (R23) and the new tau (Eq. 31-33, R4)
    const float tp = B.tau_in[k];
    // (1/cs^2) (2 tau / (2 tau + 1)) / (2 tau rho cs^2) = 9 / ((2 tau + 1) rho)
    const float fac = 9.0f * irho / (2.0f * tp + 1.0f);
    const float Dxx = -fac * Pxx, Dyy = -fac * Pyy, Dxy = -fac * Pxy;
    const float gd = sqrtf(2.0f * (Dxx * Dxx + Dyy * Dyy + 2.0f * Dxy * Dxy));
    const float C3 = 1.0f - Cc[0] - (NH == 2 ? Cc[NH - 1] : 0.f);
    const float tau1 = P.powerlaw ? tau_powerlaw(P, gd, irho) : P.tau[0];
    const float tn = tau_mix(P, Cc[0], NH == 2 ? Cc[NH - 1] : 0.f, C3, tau1);
    const float om = 1.0f / (tn + 0.5f);
    // pass B: g* = g - om (g - g^eq) + forcing, over g in shared memory
#pragma unroll
    for (int a = 0; a < 9; ++a) s.g[a][c2] = (1.0f - om) * s.g[a][c2] + s.eqf[a][q];
    if (lx >= 0 && lx < TX && ly >= 0 && ly < TY && x0 + lx < nx && gy < ny) {
      B.tau_out[k] = tn;
      if (B.shear) B.shear[k] = gd;
      if (B.SV) {
#pragma unroll
        for (int i = 0; i < NH; ++i) B.SV[(long long)i * plane + k] = sv[i];
      }
      if (!(isfinite(tn) && isfinite(p) && isfinite(ux) && isfinite(uy))) atomicOr(B.err, 1u);
    }
  }
  __syncthreads();

  // ---- stage 3: streaming (pull) with bounce-back, destination-side term
  if (tid >= TX * TY) return;
  const int tx = tid % TX, ty = tid / TX;
  const int x = x0 + tx, y = y0 + ty;
  if (x >= nx || y >= ny) return;
  const long long ky = (long long)y * pitch + x;
  const int yc1 = i1<TX>(tx, ty), yc2 = i2<TX>(tx, ty);
  const float uxy = s.ux[yc2], uyy = s.uy[yc2];
  const float uuy = uxy * uxy + uyy * uyy;
  float svy[NH], csum[NH];
#pragma unroll
  for (int i = 0; i < NH; ++i) {
    svy[i] = 0.5f * s.sv[i][yc1];
    csum[i] = 0.f;
  }
  float gy[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    int s1 = yc1 - ey(a) * S::W1 - ex(a);
    int s2 = yc2 - ey(a) * S::W2 - ex(a);
    int b = a;
    if (!per) {
      const int ys = y - ey(a);
      if (ys < 0 || ys >= ny) {  // half-way bounce-back: the population left y in -e_a
        s1 = yc1;
        s2 = yc2;
        b = opp(a);
      }
    }
    if constexpr (FORM == 2) {
      gy[a] = s.g[b][s2];
    } else {
      B.g_out[(long long)a * plane + ky] = s.g[b][s2];
    }
    const float euy = ex(a) * uxy + ey(a) * uyy;
    const float Gy = wt(a) * (1.0f + 3.0f * euy + 4.5f * euy * euy - 1.5f * uuy);
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      const float hv = s.hs[i][b][s1] + svy[i] * Gy;
      if constexpr (FORM == 0) {
        B.h_out[((long long)i * 9 + a) * plane + ky] = hv;
      } else {
        csum[i] += hv;
      }
    }
  }
  if constexpr (FORM != 0) {
#pragma unroll
    for (int i = 0; i < NH; ++i) B.h_out[(long long)i * plane + ky] = csum[i];
  }
  if constexpr (FORM == 2) {
    const float Pn = g16_reference(gy);
    B.g_out[(9 * plane) / 2 + ky] = Pn;
    __half *gh = reinterpret_cast<__half *>(B.g_out);
#pragma unroll
    for (int a = 0; a < 9; ++a) gh[(long long)a * plane + ky] = g16_encode(gy[a], Pn, a, P.g16_scale);
  }
}

// One lattice: tile (blockIdx.x, blockIdx.y).
template <int TX, int TY, int NH, int FORM, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_step_fused(DevParams P, FusedBuffers B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fused_tile<TX, TY, NH, FORM, NT>(P, B, blockIdx.x * TX, blockIdx.y * TY,
                                      *reinterpret_cast<Smem<TX, TY, NH> *>(smem_raw));
}

// Many lattices in one launch: CTA b takes work item b = (case, tile origin);
// the case's parameters and buffers are staged in shared memory.  parity
// selects which of the case's two buffer sets is the input this step.
template <int TX, int TY, int NH, int FORM, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_step_batched(const BatchCase *__restrict__ cases,
                                                           const WorkItem *__restrict__ work, int parity) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DevParams sP;
  __shared__ FusedBuffers sB;
  const WorkItem w = work[blockIdx.x];
  if (threadIdx.x == 0) {
    sP = cases[w.case_id].P;
    sB = cases[w.case_id].B[cases[w.case_id].base_parity ^ parity];
  }
  __syncthreads();
  fused_tile<TX, TY, NH, FORM, NT>(sP, sB, w.x0, w.y0, *reinterpret_cast<Smem<TX, TY, NH> *>(smem_raw));
}

// ---------------------------------------------------------------- launcher

template <int TX, int TY, int NH, int FORM, int NT, int MINB>
static cudaError_t launch_fused_t(const DevParams &P, const FusedBuffers &B, cudaStream_t s) {
  static_assert(NT >= TX * TY, "one thread per output node in stage 3");
  const size_t smem = sizeof(Smem<TX, TY, NH>);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_step_fused<TX, TY, NH, FORM, NT, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const dim3 grd((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
  k_step_fused<TX, TY, NH, FORM, NT, MINB><<<grd, NT, smem, s>>>(P, B);
  return cudaGetLastError();
}

// nwork == 0 only sets the kernel's shared-memory attribute (done before any
// stream capture).
template <int TX, int TY, int NH, int FORM, int NT, int MINB>
static cudaError_t launch_batched_t(const BatchCase *cases, const WorkItem *work, int nwork, int parity,
                                   cudaStream_t s) {
  const size_t smem = sizeof(Smem<TX, TY, NH>);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_step_batched<TX, TY, NH, FORM, NT, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (nwork <= 0) return cudaSuccess;
  k_step_batched<TX, TY, NH, FORM, NT, MINB><<<nwork, NT, smem, s>>>(cases, work, parity);
  return cudaGetLastError();
}

// Launch configurations the autotuner chooses from: output tile TX x TY,
// threads per CTA (sized to one of the rings so that a heavy stage runs in a
// single pass) and the minimum resident CTAs per SM passed to the compiler.
template <int NH, int FORM>
struct VariantTable {
  static constexpr int kCount = FORM == 2 ? 2 : (NH == 1 ? 5 : 2);
  static const char *name(int v) {
    static const char *n1[5] = {"32x8/352/3", "32x8/448/2", "32x16/640/2", "64x8/704/1", "32x8/352/2"};
    static const char *n2[2] = {"32x8/352/2", "32x8/448/2"};
    static const char *n16[2] = {"32x8/352/3", "32x8/352/2"};
    return (FORM == 2 && NH == 1) ? n16[v] : (NH == 1 ? n1[v] : n2[v]);
  }
  static void tile(int v, int *tx, int *ty) {
    static const int t1[5][2] = {{32, 8}, {32, 8}, {32, 16}, {64, 8}, {32, 8}};
    *tx = t1[(NH == 1 && FORM != 2) ? v : 0][0];
    *ty = t1[(NH == 1 && FORM != 2) ? v : 0][1];
  }
  static cudaError_t launch_batched(int v, const BatchCase *c, const WorkItem *w, int n, int parity,
                                    cudaStream_t s) {
    if constexpr (FORM == 2) {
      return cudaErrorNotSupported;  // batches hold FP32 states
    } else if constexpr (NH == 1) {
      switch (v) {
        case 1: return launch_batched_t<32, 8, NH, FORM, 448, 2>(c, w, n, parity, s);
        case 2: return launch_batched_t<32, 16, NH, FORM, 640, 2>(c, w, n, parity, s);
        case 3: return launch_batched_t<64, 8, NH, FORM, 704, 1>(c, w, n, parity, s);
        case 4: return launch_batched_t<32, 8, NH, FORM, 352, 2>(c, w, n, parity, s);
        default: return launch_batched_t<32, 8, NH, FORM, 352, 3>(c, w, n, parity, s);
      }
    } else {
      switch (v) {
        case 1: return launch_batched_t<32, 8, NH, FORM, 448, 2>(c, w, n, parity, s);
        default: return launch_batched_t<32, 8, NH, FORM, 352, 2>(c, w, n, parity, s);
      }
    }
  }
  static cudaError_t launch(int v, const DevParams &P, const FusedBuffers &B, cudaStream_t s) {
    if constexpr (FORM == 2 && NH == 1) {
      return v == 1 ? launch_fused_t<32, 8, NH, FORM, 352, 2>(P, B, s) : launch_fused_t<32, 8, NH, FORM, 352, 3>(P, B, s);
    } else if constexpr (NH == 1) {
      switch (v) {
        case 1: return launch_fused_t<32, 8, NH, FORM, 448, 2>(P, B, s);
        case 2: return launch_fused_t<32, 16, NH, FORM, 640, 2>(P, B, s);
        case 3: return launch_fused_t<64, 8, NH, FORM, 704, 1>(P, B, s);
        case 4: return launch_fused_t<32, 8, NH, FORM, 352, 2>(P, B, s);
        default: return launch_fused_t<32, 8, NH, FORM, 352, 3>(P, B, s);
      }
    } else {
      switch (v) {
        case 1: return launch_fused_t<32, 8, NH, FORM, 448, 2>(P, B, s);
        default: return launch_fused_t<32, 8, NH, FORM, 352, 2>(P, B, s);
      }
    }
  }
};

static int form_of(const DevParams &P) { return P.g16 ? 2 : (P.collapse_h ? 1 : 0); }

int fused_variant_count(const DevParams &P) {
  if (form_of(P) == 2) return P.nh == 1 ? VariantTable<1, 2>::kCount : VariantTable<2, 2>::kCount;
  return P.nh == 1 ? VariantTable<1, 0>::kCount : VariantTable<2, 0>::kCount;
}

const char *fused_variant_name(const DevParams &P, int v) {
  if (v < 0 || v >= fused_variant_count(P)) v = 0;
  if (form_of(P) == 2) return P.nh == 1 ? VariantTable<1, 2>::name(v) : VariantTable<2, 2>::name(v);
  return P.nh == 1 ? VariantTable<1, 0>::name(v) : VariantTable<2, 0>::name(v);
}

cudaError_t launch_fused_step(const DevParams &P, const FusedBuffers &B, cudaStream_t s, int v) {
  if (v < 0 || v >= fused_variant_count(P)) v = 0;
  switch (form_of(P)) {
    case 2: return P.nh == 1 ? VariantTable<1, 2>::launch(v, P, B, s) : VariantTable<2, 2>::launch(v, P, B, s);
    case 1: return P.nh == 1 ? VariantTable<1, 1>::launch(v, P, B, s) : VariantTable<2, 1>::launch(v, P, B, s);
    default: return P.nh == 1 ? VariantTable<1, 0>::launch(v, P, B, s) : VariantTable<2, 0>::launch(v, P, B, s);
  }
}

void fused_variant_tile(const DevParams &P, int v, int *tx, int *ty) {
  if (v < 0 || v >= fused_variant_count(P)) v = 0;
  if (P.nh == 1) VariantTable<1, 0>::tile(v, tx, ty);
  else VariantTable<2, 0>::tile(v, tx, ty);
}

cudaError_t launch_batched_step(int nh, bool collapse_h, const BatchCase *cases, const WorkItem *work, int nwork,
                                int parity, cudaStream_t s, int v) {
  const int count = nh == 1 ? VariantTable<1, 0>::kCount : VariantTable<2, 0>::kCount;
  if (v < 0 || v >= count) v = 0;
  if (collapse_h) {
    if (nh == 1) return VariantTable<1, 1>::launch_batched(v, cases, work, nwork, parity, s);
    return VariantTable<2, 1>::launch_batched(v, cases, work, nwork, parity, s);
  }
  if (nh == 1) return VariantTable<1, 0>::launch_batched(v, cases, work, nwork, parity, s);
  return VariantTable<2, 0>::launch_batched(v, cases, work, nwork, parity, s);
}

// Conversions between the FP32 populations and the FORM 2 storage (initial
// state, field readback), one thread per node.
__global__ void k_g16_encode(DevParams P, const float *__restrict__ g32, float *__restrict__ g16) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.plane) return;
  float g[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) g[a] = g32[a * P.plane + k];
  const float Pn = g16_reference(g);
  g16[(9 * P.plane) / 2 + k] = Pn;
  __half *gh = reinterpret_cast<__half *>(g16);
#pragma unroll
  for (int a = 0; a < 9; ++a) gh[a * P.plane + k] = g16_encode(g[a], Pn, a, P.g16_scale);
}

__global__ void k_g16_decode(DevParams P, const float *__restrict__ g16, float *__restrict__ g32) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.plane) return;
  const float Pref = g16[(9 * P.plane) / 2 + k];
  const __half *gh = reinterpret_cast<const __half *>(g16);
#pragma unroll
  for (int a = 0; a < 9; ++a) g32[a * P.plane + k] = g16_decode(Pref, gh[a * P.plane + k], a, P.g16_inv_scale);
}

cudaError_t launch_g16_encode(const DevParams &P, const float *g32, float *g16, cudaStream_t s) {
  k_g16_encode<<<(unsigned)((P.plane + 255) / 256), 256, 0, s>>>(P, g32, g16);
  return cudaGetLastError();
}

cudaError_t launch_g16_decode(const DevParams &P, const float *g16, float *g32, cudaStream_t s) {
  k_g16_decode<<<(unsigned)((P.plane + 255) / 256), 256, 0, s>>>(P, g16, g32);
  return cudaGetLastError();
}

bool fused_supported(const DevParams &P) { return P.fd_scheme == 0; }

}  // namespace lbm
