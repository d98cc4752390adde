// Fused form of the coupled D2Q9 step (arXiv 2207.09431, Sec. 2.2-2.3): one
// kernel per time step, pull scheme, one CTA per TX x TY tile of output nodes.
//
// A population arriving at node y in direction a left x = y - e_a, so the tile
// needs the collision of its one-node ring R1; that collision needs p and mu
// on the two-node ring R2 (gradients and directional derivatives), which in
// turn need C on the three-node ring R3 (Laplacian inside mu).  The stages:
//   0  C_i = sum_a h_a^i (Eq. 22) and rho (mixture law R1) on R3
//   1  mu (Eq. 5), grad C, grad rho, u (Eq. 23), p (Eq. 24 / R3) on R2
//   2  S_i + V_i (Eq. 6, 21), new tau (Eq. 25-33) and per-node collision
//      coefficients on R1
//   3  per output node and direction: collision of g (Eq. 14) and h (Eq. 18,
//      tau_h = 1/2) at the source node, half-way bounce-back at walls,
//      destination-side source term (R9), coalesced stores.
// Intermediate values live in shared memory only; global memory sees the
// populations and tau read once and written once (halo reads hit L2).
// Ghost rows beyond a wall hold mirrored values (R10): loaded data is mirrored
// pointwise; stencil-derived values (mu, p) are copied from the mirror slot.
#include "lbm_device.cuh"
#include "lbm_kernels.h"

namespace lbm {

namespace {

__device__ __forceinline__ int map_x(int gx, int nx) {
  gx %= nx;
  return gx < 0 ? gx + nx : gx;
}

__device__ __forceinline__ int map_y(int gy, int ny, int periodic) {
  if (periodic) {
    gy %= ny;
    return gy < 0 ? gy + ny : gy;
  }
  int m = gy % (2 * ny);
  if (m < 0) m += 2 * ny;
  return m < ny ? m : 2 * ny - 1 - m;
}

template <int TX, int TY, int NH>
struct Smem {
  static constexpr int W3 = TX + 6, H3 = TY + 6, N3 = W3 * H3;
  static constexpr int W2 = TX + 4, H2 = TY + 4, N2 = W2 * H2;
  static constexpr int W1 = TX + 2, H1 = TY + 2, N1 = W1 * H1;
  // R3: order parameters and density
  float C[NH][N3];
  float rho[N3];
  // R2: chemical potentials of the transported components, mu_j - mu_3 for
  // the surface force, pressure, velocity, isotropic gradients of C and rho
  float mu[NH][N2];
  float dmu[NH][N2];
  float p[N2], ux[N2], uy[N2];
  float gCx[NH][N2], gCy[NH][N2], grx[N2], gry[N2];
  // R1: collision coefficients
  float om[N1], udr[N1], udFs[N1], udp[N1];
  float kap[NH][N1], udC[NH][N1], sv[NH][N1];
};

template <int TX, int TY, int NH>
__device__ __forceinline__ int i3(int lx, int ly) { return (ly + 3) * (TX + 6) + (lx + 3); }
template <int TX, int TY, int NH>
__device__ __forceinline__ int i2(int lx, int ly) { return (ly + 2) * (TX + 4) + (lx + 2); }
template <int TX, int TY, int NH>
__device__ __forceinline__ int i1(int lx, int ly) { return (ly + 1) * (TX + 2) + (lx + 1); }

}  // namespace

// STORE_H = true: the state holds the populations h^i (the method's state).
// STORE_H = false: the state holds C_i only.  With tau_h = 1/2 the collision
// of Eq. 18 depends on h only through C_i = sum_a h_a^i, so C_i(t+1) =
// sum_a h_a^i(t+1) carries the same information (same results up to the order
// of the FP32 sums) at 88 instead of 152 bytes per node-step.
template <int TX, int TY, int NH, bool STORE_H>
__global__ void __launch_bounds__(TX *TY) k_step_fused(DevParams P, FusedBuffers B) {
  using S = Smem<TX, TY, NH>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S &s = *reinterpret_cast<S *>(smem_raw);
  const int tid = threadIdx.y * TX + threadIdx.x;
  constexpr int NT = TX * TY;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const long long plane = P.plane;
  const int nx = P.nx, ny = P.ny, per = P.periodic_y;

  // ---- stage 0: C and rho on R3
  for (int q = tid; q < S::N3; q += NT) {
    const int lx = q % S::W3 - 3, ly = q / S::W3 - 3;
    const long long k = (long long)map_y(y0 + ly, ny, per) * P.pitch + map_x(x0 + lx, nx);
    float c[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      float acc = 0.f;
      if constexpr (STORE_H) {
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

  // ---- stage 1: mu, gradients, u, p on R2 (real nodes)
  for (int q = tid; q < S::N2; q += NT) {
    const int lx = q % S::W2 - 2, ly = q / S::W2 - 2;
    const int gy = y0 + ly;
    if (!per && (gy < 0 || gy >= ny)) continue;
    const long long k = (long long)(per ? map_y(gy, ny, 1) : gy) * P.pitch + map_x(x0 + lx, nx);
    float Cn[9][3], rn[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const int j3 = i3<TX, TY, NH>(lx + c_ex[a], ly + c_ey[a]);
      Cn[a][0] = s.C[0][j3];
      Cn[a][1] = NH == 2 ? s.C[NH - 1][j3] : 0.f;
      Cn[a][2] = 1.0f - Cn[a][0] - Cn[a][1];
      rn[a] = s.rho[j3];
    }
    float C[3], lap[3], gx[3], gyv[3], mu[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float sx = 0.f, sy = 0.f, lp = 0.f;
#pragma unroll
      for (int a = 1; a < 9; ++a) {
        sx += c_w[a] * c_ex[a] * Cn[a][j];
        sy += c_w[a] * c_ey[a] * Cn[a][j];
        lp += c_w[a] * (Cn[a][j] - Cn[0][j]);
      }
      C[j] = Cn[0][j];
      gx[j] = 3.0f * sx;
      gyv[j] = 3.0f * sy;
      lap[j] = 6.0f * lp;
    }
    float rx = 0.f, ry = 0.f;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      rx += c_w[a] * c_ex[a] * rn[a];
      ry += c_w[a] * c_ey[a] * rn[a];
    }
    rx *= 3.0f;
    ry *= 3.0f;
    chem_potentials(P, C, lap, mu);
    const float Fsx = mu[0] * gx[0] + mu[1] * gx[1] + mu[2] * gx[2];
    const float Fsy = mu[0] * gyv[0] + mu[1] * gyv[1] + mu[2] * gyv[2];
    const float rho = rn[0];
    float m0 = 0.f, mx = 0.f, my = 0.f;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const float ga = B.g_in[(long long)a * plane + k];
      m0 += ga;
      mx += c_ex[a] * ga;
      my += c_ey[a] * ga;
    }
    const float ux = (3.0f * mx + 0.5f * (Fsx + P.force_x)) / rho;
    const float uy = (3.0f * my + 0.5f * (Fsy - rho * P.gravity)) / rho;
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
      const int src = i2<TX, TY, NH>(lx, my);
#pragma unroll
      for (int i = 0; i < NH; ++i) s.mu[i][q] = s.mu[i][src];
      s.p[q] = s.p[src];
    }
    __syncthreads();
  }

  // ---- stage 2: sources, new tau and collision coefficients on R1
  for (int q = tid; q < S::N1; q += NT) {
    const int lx = q % S::W1 - 1, ly = q / S::W1 - 1;
    const int gy = y0 + ly;
    if (!per && (gy < 0 || gy >= ny)) continue;
    const int gxm = map_x(x0 + lx, nx);
    const int gym = per ? map_y(gy, ny, 1) : gy;
    const long long k = (long long)gym * P.pitch + gxm;
    const int c2 = i2<TX, TY, NH>(lx, ly);
    const int c3 = i3<TX, TY, NH>(lx, ly);
    const float ux = s.ux[c2], uy = s.uy[c2], p = s.p[c2], rho = s.rho[c3];
    // gradients of p and mu on the R2 stencil
    float px = 0.f, py = 0.f;
    float mgx[NH], mgy[NH], mlap[NH];
#pragma unroll
    for (int i = 0; i < NH; ++i) mgx[i] = mgy[i] = mlap[i] = 0.f;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
      const int j2 = i2<TX, TY, NH>(lx + c_ex[a], ly + c_ey[a]);
      px += c_w[a] * c_ex[a] * s.p[j2];
      py += c_w[a] * c_ey[a] * s.p[j2];
#pragma unroll
      for (int i = 0; i < NH; ++i) {
        const float m = s.mu[i][j2];
        mgx[i] += c_w[a] * c_ex[a] * m;
        mgy[i] += c_w[a] * c_ey[a] * m;
        mlap[i] += c_w[a] * (m - s.mu[i][c2]);
      }
    }
    px *= 3.0f;
    py *= 3.0f;
    float Fsx = 0.f, Fsy = 0.f;
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      Fsx += s.dmu[i][c2] * s.gCx[i][c2];
      Fsy += s.dmu[i][c2] * s.gCy[i][c2];
    }
    const float Fby = -rho * P.gravity;
    const float udr = ux * s.grx[c2] + uy * s.gry[c2];
    const float udFs = ux * Fsx + uy * Fsy;
    const float udFb = ux * P.force_x + uy * Fby;
    float Cc[3] = {s.C[0][c3], NH == 2 ? s.C[NH - 1][c3] : 0.f, 0.f};
    Cc[2] = 1.0f - Cc[0] - Cc[1];
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      const float C = Cc[i];
      const float D0s = P.D0 / P.Sig[i];
      const float lapmu = 6.0f * mlap[i];
      float sv;
      if (P.mobility == 1)
        sv = D0s * C * (1.0f - C) * lapmu +
             D0s * (1.0f - 2.0f * C) * (s.gCx[i][c2] * 3.0f * mgx[i] + s.gCy[i][c2] * 3.0f * mgy[i]);
      else
        sv = D0s * lapmu;
      s.sv[i][q] = sv;
      s.kap[i][q] = C / (rho * kCs2);
      s.udC[i][q] = ux * s.gCx[i][c2] + uy * s.gCy[i][c2];
    }
    // strain rate from the non-equilibrium part with the previous tau (R23)
    const float tp = B.tau_in[k];
    const float uu = ux * ux + uy * uy;
    float Pxx = 0.f, Pyy = 0.f, Pxy = 0.f;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const float ex = (float)c_ex[a], ey = (float)c_ey[a], w = c_w[a];
      const float eu = ex * ux + ey * uy;
      const float G = w * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * uu);
      const int jp = i3<TX, TY, NH>(lx + c_ex[a], ly + c_ey[a]);
      const int jm = i3<TX, TY, NH>(lx - c_ex[a], ly - c_ey[a]);
      const float dr = 0.5f * (s.rho[jp] - s.rho[jm]);
      float eFs = -udFs;
#pragma unroll
      for (int i = 0; i < NH; ++i) eFs += s.dmu[i][c2] * 0.5f * (s.C[i][jp] - s.C[i][jm]);
      const float eFb = ex * P.force_x + ey * Fby - udFb;
      const float phi = (dr - udr) * kCs2 * (G - w) + (eFs + eFb) * G;
      const float geq = w * p + rho * kCs2 * (G - w) - 0.5f * phi;
      const float fneq = B.g_in[(long long)a * plane + k] - geq;
      Pxx += fneq * ex * ex;
      Pyy += fneq * ey * ey;
      Pxy += fneq * ex * ey;
    }
    const float fac = 3.0f * (2.0f * tp / (2.0f * tp + 1.0f));
    const float den = 2.0f * tp * rho * kCs2;
    const float Dxx = -fac * Pxx / den, Dyy = -fac * Pyy / den, Dxy = -fac * Pxy / den;
    const float gd = sqrtf(2.0f * (Dxx * Dxx + Dyy * Dyy + 2.0f * Dxy * Dxy));
    const float tau1 = P.powerlaw ? tau_powerlaw(P, gd, rho) : P.tau[0];
    const float tn = tau_mix(P, Cc[0], Cc[1], Cc[2], tau1);
    s.om[q] = 1.0f / (tn + 0.5f);
    s.udr[q] = udr;
    s.udFs[q] = udFs;
    s.udp[q] = ux * px + uy * py;
    if (lx >= 0 && lx < TX && ly >= 0 && ly < TY && x0 + lx < nx && gy < ny) {
      B.tau_out[k] = tn;
      if (B.shear) B.shear[k] = gd;
      if (B.SV) {
#pragma unroll
        for (int i = 0; i < NH; ++i) B.SV[(long long)i * plane + k] = s.sv[i][q];
      }
      if (!(isfinite(tn) && isfinite(p) && isfinite(ux) && isfinite(uy))) atomicOr(B.err, 1u);
    }
  }
  __syncthreads();

  // ---- stage 3: collision at the source node, streaming, stores
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = x0 + tx, y = y0 + ty;
  if (x >= nx || y >= ny) return;
  const long long ky = (long long)y * P.pitch + x;
  const int yc1 = i1<TX, TY, NH>(tx, ty);
  const int yc2 = i2<TX, TY, NH>(tx, ty);
  const float uxy = s.ux[yc2], uyy = s.uy[yc2];
  const float uuy = uxy * uxy + uyy * uyy;
  float svy[NH], csum[NH];
#pragma unroll
  for (int i = 0; i < NH; ++i) {
    svy[i] = s.sv[i][yc1];
    csum[i] = 0.f;
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    int sxl = tx - c_ex[a], syl = ty - c_ey[a], b = a;
    long long ks;
    const int ys = y - c_ey[a];
    if (!per && (ys < 0 || ys >= ny)) {
      sxl = tx;
      syl = ty;
      b = c_opp[a];
      ks = ky;
    } else {
      ks = (long long)(per ? map_y(ys, ny, 1) : ys) * P.pitch + map_x(x - c_ex[a], nx);
    }
    const float gb = B.g_in[(long long)b * plane + ks];
    const int x1 = i1<TX, TY, NH>(sxl, syl);
    const int x2 = i2<TX, TY, NH>(sxl, syl);
    const int x3 = i3<TX, TY, NH>(sxl, syl);
    const int p3 = i3<TX, TY, NH>(sxl + c_ex[b], syl + c_ey[b]);
    const int m3 = i3<TX, TY, NH>(sxl - c_ex[b], syl - c_ey[b]);
    const int p2 = i2<TX, TY, NH>(sxl + c_ex[b], syl + c_ey[b]);
    const int m2 = i2<TX, TY, NH>(sxl - c_ex[b], syl - c_ey[b]);
    const float ex = (float)c_ex[b], ey = (float)c_ey[b], w = c_w[b];
    const float ux = s.ux[x2], uy = s.uy[x2], p = s.p[x2], rho = s.rho[x3];
    const float eu = ex * ux + ey * uy;
    const float G = w * (1.0f + 3.0f * eu + 4.5f * eu * eu - 1.5f * (ux * ux + uy * uy));
    const float Fby = -rho * P.gravity;
    const float eFb = ex * P.force_x + ey * Fby - (ux * P.force_x + uy * Fby);
    float eFs = -s.udFs[x1];
    float dC[NH];
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      dC[i] = 0.5f * (s.C[i][p3] - s.C[i][m3]);
      eFs += s.dmu[i][x2] * dC[i];
    }
    const float dr = 0.5f * (s.rho[p3] - s.rho[m3]);
    const float phig = (dr - s.udr[x1]) * kCs2 * (G - w) + (eFs + eFb) * G;
    const float geq = w * p + rho * kCs2 * (G - w) - 0.5f * phig;
    const float om = s.om[x1];
    B.g_out[(long long)a * plane + ky] = gb - om * (gb - geq) + phig;
    const float dp = 0.5f * (s.p[p2] - s.p[m2]);
    const float ep = dp - s.udp[x1];
    // destination-side term at y uses Gamma_a(u(y))
    const float euy = c_ex[a] * uxy + c_ey[a] * uyy;
    const float Gy = c_w[a] * (1.0f + 3.0f * euy + 4.5f * euy * euy - 1.5f * uuy);
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      const float phih = (dC[i] - s.udC[i][x1] - s.kap[i][x1] * (ep - eFs - eFb)) * G;
      const float hstar = s.C[i][x3] * G + 0.5f * phih + 0.5f * s.sv[i][x1] * G;
      const float hy = hstar + 0.5f * svy[i] * Gy;
      if constexpr (STORE_H) {
        B.h_out[((long long)i * 9 + a) * plane + ky] = hy;
      } else {
        csum[i] += hy;
      }
    }
  }
  if constexpr (!STORE_H) {
#pragma unroll
    for (int i = 0; i < NH; ++i) B.h_out[(long long)i * plane + ky] = csum[i];
  }
}

// ---------------------------------------------------------------- launcher

template <int TX, int TY, int NH, bool STORE_H>
static void launch_fused_t(const DevParams &P, const FusedBuffers &B, cudaStream_t s) {
  const size_t smem = sizeof(Smem<TX, TY, NH>);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_step_fused<TX, TY, NH, STORE_H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    configured = true;
  }
  const dim3 blk(TX, TY);
  const dim3 grd((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
  k_step_fused<TX, TY, NH, STORE_H><<<grd, blk, smem, s>>>(P, B);
}

void launch_fused_step(const DevParams &P, const FusedBuffers &B, cudaStream_t s) {
  if (P.collapse_h) {
    if (P.nh == 1) launch_fused_t<32, 8, 1, false>(P, B, s);
    else launch_fused_t<32, 8, 2, false>(P, B, s);
  } else {
    if (P.nh == 1) launch_fused_t<32, 8, 1, true>(P, B, s);
    else launch_fused_t<32, 8, 2, true>(P, B, s);
  }
}

bool fused_supported(const DevParams &P) { return P.fd_scheme == 0; }

}  // namespace lbm
