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

#include "lbm_kernels.h"
#include "lbm_node.cuh"

namespace lbm {

namespace {

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
  // R1: post-collision h* and the diffusion sources
  float hs[NH][9][N1];
  float sv[NH][N1];
};

template <int TX>
__device__ __forceinline__ int i3(int lx, int ly) { return (ly + 3) * (TX + 6) + (lx + 3); }
template <int TX>
__device__ __forceinline__ int i2(int lx, int ly) { return (ly + 2) * (TX + 4) + (lx + 2); }
template <int TX>
__device__ __forceinline__ int i1(int lx, int ly) { return (ly + 1) * (TX + 2) + (lx + 1); }

}  // namespace

// FORM 0: the state holds the populations h^i (the method's state).
// FORM 1: the state holds C_i only.  With tau_h = 1/2 the collision of Eq. 18
// depends on h only through C_i = sum_a h_a^i, so C_i(t+1) = sum_a h_a^i(t+1)
// carries the same information (same results up to the order of the FP32
// sums) at 88 instead of 152 bytes per node-step; the destination-side term
// then sums to S_i / 2 because the Gamma_a sum to one.
// FORM 2: as FORM 1, and g is stored as FP16 deviations from a per-node
// reference: d_a = (g_a - w_a P) * scale with P = sum_a g_a kept in FP32 (the
// pressure-sized part stays in FP32, only the small deviations go to FP16),
// 60 bytes per node-step.  In memory: 9 half planes interleaved in blocks of
// 32 columns (pop_index), then the planar FP32 P plane, inside the space of the
// 9 FP32 planes.
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
    float c[NH];
    load_order_parameters<NH, FORM>(B, plane, k, c);
#pragma unroll
    for (int i = 0; i < NH; ++i) s.C[i][q] = c[i];
    s.rho[q] = node_rho<NH>(P, c);
  }
  __syncthreads();

  // ---- stage 1: g into shared memory; mu, gradients, u, p on R2 (real rows)
  for (int q = tid; q < S::N2; q += NT) {
    const int lx = q % S::W2 - 2, ly = q / S::W2 - 2;
    const int gy = y0 + ly;
    if (!per && (gy < 0 || gy >= ny)) continue;
    const long long k = (long long)(per ? wrap_periodic(gy, ny) : gy) * pitch + wrap_periodic(x0 + lx, nx);
    float g[9];
    load_populations<FORM>(P, B, plane, k, g);
    float cn[NH][9], rn[9];
    const int c0 = i3<TX>(lx, ly);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const int j3 = c0 + ey(a) * S::W3 + ex(a);
      s.g[a][q] = g[a];
#pragma unroll
      for (int i = 0; i < NH; ++i) cn[i][a] = s.C[i][j3];
      rn[a] = s.rho[j3];
    }
    NodeFields f;
    node_fields<NH>(P, g, cn, rn, f);
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      s.mu[i][q] = f.mu[i];
      s.dmu[i][q] = f.mu[i] - f.mu[2];
      s.gCx[i][q] = f.gCx[i];
      s.gCy[i][q] = f.gCy[i];
    }
    s.p[q] = f.p;
    s.ux[q] = f.ux;
    s.uy[q] = f.uy;
    s.grx[q] = f.rx;
    s.gry[q] = f.ry;
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
    float pn[9], rn[9], cn[NH][9], mun[NH][9], g[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const int j2 = c2 + ey(a) * S::W2 + ex(a), j3 = c3 + ey(a) * S::W3 + ex(a);
      pn[a] = s.p[j2];
      rn[a] = s.rho[j3];
      g[a] = s.g[a][c2];
#pragma unroll
      for (int i = 0; i < NH; ++i) {
        cn[i][a] = s.C[i][j3];
        mun[i][a] = s.mu[i][j2];
      }
    }
    NodeCenter c;
    c.ux = s.ux[c2];
    c.uy = s.uy[c2];
    c.p = pn[0];
    c.rho = rn[0];
    c.irho = __fdividef(1.0f, rn[0]);
    c.grx = s.grx[c2];
    c.gry = s.gry[c2];
    pair_diff(rn, c.Dr);
#pragma unroll
    for (int i = 0; i < NH; ++i) {
      c.dmu[i] = s.dmu[i][c2];
      c.gCx[i] = s.gCx[i][c2];
      c.gCy[i] = s.gCy[i][c2];
      c.C[i] = cn[i][0];
      pair_diff(cn[i], c.DC[i]);
    }
    float hs[NH][9], sv[NH], tn, gd2;
    node_collide<NH>(P, c, pn, mun, g, B.tau_in[k], hs, sv, tn, gd2);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      s.g[a][c2] = g[a];
#pragma unroll
      for (int i = 0; i < NH; ++i) s.hs[i][a][q] = hs[i][a];
    }
#pragma unroll
    for (int i = 0; i < NH; ++i) s.sv[i][q] = sv[i];
    if (lx >= 0 && lx < TX && ly >= 0 && ly < TY && x0 + lx < nx && gy < ny)
      store_diagnostics<NH>(B, plane, k, tn, gd2, sv, c);
  }
  __syncthreads();

  // ---- stage 3: streaming (pull) with bounce-back, destination-side term
  if (tid >= TX * TY) return;
  const int tx = tid % TX, ty = tid / TX;
  const int x = x0 + tx, y = y0 + ty;
  if (x >= nx || y >= ny) return;
  const long long ky = (long long)y * pitch + x;
  const int yc1 = i1<TX>(tx, ty), yc2 = i2<TX>(tx, ty);
  float gy[9], hy[NH][9], svy[NH];
#pragma unroll
  for (int i = 0; i < NH; ++i) svy[i] = s.sv[i][yc1];
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
    gy[a] = s.g[b][s2];
#pragma unroll
    for (int i = 0; i < NH; ++i) hy[i][a] = s.hs[i][b][s1];
  }
  store_node<NH, FORM>(P, B, plane, ky, gy, hy, svy, s.ux[yc2], s.uy[yc2]);
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

int tile_variant_count(const DevParams &P) {
  if (form_of(P) == 2) return P.nh == 1 ? VariantTable<1, 2>::kCount : VariantTable<2, 2>::kCount;
  return P.nh == 1 ? VariantTable<1, 0>::kCount : VariantTable<2, 0>::kCount;
}

// Configurations 0 .. sweep_variant_count - 1 are row sweeps, the rest tiles.
int fused_variant_count(const DevParams &P) { return sweep_variant_count(P) + tile_variant_count(P); }

const char *fused_variant_name(const DevParams &P, int v) {
  if (v < 0 || v >= fused_variant_count(P)) v = 0;
  const int ns = sweep_variant_count(P);
  if (v < ns) return sweep_variant_name(P, v);
  v -= ns;
  if (form_of(P) == 2) return P.nh == 1 ? VariantTable<1, 2>::name(v) : VariantTable<2, 2>::name(v);
  return P.nh == 1 ? VariantTable<1, 0>::name(v) : VariantTable<2, 0>::name(v);
}

cudaError_t launch_fused_step(const DevParams &P, const FusedBuffers &B, cudaStream_t s, int v) {
  if (v < 0 || v >= fused_variant_count(P)) v = 0;
  const int ns = sweep_variant_count(P);
  if (v < ns) return launch_sweep_step(P, B, s, v);
  v -= ns;
  switch (form_of(P)) {
    case 2: return P.nh == 1 ? VariantTable<1, 2>::launch(v, P, B, s) : VariantTable<2, 2>::launch(v, P, B, s);
    case 1: return P.nh == 1 ? VariantTable<1, 1>::launch(v, P, B, s) : VariantTable<2, 1>::launch(v, P, B, s);
    default: return P.nh == 1 ? VariantTable<1, 0>::launch(v, P, B, s) : VariantTable<2, 0>::launch(v, P, B, s);
  }
}

int batched_variant_count(int nh) {
  return sweep_batched_count(nh) + (nh == 1 ? VariantTable<1, 0>::kCount : VariantTable<2, 0>::kCount);
}

bool batched_variant_is_sweep(int nh, int v) { return v >= 0 && v < sweep_batched_count(nh); }

// Tile of configuration v (sweeps: strip width and segment rows).
void batched_variant_tile(int nh, int v, int *tx, int *ty) {
  if (v < 0 || v >= batched_variant_count(nh)) v = 0;
  const int ns = sweep_batched_count(nh);
  if (v < ns) return sweep_batched_shape(nh, v, tx, ty);
  v -= ns;
  if (nh == 1) VariantTable<1, 0>::tile(v, tx, ty);
  else VariantTable<2, 0>::tile(v, tx, ty);
}

cudaError_t launch_batched_step(int nh, int form, const BatchCase *cases, const WorkItem *work, int nwork,
                                int parity, cudaStream_t s, int v) {
  if (v < 0 || v >= batched_variant_count(nh)) v = 0;
  const int ns = sweep_batched_count(nh);
  if (v < ns) return launch_sweep_batched(nh, form, cases, work, nwork, parity, s, v);
  v -= ns;
  if (form == 2) {
    if (nh == 1) return VariantTable<1, 2>::launch_batched(v, cases, work, nwork, parity, s);
    return VariantTable<2, 2>::launch_batched(v, cases, work, nwork, parity, s);
  }
  if (form == 1) {
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
  for (int a = 0; a < 9; ++a) g[a] = g32[pop_index(k, a, 9)];
  const float Pn = g16_reference(g);
  g16[(9 * P.plane) / 2 + k] = Pn;
  __half *gh = reinterpret_cast<__half *>(g16);
#pragma unroll
  for (int a = 0; a < 9; ++a) gh[pop_index(k, a, 9)] = g16_encode(g[a], Pn, a, P.g16_scale);
}

__global__ void k_g16_decode(DevParams P, const float *__restrict__ g16, float *__restrict__ g32) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.plane) return;
  const float Pref = g16[(9 * P.plane) / 2 + k];
  const __half *gh = reinterpret_cast<const __half *>(g16);
#pragma unroll
  for (int a = 0; a < 9; ++a) g32[pop_index(k, a, 9)] = g16_decode(Pref, gh[pop_index(k, a, 9)], a, P.g16_inv_scale);
}

cudaError_t launch_g16_encode(const DevParams &P, const float *g32, float *g16, cudaStream_t s) {
  k_g16_encode<<<(unsigned)((P.plane + 255) / 256), 256, 0, s>>>(P, g32, g16);
  return cudaGetLastError();
}

cudaError_t launch_g16_decode(const DevParams &P, const float *g16, float *g32, cudaStream_t s) {
  k_g16_decode<<<(unsigned)((P.plane + 255) / 256), 256, 0, s>>>(P, g16, g32);
  return cudaGetLastError();
}

bool fused_supported(const DevParams &P) { return P.fd_scheme == 0 && !P.open_x; }

}  // namespace lbm
