// Row-sweep form of the fused coupled D2Q9 step (arXiv 2207.09431, Sec.
// 2.2-2.3): one kernel per time step, pull scheme, the same per-node
// arithmetic as the tile form (lbm_node.cuh).
//
// A CTA owns a strip of TX columns and a segment of rows and walks up the
// segment RS rows per pipeline step.  The four stages of the step run skewed
// by one pipeline step each, so that within a step no stage reads what
// another stage writes in the same step and a single barrier per step
// suffices:
//   stage 0  C and rho                      rows [j + 3RS + 3, j + 4RS + 3)
//   stage 1  mu, p, u, isotropic gradients   rows [j + 2RS + 2, j + 3RS + 2)
//   stage 2  collision (h*, tau, g*)         rows [j + RS + 1,  j + 2RS + 1)
//   stage 3  streaming of output rows        rows [j, j + RS)
// Every stage reads rows that earlier steps produced (stage 1 needs C one row
// beyond its own, stage 2 needs mu and p one row beyond, stage 3 the
// collision one row beyond).  Each quantity lives in a shared-memory ring
// indexed by row, deep enough for the rows alive at once.  A node's stage
// 0-2 work is done once per segment instead of once per overlapping tile
// halo: the halo is recomputed only across strip edges (3, 2, 1 columns per
// side) and at segment ends (3, 2, 1 rows per end).
//
// Each thread owns one item of every stage (NT >= RS (TX + 6)), with its
// column fixed for the whole sweep and the ring slots of its rows kept in
// registers.  The global loads of the next step (state of stage 0, g of stage
// 1, previous tau of stage 2) are issued in the middle of a step, after stage
// 1, and consumed in the next one, so their latency overlaps a whole step of
// shared-memory work; a node's population directions lie at constant offsets
// of one address (the interleaved layout of pop_index).
//
// Ghost rows beyond a wall (reading R10): stage 0 loads mirrored rows;
// stencils of mu and p in stage 2 read the mirror row, which is the centre
// row itself for the one-row reach of those stencils; stage 3 bounces back.
#include <cuda_fp16.h>

#include "lbm_kernels.h"
#include "lbm_node.cuh"

namespace lbm {

namespace {

// Ring records: (C_1 .. C_NH, rho) and (mu_1 .. mu_NH, p) are one vector each,
// so that a stencil point costs one shared-memory access.
template <int NH>
struct PairVec;
template <>
struct PairVec<1> {
  using T = float2;
  static __device__ __forceinline__ T make(const float *c, float last) { return make_float2(c[0], last); }
  static __device__ __forceinline__ float comp(const T &v, int) { return v.x; }
  static __device__ __forceinline__ float last(const T &v) { return v.y; }
};
template <>
struct PairVec<2> {
  using T = float4;
  static __device__ __forceinline__ T make(const float *c, float last) { return make_float4(c[0], c[1], last, 0.f); }
  static __device__ __forceinline__ float comp(const T &v, int q) { return q == 0 ? v.x : v.y; }
  static __device__ __forceinline__ float last(const T &v) { return v.z; }
};

// Post-collision populations of the 1-ring, stage 2 -> stage 3: stage 3 reads
// g*_b and h*_b of one source node and direction together, so with one
// h set they are one float2 per direction and node.
template <int NH, int DB, int W1>
struct PostRing {
  float gs[9][DB][W1];
  float hs[NH][9][DB][W1];
  __device__ __forceinline__ void put(int a, int r, int c, float g, const float (&h)[NH][9]) {
    gs[a][r][c] = g;
#pragma unroll
    for (int q = 0; q < NH; ++q) hs[q][a][r][c] = h[q][a];
  }
  __device__ __forceinline__ void get(int b, int r, int c, int a, float (&g)[9], float (&h)[NH][9]) const {
    g[a] = gs[b][r][c];
#pragma unroll
    for (int q = 0; q < NH; ++q) h[q][a] = hs[q][b][r][c];
  }
};
template <int DB, int W1>
struct PostRing<1, DB, W1> {
  float2 gh[9][DB][W1];
  __device__ __forceinline__ void put(int a, int r, int c, float g, const float (&h)[1][9]) {
    gh[a][r][c] = make_float2(g, h[0][a]);
  }
  __device__ __forceinline__ void get(int b, int r, int c, int a, float (&g)[9], float (&h)[1][9]) const {
    const float2 v = gh[b][r][c];
    g[a] = v.x;
    h[0][a] = v.y;
  }
};

// REC: the collision's own C_i, rho, 1 / rho and the pair differences of rho
// and C_i travel from stage 1 in the record, and stage 2 reads no (C, rho)
// ring.  Used by the C state forms; the population form reads them again from
// the ring, because the larger record would push the shared memory of three
// CTAs past the carveout that leaves its (larger) loads in flight enough L1.
template <int TX, int RS, int NH, bool REC>
struct PipeSmem {
  using PV = PairVec<NH>;
  using V = typename PV::T;
  static constexpr int W3 = TX + 6, W2 = TX + 4, W1 = TX + 2;
  // ring depths: rows alive at once (written this step or read this step)
  static constexpr int D3 = REC ? 2 * RS + 2 : 3 * RS + 3, D2 = 2 * RS + 2, DA = 2 * RS + 1, DB = 2 * RS + 2;
  // stage 1 -> stage 2 record of a 1-ring node, in float4 words: g_0..g_8,
  // u_x, u_y, grad rho, then mu_i - mu_3, d_x C_i, d_y C_i per component, and
  // (REC) C_i, rho, 1 / rho and the pair differences of rho and of each C_i
  static constexpr int NR = REC ? 19 + 8 * NH : 13 + 3 * NH, NQ = (NR + 3) / 4;
  float4 da[NQ][DA][W1];
  V cr[D3][W3];  // (C_i, rho) of the 3-ring
  V mp[D2][W2];  // (mu_i, p) of the 2-ring
  // stage 2 -> stage 3: velocity of the collision node, g*, h*, sources
  float2 uvb[DB][W1];
  PostRing<NH, DB, W1> post;
  float svb[NH][DB][W1];
};

// Ring slot arithmetic: every thread's rows move up RS rows per step, so its
// slots are kept in registers and advanced, and the slots of the rows next to
// a slot are one step around the ring.
template <int D, int N>
__device__ __forceinline__ int ring_add(int s) {
  static_assert(N < D, "advance within one turn of the ring");
  s += N;
  return s >= D ? s - D : s;
}
template <int D>
__device__ __forceinline__ int ring_up(int s) { return s == D - 1 ? 0 : s + 1; }
template <int D>
__device__ __forceinline__ int ring_dn(int s) { return s == 0 ? D - 1 : s - 1; }
// slot of row r + ey from those of rows r - 1, r, r + 1
__device__ __forceinline__ int row_slot(int dy, int sdn, int s, int sup) { return dy < 0 ? sdn : (dy > 0 ? sup : s); }

// The sweep of one strip [x0, x0 + TX) over output rows [ys, ye).  PER: 0 walls
// in y, 1 periodic y, 2 taken from P at run time (batches mix both).
template <int TX, int RS, int NH, int FORM, int PER, int NT>
__device__ __forceinline__ void sweep_body(const DevParams &P, const FusedBuffers &B, int x0, int ys, int ye,
                                           PipeSmem<TX, RS, NH, FORM != 0> &s) {
  constexpr bool REC = FORM != 0;
  using S = PipeSmem<TX, RS, NH, REC>;
  using PV = typename S::PV;
  using V = typename S::V;
  static_assert(NT >= RS * S::W3, "one item of every stage per thread");
  const int per = PER == 2 ? P.periodic_y : PER;
  const int nx = P.nx, ny = P.ny, pitch = P.pitch;
  const long long plane = P.plane;
  const int t = threadIdx.x;

  // this thread's item of each stage: row offset within the step, column
  const bool v0 = t < RS * S::W3, v1 = t < RS * S::W2, v2 = t < RS * S::W1, v3 = t < RS * TX;
  const int d0 = t / S::W3, c0 = t % S::W3;
  const int d1 = t / S::W2, c1 = t % S::W2;
  const int d2 = t / S::W1, c2 = t % S::W1;
  const int d3 = t / TX, c3 = t % TX;
  const int x0c = wrap_periodic(x0 - 3 + c0, nx);
  const int x1c = wrap_periodic(x0 - 2 + c1, nx);
  const int x2 = x0 - 1 + c2, x2c = wrap_periodic(x2, nx);
  const int x3 = x0 + c3;
  const bool own2 = c2 >= 1 && c2 <= TX && x2 < nx;
  const bool out3 = v3 && x3 < nx;

  // first step: stage 0 starts at row ys - 3, and j stays aligned with ys
  const int j0 = ys - 3 * RS - RS * ((6 + RS - 1) / RS);
  // Ring rows are counted from j0: the slot of row r in a ring of depth D is
  // (r - j0) mod D.  The slots of this thread's rows at the first step:
  int s0 = (3 * RS + 3 + d0) % S::D3;                                        // stage 0 row
  int s1c = (2 * RS + 2 + d1) % S::D3, s1m = (2 * RS + 2 + d1) % S::D2;      // stage 1 row
  int s1a = (2 * RS + 2 + d1) % S::DA;
  int s2c = (RS + 1 + d2) % S::D3, s2m = (RS + 1 + d2) % S::D2;              // stage 2 row
  int s2a = (RS + 1 + d2) % S::DA, s2b = (RS + 1 + d2) % S::DB;
  int s3 = d3 % S::DB;                                                       // stage 3 row

  // Global loads run one pipeline step ahead: the values a step consumes were
  // requested during the previous step, so their latency overlaps a whole
  // step of shared-memory work.  A thread's stage items move up RS rows per
  // step, so the next step's items are this step's plus RS.
  constexpr int NS0 = FORM == 0 ? 9 * NH : NH;
  float nh[NS0];            // state values of the next stage-0 item
  float ng[9];              // g of the next stage-1 item (FP32 forms)
  __half ngh[9];            // ... (FP16 form: the nine deviations
  float nP = 0.f;           //      and their FP32 reference)
  float nt = 0.f;           // previous tau of the next stage-2 item
  // A step is interior when the rows of its stage 0-2 items all lie inside
  // the segment's halo and inside the lattice (the same for every thread):
  // then every item is active, no row is mirrored and none wraps.  Used by the
  // population form; the C forms ran slower with it (measured) and keep the
  // general tests.
  const int lo_row = max(ys - 1, 0), hi_row = min(ye + 3, ny);
  auto interior = [&](int j) { return FORM == 0 && j + RS + 1 >= lo_row && j + 4 * RS + 3 <= hi_row; };
  auto item_rows = [&](int j, int &r0, int &r1, int &r2, bool &a0, bool &a1, bool &a2) {
    r0 = j + 3 * RS + 3 + d0;
    r1 = j + 2 * RS + 2 + d1;
    r2 = j + RS + 1 + d2;
    if (interior(j)) {
      a0 = v0;
      a1 = v1;
      a2 = v2;
    } else {
      a0 = v0 && r0 >= ys - 3 && r0 < ye + 3;
      a1 = v1 && r1 >= ys - 2 && r1 < ye + 2 && (per || (r1 >= 0 && r1 < ny));
      a2 = v2 && r2 >= ys - 1 && r2 < ye + 1 && (per || (r2 >= 0 && r2 < ny));
    }
  };
  auto issue = [&](int j) {
    int r0, r1, r2;
    bool a0, a1, a2;
    item_rows(j, r0, r1, r2, a0, a1, a2);
    const bool in = interior(j);
    if (a0) {
      const long long k0 = (long long)(in ? r0 : row_read(r0, ny, per)) * pitch + x0c;
      if constexpr (FORM == 0) {
        const float *hp = B.h_in + pop_index(k0, 0, NS0);
#pragma unroll
        for (int q = 0; q < NS0; ++q) nh[q] = hp[q * 32];
      } else {
#pragma unroll
        for (int q = 0; q < NS0; ++q) nh[q] = B.h_in[(long long)q * plane + k0];
      }
    }
    if (a1) {
      const long long k1 = (long long)(per && !in ? wrap_periodic(r1, ny) : r1) * pitch + x1c;
      if constexpr (FORM == 2) {
        const __half *gh = reinterpret_cast<const __half *>(B.g_in) + pop_index(k1, 0, 9);
        nP = B.g_in[(9 * plane) / 2 + k1];
#pragma unroll
        for (int a = 0; a < 9; ++a) ngh[a] = gh[a * 32];
      } else {
        const float *gp = B.g_in + pop_index(k1, 0, 9);
#pragma unroll
        for (int a = 0; a < 9; ++a) ng[a] = gp[a * 32];
      }
    }
    if (a2) nt = B.tau_in[(long long)(per && !in ? wrap_periodic(r2, ny) : r2) * pitch + x2c];
  };
  issue(j0);

  // ---- stage 0: C and rho of row r0 (3-ring column c0), from the loads of
  // the previous step
  auto stage0 = [&]() {
    float cst[NH];
#pragma unroll
    for (int q = 0; q < NH; ++q) {
      if constexpr (FORM == 0) {
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < 9; ++a) acc += nh[q * 9 + a];
        cst[q] = acc;
      } else {
        cst[q] = nh[q];
      }
    }
    s.cr[s0][c0] = PV::make(cst, node_rho<NH>(P, cst));
  };
  // ---- stage 1: fields of row r1 (2-ring column c1): the arithmetic, then
  // the stores of its results
  auto stage1_compute = [&](const float (&gv)[9], NodeFields &f) {
    const int cdn = ring_dn<S::D3>(s1c), cup = ring_up<S::D3>(s1c);
    float cn[NH][9], rn[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const V v = s.cr[row_slot(ey(a), cdn, s1c, cup)][c1 + 1 + ex(a)];
#pragma unroll
      for (int q = 0; q < NH; ++q) cn[q][a] = PV::comp(v, q);
      rn[a] = PV::last(v);
    }
    node_fields<NH>(P, gv, cn, rn, f);
  };
  auto stage1_store = [&](const float (&gv)[9], const NodeFields &f) {
    s.mp[s1m][c1] = PV::make(f.mu, f.p);
    if (c1 >= 1 && c1 <= TX + 2) {
      float rec[4 * S::NQ];
#pragma unroll
      for (int a = 0; a < 9; ++a) rec[a] = gv[a];
      rec[9] = f.ux;
      rec[10] = f.uy;
      rec[11] = f.rx;
      rec[12] = f.ry;
#pragma unroll
      for (int q = 0; q < NH; ++q) {
        rec[13 + q] = f.mu[q] - f.mu[2];
        rec[13 + NH + q] = f.gCx[q];
        rec[13 + 2 * NH + q] = f.gCy[q];
      }
      if constexpr (REC) {
#pragma unroll
        for (int q = 0; q < NH; ++q) rec[13 + 3 * NH + q] = f.C[q];
        rec[13 + 4 * NH] = f.rho;
        rec[14 + 4 * NH] = f.irho;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          rec[15 + 4 * NH + k] = f.Dr[k];
#pragma unroll
          for (int q = 0; q < NH; ++q) rec[19 + 4 * NH + 4 * q + k] = f.DC[q][k];
        }
      }
#pragma unroll
      for (int k = S::NR; k < 4 * S::NQ; ++k) rec[k] = 0.f;
#pragma unroll
      for (int k = 0; k < S::NQ; ++k)
        s.da[k][s1a][c1 - 1] = make_float4(rec[4 * k], rec[4 * k + 1], rec[4 * k + 2], rec[4 * k + 3]);
    }
  };
  auto stage1_values = [&](float (&gv)[9]) {
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      if constexpr (FORM == 2) gv[a] = g16_decode(nP, ngh[a], a, P.g16_inv_scale);
      else gv[a] = ng[a];
    }
  };
  // ---- stage 3: arriving populations of output row r3
  auto stage3 = [&](int j, int r3) {
    const int sdn = ring_dn<S::DB>(s3), sup = ring_up<S::DB>(s3);
    float gy[9], hy[NH][9], svy[NH];
#pragma unroll
    for (int q = 0; q < NH; ++q) svy[q] = s.svb[q][s3][c3 + 1];
    const float2 uv = s.uvb[s3][c3 + 1];
    if (per || (j >= 1 && j + RS <= ny - 1)) {
      // no output row of this step is next to a wall
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        const int ss = row_slot(-ey(a), sdn, s3, sup), cs = c3 + 1 - ex(a);  // source row r3 - e_a
        s.post.get(a, ss, cs, a, gy, hy);
      }
    } else {
      const bool lo = r3 == 0, hi = r3 == ny - 1;
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        // half-way bounce-back: a source row beyond the wall means the
        // population left r3 in -e_a
        const bool bb = (ey(a) > 0 && lo) || (ey(a) < 0 && hi);
        const int ss = bb ? s3 : row_slot(-ey(a), sdn, s3, sup);
        const int cs = bb ? c3 + 1 : c3 + 1 - ex(a);
        const int b = bb ? opp(a) : a;
        s.post.get(b, ss, cs, a, gy, hy);
      }
    }
    store_node<NH, FORM>(P, B, plane, (long long)r3 * pitch + x3, gy, hy, svy, uv.x, uv.y);
  };
  // ---- stage 2: collision of row r2 (1-ring column c2): the arithmetic,
  // then the stores of its results
  struct Collided {
    NodeCenter nc;
    float g2[9], hs[NH][9], sv[NH], tn, gd2;
  };
  auto stage2_compute = [&](int r2, float tprev, Collided &o) {
    const int cdn = ring_dn<S::D3>(s2c), cup = ring_up<S::D3>(s2c);
    int mdn = ring_dn<S::D2>(s2m), mup = ring_up<S::D2>(s2m);
    if (!per) {
      // mu and p one row beyond a wall: the mirror row is row r2 itself
      if (r2 == 0) mdn = s2m;
      if (r2 == ny - 1) mup = s2m;
    }
    float pn[9], mun[NH][9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const V mp = s.mp[row_slot(ey(a), mdn, s2m, mup)][c2 + 1 + ex(a)];
      pn[a] = PV::last(mp);
#pragma unroll
      for (int q = 0; q < NH; ++q) mun[q][a] = PV::comp(mp, q);
    }
    float rec[4 * S::NQ];
#pragma unroll
    for (int k = 0; k < S::NQ; ++k) {
      const float4 w = s.da[k][s2a][c2];
      rec[4 * k] = w.x;
      rec[4 * k + 1] = w.y;
      rec[4 * k + 2] = w.z;
      rec[4 * k + 3] = w.w;
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) o.g2[a] = rec[a];
    NodeCenter &nc = o.nc;
    nc.ux = rec[9];
    nc.uy = rec[10];
    nc.grx = rec[11];
    nc.gry = rec[12];
    nc.p = pn[0];
#pragma unroll
    for (int q = 0; q < NH; ++q) {
      nc.dmu[q] = rec[13 + q];
      nc.gCx[q] = rec[13 + NH + q];
      nc.gCy[q] = rec[13 + 2 * NH + q];
    }
    if constexpr (REC) {
#pragma unroll
      for (int q = 0; q < NH; ++q) nc.C[q] = rec[13 + 3 * NH + q];
      nc.rho = rec[13 + 4 * NH];
      nc.irho = rec[14 + 4 * NH];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        nc.Dr[k] = rec[15 + 4 * NH + k];
#pragma unroll
        for (int q = 0; q < NH; ++q) nc.DC[q][k] = rec[19 + 4 * NH + 4 * q + k];
      }
    } else {
      // C and rho of the 3x3 stencil from the ring
      float rn[9], cn[NH][9];
#pragma unroll
      for (int a = 0; a < 9; ++a) {
        const V cr = s.cr[row_slot(ey(a), cdn, s2c, cup)][c2 + 2 + ex(a)];
        rn[a] = PV::last(cr);
#pragma unroll
        for (int q = 0; q < NH; ++q) cn[q][a] = PV::comp(cr, q);
      }
      nc.rho = rn[0];
      nc.irho = __fdividef(1.0f, rn[0]);
      pair_diff(rn, nc.Dr);
#pragma unroll
      for (int q = 0; q < NH; ++q) {
        nc.C[q] = cn[q][0];
        pair_diff(cn[q], nc.DC[q]);
      }
    }
    node_collide<NH>(P, nc, pn, mun, o.g2, tprev, o.hs, o.sv, o.tn, o.gd2);
  };
  auto stage2_store = [&](int r2, long long k2, const Collided &o) {
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      s.post.put(a, s2b, c2, o.g2[a], o.hs);
    }
#pragma unroll
    for (int q = 0; q < NH; ++q) s.svb[q][s2b][c2] = o.sv[q];
    s.uvb[s2b][c2] = make_float2(o.nc.ux, o.nc.uy);
    if (own2 && r2 >= ys && r2 < ye) store_diagnostics<NH>(B, plane, k2, o.tn, o.gd2, o.sv, o.nc);
  };

  for (int j = j0; j < ye; j += RS) {
    int r0, r1, r2;
    bool a0, a1, a2;
    item_rows(j, r0, r1, r2, a0, a1, a2);
    const int r3 = j + d3;
    const bool a3 = out3 && r3 >= ys && r3 < ye;
    const long long k2 = (long long)(per && !interior(j) ? wrap_periodic(r2, ny) : r2) * pitch + x2c;

    if (a0) stage0();
    if (a1) {
      float gv[9];
      stage1_values(gv);
      NodeFields f;
      stage1_compute(gv, f);
      stage1_store(gv, f);
    }
    const float tprev = nt;
    issue(j + RS);  // the next step's loads
    if (a3) stage3(j, r3);
    if (a2) {
      Collided o;
      stage2_compute(r2, tprev, o);
      stage2_store(r2, k2, o);
    }

    s0 = ring_add<S::D3, RS>(s0);
    s1c = ring_add<S::D3, RS>(s1c);
    s1m = ring_add<S::D2, RS>(s1m);
    s1a = ring_add<S::DA, RS>(s1a);
    s2c = ring_add<S::D3, RS>(s2c);
    s2m = ring_add<S::D2, RS>(s2m);
    s2a = ring_add<S::DA, RS>(s2a);
    s2b = ring_add<S::DB, RS>(s2b);
    s3 = ring_add<S::DB, RS>(s3);
    __syncthreads();
  }
}

// Rows of a pipeline fill: the steps before a segment's first output row, as
// rows of work (stage 0 starts 3 RS + RS ceil(6 / RS) rows before it).
template <int RS>
__host__ __device__ constexpr int fill_rows() { return 3 * RS + RS * ((6 + RS - 1) / RS); }

// CTA (x, y) sweeps strip x over rows [y seg_len, (y + 1) seg_len).
template <int TX, int RS, int NH, int FORM, int PER, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_step_sweep(DevParams P, FusedBuffers B, int seg_len) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ys = blockIdx.y * seg_len;
  sweep_body<TX, RS, NH, FORM, PER, NT>(P, B, blockIdx.x * TX, ys, min(ys + seg_len, P.ny),
                                        *reinterpret_cast<PipeSmem<TX, RS, NH, FORM != 0> *>(smem_raw));
}

// Many lattices in one launch: CTA b sweeps work item b = (case, strip origin,
// rows [y0, y1)); the case's parameters and buffers are staged in shared memory.
// parity selects which of the case's two buffer sets is the input this step.
template <int TX, int RS, int NH, int FORM, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_sweep_batched(const BatchCase *__restrict__ cases,
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
  sweep_body<TX, RS, NH, FORM, 2, NT>(sP, sB, w.x0, w.y0, w.y1,
                                      *reinterpret_cast<PipeSmem<TX, RS, NH, FORM != 0> *>(smem_raw));
}

// Grid-wide barrier between the time steps of the persistent batched sweep.
// One thread per CTA arrives (after a fence that publishes the CTA's writes
// of this step) and polls the generation word; the CTA's other threads wait
// at the CTA barrier, which orders them after that thread's acquire.  Every
// poll also reads the status word, so that a wait elsewhere that ran out ends
// this one too; after spin_limit polls the wait sets kSyncTimeout itself.
// Returns false when the kernel must stop.
__device__ __forceinline__ bool grid_barrier(GridSync *gs, unsigned nblocks, long long spin_limit) {
  __shared__ int go_on;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = &gs->gen;
    volatile unsigned *vstatus = &gs->status;
    const unsigned g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&gs->count, 1u) + 1u == nblocks) {
      atomicExch(&gs->count, 0u);
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    } else {
      long long polls = 0;
      while (*vgen == g) {
        if (*vstatus != 0u) {
          ok = 0;
          break;
        }
        if (++polls > spin_limit) {
          atomicOr(&gs->status, kSyncTimeout);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*vstatus != 0u) ok = 0;
    go_on = ok;
  }
  __syncthreads();
  return go_on != 0;
}

// The batched sweep as one persistent launch: in every time step CTA b takes
// work item b first and then, while items are left, the next one from the
// step's counter (items longest first, so that this approximates the
// longest-processing-time schedule online); all CTAs (resident at once: a
// cooperative launch) meet at the grid barrier before the next step reads
// what this one wrote.  Every CTA takes items until the counter runs past the
// list, before it reaches the barrier, so a step's counter is idle from that
// barrier on: block 0 clears it during the step after, for the step after that.
template <int TX, int RS, int NH, int FORM, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_sweep_persistent(const BatchCase *__restrict__ cases,
                                                               const WorkItem *__restrict__ work, int nwork,
                                                               int parity0, int nsteps, GridSync *sync,
                                                               long long spin_limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DevParams sP;
  __shared__ FusedBuffers sB;
  __shared__ int s_next;
  for (int t = 0; t < nsteps; ++t) {
    const int parity = (parity0 + t) & 1;
    if (blockIdx.x == 0 && threadIdx.x == 0) sync->next[(t + 1) & 1] = 0u;  // last used in step t - 1
    for (int i = blockIdx.x; i < nwork;) {
      const WorkItem w = work[i];
      if (threadIdx.x == 0) {
        sP = cases[w.case_id].P;
        sB = cases[w.case_id].B[cases[w.case_id].base_parity ^ parity];
      }
      __syncthreads();
      sweep_body<TX, RS, NH, FORM, 2, NT>(sP, sB, w.x0, w.y0, w.y1,
                                          *reinterpret_cast<PipeSmem<TX, RS, NH, FORM != 0> *>(smem_raw));
      __syncthreads();  // sP and sB are rewritten by the next item
      if (threadIdx.x == 0) s_next = (int)gridDim.x + (int)atomicAdd(&sync->next[t & 1], 1u);
      __syncthreads();
      i = s_next;
    }
    if (t + 1 < nsteps && !grid_barrier(sync, gridDim.x, spin_limit)) return;
  }
}

// Segment length for a strip count: the number of segments per strip that
// minimises the rows the slowest CTA sweeps, waves x (segment rows + the
// pipeline fill of fill rows), with the rows of a strip split evenly (a multiple of
// rs each, the last segment the shortest).
int choose_segment(int ny, int strips, int resident, int rs, int fill) {
  int best_len = ny;
  long long best_cost = -1;
  for (int nseg = 1; nseg <= (ny + rs - 1) / rs; ++nseg) {
    int len = (ny + nseg - 1) / nseg;
    len = (len + rs - 1) / rs * rs;
    if ((ny + len - 1) / len != nseg) continue;  // rounding merged two segments
    const long long total = (long long)strips * nseg;
    const long long waves = (total + resident - 1) / resident;
    const long long cost = waves * (len + fill);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best_len = len;
    }
  }
  return best_len;
}

template <int TX, int RS, int NH, int FORM, int PER, int NT, int MINB>
cudaError_t launch_sweep_per(const DevParams &P, const FusedBuffers &B, cudaStream_t st) {
  const size_t smem = sizeof(PipeSmem<TX, RS, NH, FORM != 0>);
  static bool configured = false;
  static int resident_per_sm = 0, sms = 0;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_step_sweep<TX, RS, NH, FORM, PER, NT, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident_per_sm,
                                                        k_step_sweep<TX, RS, NH, FORM, PER, NT, MINB>, NT, smem);
    if (e != cudaSuccess) return e;
    if (resident_per_sm < 1) return cudaErrorInvalidConfiguration;
    configured = true;
  }
  const int strips = (P.nx + TX - 1) / TX;
  const int len = choose_segment(P.ny, strips, resident_per_sm * sms, RS, fill_rows<RS>());
  const dim3 grd(strips, (P.ny + len - 1) / len);
  k_step_sweep<TX, RS, NH, FORM, PER, NT, MINB><<<grd, NT, smem, st>>>(P, B, len);
  return cudaGetLastError();
}

// Walls and periodic y are separate instantiations: the wall checks of every
// stage vanish from the periodic kernel and vice versa.
template <int TX, int RS, int NH, int FORM, int NT, int MINB>
cudaError_t launch_sweep_t(const DevParams &P, const FusedBuffers &B, cudaStream_t st) {
  return P.periodic_y ? launch_sweep_per<TX, RS, NH, FORM, 1, NT, MINB>(P, B, st)
                      : launch_sweep_per<TX, RS, NH, FORM, 0, NT, MINB>(P, B, st);
}

}  // namespace

// Launch configurations of the row sweep: strip width x rows per pipeline
// step / threads / minimum resident CTAs per SM.
int sweep_variant_count(const DevParams &P) { return P.nh == 1 ? 13 : 4; }

int sweep_default_variant(const DevParams &P) { return P.nh == 1 ? 9 : 0; }

const char *sweep_variant_name(const DevParams &P, int v) {
  static const char *n1[13] = {"64x2/160/3", "32x4/160/3", "128x1/160/2", "64x4/288/2", "64x1/96/5",
                               "32x8/320/2", "62x2/160/3", "126x1/160/2", "30x4/160/3", "60x2/160/3",
                               "28x4/160/3", "58x2/128/3", "58x2/128/4"};
  static const char *n2[4] = {"64x2/160/2", "32x4/160/2", "64x1/96/4", "62x2/160/2"};
  if (v < 0 || v >= sweep_variant_count(P)) v = 0;
  return P.nh == 1 ? n1[v] : n2[v];
}

template <int NH, int FORM>
static cudaError_t sweep_dispatch(int v, const DevParams &P, const FusedBuffers &B, cudaStream_t s) {
  if constexpr (NH == 1) {
    switch (v) {
      case 1: return launch_sweep_t<32, 4, NH, FORM, 160, 3>(P, B, s);
      case 2: return launch_sweep_t<128, 1, NH, FORM, 160, 2>(P, B, s);
      case 3: return launch_sweep_t<64, 4, NH, FORM, 288, 2>(P, B, s);
      case 4: return launch_sweep_t<64, 1, NH, FORM, 96, 5>(P, B, s);
      case 5: return launch_sweep_t<32, 8, NH, FORM, 320, 2>(P, B, s);
      // strips whose collision rows are a whole number of warps (RS (TX + 2) = 128)
      case 6: return launch_sweep_t<62, 2, NH, FORM, 160, 3>(P, B, s);
      case 7: return launch_sweep_t<126, 1, NH, FORM, 160, 2>(P, B, s);
      case 8: return launch_sweep_t<30, 4, NH, FORM, 160, 3>(P, B, s);
      // ... and whose field rows are (RS (TX + 4) = 128)
      case 9: return launch_sweep_t<60, 2, NH, FORM, 160, 3>(P, B, s);
      case 10: return launch_sweep_t<28, 4, NH, FORM, 160, 3>(P, B, s);
      // ... and whose order-parameter rows are (RS (TX + 6) = 128): four warps
      case 11: return launch_sweep_t<58, 2, NH, FORM, 128, 3>(P, B, s);
      case 12: return launch_sweep_t<58, 2, NH, FORM, 128, 4>(P, B, s);
      default: return launch_sweep_t<64, 2, NH, FORM, 160, 3>(P, B, s);
    }
  } else {
    switch (v) {
      case 1: return launch_sweep_t<32, 4, NH, FORM, 160, 2>(P, B, s);
      case 2: return launch_sweep_t<64, 1, NH, FORM, 96, 4>(P, B, s);
      case 3: return launch_sweep_t<62, 2, NH, FORM, 160, 2>(P, B, s);
      default: return launch_sweep_t<64, 2, NH, FORM, 160, 2>(P, B, s);
    }
  }
}

// Batched sweeps (work items of the strip width and segment length of the
// configuration; segments of 48 or 96 rows keep thousands of items for an
// ensemble of small lattices).
template <int TX, int RS, int NH, int FORM, int NT, int MINB>
static cudaError_t launch_sweep_batched_t(const BatchCase *cases, const WorkItem *work, int nwork, int parity,
                                          cudaStream_t st) {
  const size_t smem = sizeof(PipeSmem<TX, RS, NH, FORM != 0>);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_batched<TX, RS, NH, FORM, NT, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (nwork <= 0) return cudaSuccess;
  k_sweep_batched<TX, RS, NH, FORM, NT, MINB><<<nwork, NT, smem, st>>>(cases, work, parity);
  return cudaGetLastError();
}

template <int TX, int RS, int NH, int FORM, int NT, int MINB>
static cudaError_t launch_sweep_persistent_t(const BatchCase *cases, const WorkItem *work, int nwork, int parity0,
                                             int nsteps, GridSync *sync, long long spin_limit, cudaStream_t st,
                                             int *grid) {
  auto kern = k_sweep_persistent<TX, RS, NH, FORM, NT, MINB>;
  const size_t smem = sizeof(PipeSmem<TX, RS, NH, FORM != 0>);
  static int resident = 0;
  if (!resident) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    resident = per_sm * sms;
  }
  const int nb = nwork < resident ? nwork : resident;
  if (grid) *grid = nb;
  if (nwork <= 0 || nsteps <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, cases, work, nwork, parity0, nsteps, sync, spin_limit);
}

template <int NH, int FORM>
static cudaError_t sweep_persistent_dispatch(int v, const BatchCase *c, const WorkItem *w, int n, int parity0,
                                             int nsteps, GridSync *sync, long long lim, cudaStream_t s, int *grid) {
  if constexpr (NH == 1) {
    switch (v) {
      case 2:
      case 6:
      case 7:
      case 8: return launch_sweep_persistent_t<60, 2, NH, FORM, 160, 3>(c, w, n, parity0, nsteps, sync, lim, s, grid);
      case 3: return launch_sweep_persistent_t<64, 2, NH, FORM, 160, 3>(c, w, n, parity0, nsteps, sync, lim, s, grid);
      default: return launch_sweep_persistent_t<58, 2, NH, FORM, 128, 3>(c, w, n, parity0, nsteps, sync, lim, s, grid);
    }
  } else {
    if (v == 1) return launch_sweep_persistent_t<62, 2, NH, FORM, 160, 2>(c, w, n, parity0, nsteps, sync, lim, s, grid);
    return launch_sweep_persistent_t<64, 2, NH, FORM, 160, 2>(c, w, n, parity0, nsteps, sync, lim, s, grid);
  }
}

int sweep_batched_count(int nh) { return nh == 1 ? 10 : 2; }

// (strip width, segment rows): short segments give many work items for the
// waves, long ones fewer pipeline fill steps per item
void sweep_batched_shape(int nh, int v, int *tx, int *rows) {
  static const int s1[10][2] = {{58, 48}, {58, 96}, {60, 48}, {64, 48}, {58, 64}, {58, 72}, {60, 64},
                                {60, 128}, {60, 200}, {58, 160}};
  static const int s2[2][2] = {{64, 48}, {62, 48}};
  if (v < 0 || v >= sweep_batched_count(nh)) v = 0;
  *tx = nh == 1 ? s1[v][0] : s2[v][0];
  *rows = nh == 1 ? s1[v][1] : s2[v][1];
}

template <int NH, int FORM>
static cudaError_t sweep_batched_dispatch(int v, const BatchCase *c, const WorkItem *w, int n, int parity,
                                          cudaStream_t s) {
  if constexpr (NH == 1) {
    switch (v) {
      case 2:
      case 6:
      case 7:
      case 8: return launch_sweep_batched_t<60, 2, NH, FORM, 160, 3>(c, w, n, parity, s);
      case 3: return launch_sweep_batched_t<64, 2, NH, FORM, 160, 3>(c, w, n, parity, s);
      default: return launch_sweep_batched_t<58, 2, NH, FORM, 128, 3>(c, w, n, parity, s);
    }
  } else {
    if (v == 1) return launch_sweep_batched_t<62, 2, NH, FORM, 160, 2>(c, w, n, parity, s);
    return launch_sweep_batched_t<64, 2, NH, FORM, 160, 2>(c, w, n, parity, s);
  }
}

cudaError_t launch_sweep_batched(int nh, int form, const BatchCase *cases, const WorkItem *work, int nwork,
                                 int parity, cudaStream_t s, int v) {
  if (v < 0 || v >= sweep_batched_count(nh)) v = 0;
  if (nh == 1) {
    if (form == 2) return sweep_batched_dispatch<1, 2>(v, cases, work, nwork, parity, s);
    if (form == 1) return sweep_batched_dispatch<1, 1>(v, cases, work, nwork, parity, s);
    return sweep_batched_dispatch<1, 0>(v, cases, work, nwork, parity, s);
  }
  if (form == 2) return sweep_batched_dispatch<2, 2>(v, cases, work, nwork, parity, s);
  if (form == 1) return sweep_batched_dispatch<2, 1>(v, cases, work, nwork, parity, s);
  return sweep_batched_dispatch<2, 0>(v, cases, work, nwork, parity, s);
}

cudaError_t launch_sweep_persistent(int nh, int form, const BatchCase *cases, const WorkItem *work, int nwork,
                                    int parity0, int nsteps, GridSync *sync, long long spin_limit, cudaStream_t s,
                                    int v, int *grid) {
  if (v < 0 || v >= sweep_batched_count(nh)) return cudaErrorInvalidValue;
  if (nh == 1) {
    if (form == 2) return sweep_persistent_dispatch<1, 2>(v, cases, work, nwork, parity0, nsteps, sync, spin_limit, s, grid);
    if (form == 1) return sweep_persistent_dispatch<1, 1>(v, cases, work, nwork, parity0, nsteps, sync, spin_limit, s, grid);
    return sweep_persistent_dispatch<1, 0>(v, cases, work, nwork, parity0, nsteps, sync, spin_limit, s, grid);
  }
  if (form == 2) return sweep_persistent_dispatch<2, 2>(v, cases, work, nwork, parity0, nsteps, sync, spin_limit, s, grid);
  if (form == 1) return sweep_persistent_dispatch<2, 1>(v, cases, work, nwork, parity0, nsteps, sync, spin_limit, s, grid);
  return sweep_persistent_dispatch<2, 0>(v, cases, work, nwork, parity0, nsteps, sync, spin_limit, s, grid);
}

cudaError_t launch_sweep_step(const DevParams &P, const FusedBuffers &B, cudaStream_t s, int v) {
  if (v < 0 || v >= sweep_variant_count(P)) v = 0;
  const int form = P.g16 ? 2 : (P.collapse_h ? 1 : 0);
  if (P.nh == 1) {
    if (form == 2) return sweep_dispatch<1, 2>(v, P, B, s);
    if (form == 1) return sweep_dispatch<1, 1>(v, P, B, s);
    return sweep_dispatch<1, 0>(v, P, B, s);
  }
  if (form == 2) return sweep_dispatch<2, 2>(v, P, B, s);
  if (form == 1) return sweep_dispatch<2, 1>(v, P, B, s);
  return sweep_dispatch<2, 0>(v, P, B, s);
}

}  // namespace lbm
