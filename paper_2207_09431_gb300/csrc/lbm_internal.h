// Internal: the handle behind lbm_handle and its helpers (shared by the C-ABI
// translation units; not part of the public interface).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_kernels.h"

namespace lbm {
// C_i of the population form into the C planes (Eq. 22).
void launch_moments(const DevParams &P, const float *h, float *C, cudaStream_t s);
// FP64 observable sums (masses, thresholded masses, sum C_g, C_g-weighted
// position and velocity, extents of C_g > 0.5) from the C planes and the FP32
// populations g, with u computed per node as the macro-field kernel computes
// it; acc (11 doubles) and ext (4 ints: xmin, -xmax, ymin, -ymax) are
// accumulated with atomics.
void launch_observables_direct(const DevParams &P, const float *C, const float *g, int gas_comp, double *acc,
                               int *ext, cudaStream_t s);
// Rows [y0, y1) of nplanes dense FP64 planes into pitched FP32 planes.
cudaError_t launch_planes_from_f64_rows(const DevParams &P, const double *src, float *dst, int nplanes, int y0,
                                        int y1, cudaStream_t s);
// Initial equilibria (modified, Eq. 14 and 18 at rest of the forcing) of rows
// [y0, y1); they read C and p up to two rows beyond.
void launch_init_rows(const DevParams &P, const StepBuffers &B, int y0, int y1, cudaStream_t s);
}  // namespace lbm

namespace lbm_detail {

constexpr int kVersion = 100;  // 0.1.0
constexpr size_t kAlign = 256;
// checkpoint magic; the last character names the population layout (2: planes
// interleaved in blocks of 32 columns)
inline constexpr char kMagic[8] = {'L', 'B', 'M', 'G', 'B', '3', '0', '2'};

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

inline int pitch_of(int nx) { return (nx + 31) / 32 * 32; }

// Number of FP32 planes the handle carves from the arena.
struct Layout {
  size_t plane_bytes;
  size_t g, h, tau, C, mu, p, ux, uy, shear, SV, small, total;
};

inline Layout layout_of(const lbm_params &p) {
  Layout L{};
  const int nh = p.ncomp - 1;
  L.plane_bytes = align_up((size_t)p.ny * pitch_of(p.nx) * sizeof(float), kAlign);
  size_t off = 0;
  auto take = [&](size_t planes) {
    size_t o = off;
    off += planes * L.plane_bytes;
    return o;
  };
  L.g = take(2 * 9);
  L.h = take(p.collapse_h ? 2 * (size_t)nh : 2 * 9 * (size_t)nh);
  L.tau = take(2);
  L.C = take(nh);
  L.mu = take(3);
  L.p = take(1);
  L.ux = take(1);
  L.uy = take(1);
  L.shear = take(1);
  L.SV = take(nh);
  L.small = off;
  off += align_up(16 * sizeof(double) + 8 * sizeof(int) + sizeof(unsigned), kAlign);
  L.total = off;
  return L;
}

inline const char *validate(const lbm_params *p) {
  if (!p) return "params is NULL";
  if (p->nx < 1 || p->ny < 3) return "need nx >= 1 and ny >= 3";
  if ((long long)p->nx * p->ny > (1LL << 31)) return "lattice too large";
  if (p->ncomp != 2 && p->ncomp != 3) return "ncomp must be 2 or 3";
  if (p->fd_scheme != 0 && p->fd_scheme != 1) return "fd_scheme must be 0 or 1";
  if (p->storage != 0 && p->storage != 1) return "storage must be 0 (FP32) or 1 (FP16 g)";
  if (p->storage == 1 && !p->collapse_h) return "FP16 storage needs collapse_h 1";
  if (p->open_x != 0 && p->open_x != 1) return "open_x must be 0 or 1";
  if (p->open_x && (p->nx < 4 || p->collapse_h || p->storage)) return "open x needs nx >= 4 and the population state";
  if (p->mobility != 0 && p->mobility != 1) return "mobility must be 0 or 1";
  if (p->gas_comp != 2 && p->gas_comp != 3) return "gas_comp must be 2 or 3";
  if (p->ncomp == 2 && p->gas_comp != 3) return "with two components the gas is component 3";
  if (p->collapse_h != 0 && p->collapse_h != 1) return "collapse_h must be 0 or 1";
  if (p->collapse_h && p->fd_scheme != 0) return "the collapsed state form needs fd_scheme 0";
  for (int i = 0; i < 3; ++i)
    if (!(p->rho[i] > 0) || !(p->tau[i] > 0)) return "densities and relaxation times must be positive";
  const double S1 = p->sigma12 + p->sigma13 - p->sigma23;
  const double S2 = p->sigma12 + p->sigma23 - p->sigma13;
  const double S3 = p->sigma13 + p->sigma23 - p->sigma12;
  if (!(S1 > 0 && S2 > 0 && S3 > 0)) return "capillary coefficients Sigma_i must be positive";
  if (!(p->xi > 0)) return "interface width xi must be positive";
  if (!(p->D0 >= 0)) return "D0 must be non-negative";
  if (p->powerlaw && !(p->pl_k > 0 && p->pl_n > 0)) return "power law needs k > 0 and n > 0";
  if (!(p->tau_min > 0 && p->tau_min <= p->tau_max)) return "need 0 < tau_min <= tau_max";
  return nullptr;
}

inline lbm::DevParams dev_params(const lbm_params &p) {
  lbm::DevParams d{};
  d.nx = p.nx;
  d.ny = p.ny;
  d.pitch = pitch_of(p.nx);
  d.ncomp = p.ncomp;
  d.nh = p.ncomp - 1;
  d.periodic_y = p.periodic_y ? 1 : 0;
  d.powerlaw = p.powerlaw ? 1 : 0;
  d.mobility = p.mobility;
  d.fd_scheme = p.fd_scheme;
  d.collapse_h = p.collapse_h;
  d.g16 = p.storage == 1 ? 1 : 0;
  d.open_x = p.open_x;
  d.u_in = (float)p.u_in;
  d.c_in[0] = (float)p.c_in[0];
  d.c_in[1] = (float)p.c_in[1];
  {
    // power-of-two scale: deviations of size rho_max stay far below the FP16
    // maximum (65504 / 2^14 = 4 rho_max) while those of size 1e-8 rho_max are
    // still normal numbers (smallest normal 6.1e-5 / 2^14 = 3.7e-9 rho_max)
    const double rmax = std::fmax(p.rho[0], std::fmax(p.rho[1], p.rho[2]));
    const int e = 14 - (int)std::ceil(std::log2(rmax));
    d.g16_scale = (float)std::ldexp(1.0, e);
    d.g16_inv_scale = (float)std::ldexp(1.0, -e);
  }
  for (int i = 0; i < 3; ++i) {
    d.rho[i] = (float)p.rho[i];
    d.tau[i] = (float)p.tau[i];
  }
  d.pl_n = (float)p.pl_n;
  d.pl_k = (float)p.pl_k;
  d.tau_min = (float)p.tau_min;
  d.tau_max = (float)p.tau_max;
  d.sig12 = (float)p.sigma12;
  d.sig13 = (float)p.sigma13;
  d.sig23 = (float)p.sigma23;
  d.Lambda = (float)p.Lambda;
  // capillary coefficients and Sigma_T (Sec. 2.1), in double then rounded
  const double S1 = p.sigma12 + p.sigma13 - p.sigma23;
  const double S2 = p.sigma12 + p.sigma23 - p.sigma13;
  const double S3 = p.sigma13 + p.sigma23 - p.sigma12;
  d.Sig[0] = (float)S1;
  d.Sig[1] = (float)S2;
  d.Sig[2] = (float)S3;
  d.SigT = (float)(3.0 / (1.0 / S1 + 1.0 / S2 + 1.0 / S3));
  d.xi = (float)p.xi;
  d.D0 = (float)p.D0;
  const double Sg[3] = {S1, S2, S3};
  for (int i = 0; i < 3; ++i) {
    d.inv_sig[i] = (float)(1.0 / Sg[i]);
    d.grad_coef[i] = (float)(0.75 * p.xi * Sg[i]);
    d.d0_sig[i] = (float)(p.D0 / Sg[i]);
  }
  d.mu_pre = (float)(4.0 * (3.0 / (1.0 / S1 + 1.0 / S2 + 1.0 / S3)) / p.xi);
  d.n1 = (float)(p.pl_n - 1.0);
  d.n1h = (float)(0.5 * (p.pl_n - 1.0));
  d.k3 = (float)(3.0 * p.pl_k);
  d.gravity = (float)p.gravity;
  d.force_x = (float)p.force_x;
  d.plane = (long long)p.ny * d.pitch;
  return d;
}

// SplitMix64 (Steele, Lea and Flood 2014) at counter i: mix(seed + (i+1) gamma).
inline uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace lbm_detail

using namespace lbm_detail;

struct lbm_handle {
  lbm_params prm;
  lbm::DevParams dp;
  Layout L;
  cudaStream_t stream;
  char *arena;
  float *g[2], *h[2], *tau[2];
  float *C, *mu, *p, *ux, *uy, *shear, *SV;
  double *acc;
  int *ext;
  unsigned *err;
  int cur;
  int variant;            // fused-step launch configuration (autotuned or the default)
  std::string kname;      // name reported by lbm_kernel_name
  bool initialized;
  long long step;
  bool have_prev;
  long long prev_step;
  double prev_v, y_int;
  std::string last_error;
  std::vector<float> stage;  // host staging (pitched FP32 planes)
  // captured runs of kStepGraph steps without diagnostics, one per starting
  // buffer (cur), for the launch configuration they were captured with
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_variant[2] = {-1, -1};
  static constexpr int kStepGraph = 16;
  // lbm_set_fields: a stream of its own for the upload of C in row chunks,
  // overlapped with the conversion and initial equilibria on `stream`
  static constexpr int kUploadChunks = 4;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t upload_ev[kUploadChunks + 1] = {};

  ~lbm_handle() {
    for (auto &g : graph)
      if (g) cudaGraphExecDestroy(g);
    for (auto &e : upload_ev)
      if (e) cudaEventDestroy(e);
    if (copy_stream) cudaStreamDestroy(copy_stream);
  }

  lbm_status fail(lbm_status s, const std::string &msg) {
    last_error = msg;
    return s;
  }
  lbm_status cuda_fail(cudaError_t e, const char *where) {
    last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return LBM_E_CUDA;
  }
  bool fused() const { return lbm::fused_supported(dp); }
  lbm::FusedBuffers fused_buffers(int in, bool diag) const {
    lbm::FusedBuffers B{};
    B.g_in = g[in];
    B.h_in = h[in];
    B.tau_in = tau[in];
    B.g_out = g[1 - in];
    B.h_out = h[1 - in];
    B.tau_out = tau[1 - in];
    B.shear = diag ? shear : nullptr;
    B.SV = diag ? SV : nullptr;
    B.err = err;
    return B;
  }
  // One time step from buffer `cur` into the other one.
  void launch_step(bool diag, cudaEvent_t *ev) {
    if (fused()) {
      if (ev) cudaEventRecord(ev[0], stream);
      lbm::launch_fused_step(dp, fused_buffers(cur, diag), stream, variant);
      if (ev) cudaEventRecord(ev[1], stream);
    } else {
      lbm::launch_split_step(dp, buffers(cur), stream, ev);
    }
    cur = 1 - cur;
  }
  int kernels_per_step() const { return fused() ? 1 : lbm::kSplitKernels; }
  lbm::StepBuffers buffers(int in) const {
    lbm::StepBuffers B{};
    B.g_in = g[in];
    B.h_in = prm.collapse_h ? nullptr : h[in];
    B.tau_in = tau[in];
    B.g_out = g[1 - in];
    B.h_out = h[1 - in];
    B.tau_out = tau[1 - in];
    B.C = prm.collapse_h ? h[in] : C;
    B.mu = mu;
    B.p = p;
    B.ux = ux;
    B.uy = uy;
    B.shear = shear;
    B.SV = SV;
    B.err = err;
    return B;
  }
  size_t plane_floats() const { return (size_t)dp.plane; }
};

