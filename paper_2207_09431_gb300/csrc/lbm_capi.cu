// Host side of the C ABI declared in include/lbm.h: parameter validation,
// arena carving, initial conditions (Sec. 4.2, Eq. 42), the step loop, field
// readback, observables post-processing (Sec. 4.1-4.2) and checkpoints.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_kernels.h"

#include "lbm_internal.h"

// Copies nplanes host planes (dense ny x nx doubles) into pitched device FP32
// planes: the doubles go to the device as they are, staged in the spare
// population buffer g[1] (free until the initial equilibria are built), and a
// kernel converts them; a NULL source sets the planes to zero.  Enqueued on
// the handle's stream; the caller synchronises.
static cudaError_t upload_planes(lbm_handle *h, float *dst, const double *src, int nplanes) {
  const size_t plane_bytes = h->L.plane_bytes;
  if (!src) return cudaMemsetAsync(dst, 0, (size_t)nplanes * plane_bytes, h->stream);
  const size_t bytes = (size_t)nplanes * h->prm.nx * h->prm.ny * sizeof(double);
  if (bytes > 9 * plane_bytes) return cudaErrorInvalidValue;  // cannot happen: 2 planes of doubles < 9 of floats
  double *staging = reinterpret_cast<double *>(h->g[1]);
  cudaError_t e = cudaMemcpyAsync(staging, src, bytes, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = lbm::launch_planes_from_f64(h->dp, staging, dst, nplanes, h->stream);
  return e;
}

// Copies nplanes pitched device planes into dense host doubles.
static cudaError_t download_planes(lbm_handle *h, const float *src, double *dst, int nplanes) {
  const int nx = h->prm.nx, ny = h->prm.ny, pitch = h->dp.pitch;
  h->stage.assign((size_t)nplanes * h->plane_floats(), 0.0f);
  for (int q = 0; q < nplanes; ++q) {
    cudaError_t e = cudaMemcpyAsync(h->stage.data() + (size_t)q * h->plane_floats(),
                                    src + (size_t)q * (h->L.plane_bytes / sizeof(float)),
                                    h->plane_floats() * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  for (int q = 0; q < nplanes; ++q)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        dst[((size_t)q * ny + y) * nx + x] = h->stage[(size_t)q * h->plane_floats() + (size_t)y * pitch + x];
  return cudaSuccess;
}

// Copies a device population array (nq planes interleaved in blocks of 32
// columns, lbm::pop_index) into dense host doubles, plane after plane.
static cudaError_t download_pops(lbm_handle *h, const float *src, double *dst, int nq) {
  const int nx = h->prm.nx, ny = h->prm.ny, pitch = h->dp.pitch;
  const size_t n = (size_t)nq * ny * pitch;
  h->stage.assign(n, 0.0f);
  cudaError_t e = cudaMemcpyAsync(h->stage.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return e;
  for (int q = 0; q < nq; ++q)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        dst[((size_t)q * ny + y) * nx + x] = h->stage[lbm::pop_index((long long)y * pitch + x, q, nq)];
  return cudaSuccess;
}

extern "C" {

int lbm_version(void) { return kVersion; }

size_t lbm_required_bytes(const lbm_params *p) {
  if (validate(p)) return 0;
  return layout_of(*p).total;
}

lbm_status lbm_create(const lbm_params *p, void *dev_arena, size_t arena_bytes, void *cuda_stream,
                      lbm_handle **out) {
  if (!out) return LBM_E_INVAL;
  *out = nullptr;
  if (validate(p)) return LBM_E_INVAL;
  if (!dev_arena || ((uintptr_t)dev_arena % kAlign) != 0) return LBM_E_INVAL;
  Layout L = layout_of(*p);
  if (arena_bytes < L.total) return LBM_E_NOMEM;
  lbm_handle *h = new (std::nothrow) lbm_handle();
  if (!h) return LBM_E_NOMEM;
  h->prm = *p;
  h->dp = dev_params(*p);
  h->L = L;
  h->stream = (cudaStream_t)cuda_stream;
  h->arena = (char *)dev_arena;
  const size_t pf = L.plane_bytes / sizeof(float);
  const int nh = p->ncomp - 1;
  for (int b = 0; b < 2; ++b) {
    h->g[b] = (float *)(h->arena + L.g) + (size_t)b * 9 * pf;
    h->h[b] = (float *)(h->arena + L.h) + (size_t)b * (p->collapse_h ? 1 : 9) * nh * pf;
    h->tau[b] = (float *)(h->arena + L.tau) + (size_t)b * pf;
  }
  h->C = (float *)(h->arena + L.C);
  h->mu = (float *)(h->arena + L.mu);
  h->p = (float *)(h->arena + L.p);
  h->ux = (float *)(h->arena + L.ux);
  h->uy = (float *)(h->arena + L.uy);
  h->shear = (float *)(h->arena + L.shear);
  h->SV = (float *)(h->arena + L.SV);
  h->acc = (double *)(h->arena + L.small);
  h->ext = (int *)(h->acc + 16);
  h->err = (unsigned *)(h->ext + 8);
  // plane stride used by the kernels must match the arena planes
  h->dp.plane = (long long)pf;
  h->cur = 0;
  h->variant = h->fused() ? lbm::sweep_default_variant(h->dp) : 0;
  h->initialized = false;
  h->step = 0;
  h->have_prev = false;
  cudaError_t e = cudaMemsetAsync(h->arena, 0, L.total, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    delete h;
    return LBM_E_CUDA;
  }
  *out = h;
  return LBM_OK;
}

// Whether lbm_set_fields may overlap the upload of C with the conversion and
// the initial equilibria: FP32 populations (the FP16 form computes its
// equilibria into the staging buffer), chunks of at least 16 rows (the
// equilibria read two rows beyond their own), and a stream that is not being
// captured.  The copy stream and its events are created on first use.
static bool upload_overlappable(lbm_handle *h) {
  if (h->dp.g16 || h->prm.ny < 16 * lbm_handle::kUploadChunks) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
  if (!h->copy_stream && cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
    h->copy_stream = nullptr;
    return false;
  }
  for (auto &ev : h->upload_ev)
    if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      ev = nullptr;
      return false;
    }
  return true;
}

// C goes up in row chunks on the copy stream; the handle's stream converts each
// chunk once it has arrived and computes the equilibria of the rows whose
// two-row neighbourhood is converted (those of the first chunk last under
// periodic y, where they read the last rows).  Same node values as one upload.
static cudaError_t upload_and_init_overlapped(lbm_handle *h, const double *C, int nh, const lbm::StepBuffers &B) {
  constexpr int n = lbm_handle::kUploadChunks;
  const int nx = h->prm.nx, ny = h->prm.ny, rows = (ny + n - 1) / n;
  const bool per = h->prm.periodic_y != 0;
  double *staging = reinterpret_cast<double *>(h->g[1]);
  // the staging buffer is free once the uploads before on the stream are done
  cudaError_t e = cudaEventRecord(h->upload_ev[n], h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, h->upload_ev[n], 0);
  for (int c = 0; c < n && e == cudaSuccess; ++c) {
    const int y0 = c * rows, y1 = std::min(ny, y0 + rows);
    for (int q = 0; q < nh && e == cudaSuccess; ++q) {
      const size_t off = ((size_t)q * ny + y0) * nx;
      e = cudaMemcpyAsync(staging + off, C + off, (size_t)(y1 - y0) * nx * sizeof(double), cudaMemcpyHostToDevice,
                          h->copy_stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->upload_ev[c], h->copy_stream);
  }
  for (int c = 0; c < n && e == cudaSuccess; ++c) {
    const int y0 = c * rows, y1 = std::min(ny, y0 + rows);
    e = cudaStreamWaitEvent(h->stream, h->upload_ev[c], 0);
    if (e == cudaSuccess) e = lbm::launch_planes_from_f64_rows(h->dp, staging, h->C, nh, y0, y1, h->stream);
    if (e == cudaSuccess && c >= 1 && (c >= 2 || !per)) {
      lbm::launch_init_rows(h->dp, B, (c - 1) * rows, c * rows, h->stream);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) {
    lbm::launch_init_rows(h->dp, B, (n - 1) * rows, ny, h->stream);
    if (per) lbm::launch_init_rows(h->dp, B, 0, rows, h->stream);
    e = cudaGetLastError();
  }
  return e;
}

lbm_status lbm_set_fields(lbm_handle *h, const double *C, const double *p, const double *ux, const double *uy) {
  if (!h) return LBM_E_INVAL;
  if (!C) return h->fail(LBM_E_INVAL, "C is NULL");
  const int nh = h->prm.ncomp - 1;
  const bool overlap = upload_overlappable(h);
  cudaError_t e = overlap ? cudaSuccess : upload_planes(h, h->C, C, nh);
  if (e == cudaSuccess) e = upload_planes(h, h->p, p, 1);
  if (e == cudaSuccess) e = upload_planes(h, h->ux, ux, 1);
  if (e == cudaSuccess) e = upload_planes(h, h->uy, uy, 1);
  if (e != cudaSuccess) return h->cuda_fail(e, "lbm_set_fields upload");
  // equilibria into buffer 0
  lbm::StepBuffers B = h->buffers(1);  // *_out of buffer index 1 is buffer 0
  if (h->dp.g16) B.g_out = h->g[1];    // FP32 equilibria into the spare, encoded below
  if (h->prm.collapse_h) {
    B.C = h->C;
    B.h_out = nullptr;
  }
  if (overlap) {
    e = upload_and_init_overlapped(h, C, nh, B);
  } else {
    lbm::launch_init(h->dp, B, h->stream);
    e = cudaGetLastError();
  }
  // the C state: the converted order parameters
  if (e == cudaSuccess && h->prm.collapse_h)
    e = cudaMemcpyAsync(h->h[0], h->C, (size_t)nh * h->L.plane_bytes, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess && h->dp.g16) e = lbm::launch_g16_encode(h->dp, h->g[1], h->g[0], h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "lbm_set_fields init kernel");
  h->cur = 0;
  h->initialized = true;
  h->step = 0;
  h->have_prev = false;
  h->last_error.clear();
  return LBM_OK;
}

lbm_status lbm_init_bubbles(lbm_handle *h, const lbm_bubble *bubbles, int nb, unsigned long long seed,
                            double noise_amp) {
  if (!h) return LBM_E_INVAL;
  if (nb < 0 || (nb > 0 && !bubbles)) return h->fail(LBM_E_INVAL, "bad bubble list");
  const int nx = h->prm.nx, ny = h->prm.ny, nh = h->prm.ncomp - 1;
  const size_t n = (size_t)nx * ny;
  std::vector<double> comp[2] = {std::vector<double>(n, 0.0), std::vector<double>(n, 0.0)};  // comps 2, 3
  bool used[2] = {false, false};
  for (int b = 0; b < nb; ++b) {
    const int c = bubbles[b].comp;
    if (c < 2 || c > 3 || (nh == 1 && c != 3)) return h->fail(LBM_E_INVAL, "disc component must be 3 (or 2 with ncomp 3)");
    used[c - 2] = true;
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        double dx = std::fabs(x - bubbles[b].cx), dy = std::fabs(y - bubbles[b].cy);
        if (dx > 0.5 * nx) dx = nx - dx;
        if (h->prm.periodic_y && dy > 0.5 * ny) dy = ny - dy;
        const double r = std::sqrt(dx * dx + dy * dy);
        comp[c - 2][(size_t)y * nx + x] += 0.5 - 0.5 * std::tanh((r - bubbles[b].r) / (0.5 * h->prm.xi));
      }
  }
  for (int c = 0; c < 2; ++c) {
    if (!used[c] || noise_amp == 0.0) continue;
    for (size_t k = 0; k < n; ++k) {
      const uint64_t z = splitmix64_at(seed, (uint64_t)(c + 1) * n + k);
      const double u01 = (double)(z >> 11) * (1.0 / 9007199254740992.0);
      comp[c][k] += noise_amp * (2.0 * u01 - 1.0);
    }
  }
  std::vector<double> Cin((size_t)nh * n);
  for (size_t k = 0; k < n; ++k) {
    Cin[k] = 1.0 - comp[0][k] - comp[1][k];
    if (nh == 2) Cin[n + k] = comp[0][k];
  }
  return lbm_set_fields(h, Cin.data(), nullptr, nullptr, nullptr);
}

lbm_status lbm_step(lbm_handle *h, long long nsteps) {
  if (!h) return LBM_E_INVAL;
  if (!h->initialized) return h->fail(LBM_E_STATE, "lbm_step before initial fields");
  if (nsteps < 0) return h->fail(LBM_E_INVAL, "nsteps < 0");
  cudaError_t e = cudaMemsetAsync(h->err, 0, sizeof(unsigned), h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "lbm_step memset");
  long long t = 0;
  // Runs of kStepGraph steps are replayed from a captured graph (on a created
  // stream; capture needs one).  The last step writes the diagnostics and is
  // launched directly; a first run with a new configuration is too, so that
  // its kernels are configured outside the capture.
  const bool capturable = h->stream != nullptr && h->stream != cudaStreamLegacy && h->stream != cudaStreamPerThread;
  const int K = lbm_handle::kStepGraph;
  if (capturable && nsteps - 1 >= K) {
    if (!h->graph[h->cur] || h->graph_variant[h->cur] != h->variant) {
      h->launch_step(false, nullptr);
      t = 1;
      const int c = h->cur;
      if (h->graph[c]) cudaGraphExecDestroy(h->graph[c]);
      h->graph[c] = nullptr;
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
      for (int k = 0; k < K && e == cudaSuccess; ++k) {
        h->launch_step(false, nullptr);
        e = cudaGetLastError();
      }
      cudaError_t ec = cudaStreamEndCapture(h->stream, &g);
      if (e == cudaSuccess) e = ec;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph[c], g, 0);
      if (g) cudaGraphDestroy(g);
      h->cur = c;  // an even number of captured steps returns to the same buffer
      if (e != cudaSuccess) {
        h->graph[c] = nullptr;
        return h->cuda_fail(e, "lbm_step graph capture");
      }
      h->graph_variant[c] = h->variant;
    }
    for (; nsteps - 1 - t >= K && e == cudaSuccess; t += K) e = cudaGraphLaunch(h->graph[h->cur], h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "lbm_step graph launch");
  }
  for (; t < nsteps; ++t) h->launch_step(t == nsteps - 1, nullptr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return h->cuda_fail(e, "lbm_step launch");
  unsigned flag = 0;
  e = cudaMemcpyAsync(&flag, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "lbm_step");
  h->step += nsteps;
  if (flag) return h->fail(LBM_E_DIVERGED, "non-finite rho, p, u or tau during lbm_step");
  return LBM_OK;
}

// FP32 populations of the current state: the state itself, or (FP16 storage)
// their decoded copy in the spare buffer.
static const float *fp32_populations(lbm_handle *h, cudaError_t *e) {
  if (!h->dp.g16) return h->g[h->cur];
  *e = lbm::launch_g16_decode(h->dp, h->g[h->cur], h->g[1 - h->cur], h->stream);
  return h->g[1 - h->cur];
}

static lbm_status compute_macros(lbm_handle *h) {
  lbm::StepBuffers B = h->buffers(h->cur);
  cudaError_t e = cudaSuccess;
  B.g_in = fp32_populations(h, &e);
  if (e != cudaSuccess) return h->cuda_fail(e, "FP16 decode");
  lbm::launch_macros(h->dp, B, h->stream);
  e = cudaGetLastError();
  if (e != cudaSuccess) return h->cuda_fail(e, "macro kernels");
  return LBM_OK;
}

lbm_status lbm_postprocess(const lbm_params *p, const double raw[15], lbm_obs *o) {
  if (!p || !raw || !o) return LBM_E_INVAL;
  std::memset(o, 0, sizeof(*o));
  for (int i = 0; i < 15; ++i) o->raw[i] = raw[i];
  for (int i = 0; i < 3; ++i) {
    o->mass[i] = raw[i];
    o->mass_thr[i] = raw[3 + i];
  }
  const int gc = (p->gas_comp == 2 || p->gas_comp == 3) ? p->gas_comp : 3;
  const double rho_l = p->rho[0], rho_g = p->rho[gc - 1];
  const double sigma = gc == 3 ? p->sigma13 : p->sigma12;
  const double g = p->gravity;
  const double n = p->powerlaw ? p->pl_n : 1.0;
  const double k = p->powerlaw ? p->pl_k : rho_l * p->tau[0] / 3.0;
  const double A = raw[6];
  const double nan = std::nan("");
  o->area = A;
  if (A > 0) {
    o->centroid[0] = raw[7] / A;  // Eq. 44
    o->centroid[1] = raw[8] / A;
    o->velocity[0] = raw[9] / A;  // Eq. 43
    o->velocity[1] = raw[10] / A;
  } else {
    o->centroid[0] = o->centroid[1] = o->velocity[0] = o->velocity[1] = nan;
  }
  const double U = o->velocity[1];
  o->rise_velocity = U;
  const double d = A > 0 ? 2.0 * std::sqrt(A / M_PI) : nan;  // area-equivalent diameter
  o->d_eq = d;
  o->aspect_E = raw[11] >= 0 ? (raw[14] - raw[13] + 1.0) / (raw[12] - raw[11] + 1.0) : nan;
  o->drag_coefficient = (A > 0 && U != 0 && g != 0) ? 4.0 * d * g * (rho_l - rho_g) / (3.0 * rho_l * U * U) : nan;
  o->Re = A > 0 ? rho_l * std::pow(std::fabs(U), 2.0 - n) * std::pow(d, n) / k : nan;  // Eq. 38
  o->Eo = A > 0 ? (rho_l - rho_g) * g * d * d / sigma : nan;                             // Eq. 40
  o->Mo = (A > 0 && U != 0)
              ? g * (rho_l - rho_g) / (rho_l * rho_l * sigma * sigma * sigma) *
                    std::pow(k * std::pow(std::fabs(U) / d, n - 1.0), 4.0)
              : nan;  // Eq. 39
  return LBM_OK;
}

lbm_status lbm_observables(lbm_handle *h, lbm_obs *out) {
  if (!h || !out) return LBM_E_INVAL;
  if (!h->initialized) return h->fail(LBM_E_STATE, "observables before initial fields");
  // C planes (the state itself in the C forms), FP32 populations, then the
  // sums with u computed per node; no macro-field planes are written
  lbm::StepBuffers B = h->buffers(h->cur);
  cudaError_t e = cudaSuccess;
  const float *g = fp32_populations(h, &e);
  if (e != cudaSuccess) return h->cuda_fail(e, "FP16 decode");
  if (B.h_in) lbm::launch_moments(h->dp, B.h_in, B.C, h->stream);
  e = cudaMemsetAsync(h->acc, 0, 16 * sizeof(double), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ext, 0x7f, 8 * sizeof(int), h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "observables memset");
  lbm::launch_observables_direct(h->dp, B.C, g, h->prm.gas_comp, h->acc, h->ext, h->stream);
  double acc[16];
  int ext[8];
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(acc, h->acc, sizeof(acc), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ext, h->ext, sizeof(ext), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "observables");
  double raw[15];
  for (int i = 0; i < 11; ++i) raw[i] = acc[i];
  const bool any = ext[0] != 0x7f7f7f7f;
  raw[11] = any ? ext[0] : -1.0;
  raw[12] = any ? -ext[1] : -1.0;
  raw[13] = any ? ext[2] : -1.0;
  raw[14] = any ? -ext[3] : -1.0;
  lbm_postprocess(&h->prm, raw, out);
  out->step = h->step;
  // centroid y at the first call plus the trapezoidal integral of the rise velocity
  if (!h->have_prev) {
    h->y_int = out->centroid[1];
    h->have_prev = true;
  } else {
    h->y_int += 0.5 * (h->prev_v + out->rise_velocity) * (double)(h->step - h->prev_step);
  }
  h->prev_step = h->step;
  h->prev_v = out->rise_velocity;
  out->y_integrated = h->y_int;
  return LBM_OK;
}

lbm_status lbm_get_field(lbm_handle *h, int id, double *out, size_t n) {
  if (!h || !out) return LBM_E_INVAL;
  if (!h->initialized) return h->fail(LBM_E_STATE, "get_field before initial fields");
  const int nh = h->prm.ncomp - 1;
  const size_t N = (size_t)h->prm.nx * h->prm.ny;
  size_t need;
  switch (id) {
    case LBM_FIELD_G: need = 9 * N; break;
    case LBM_FIELD_H: need = (size_t)9 * nh * N; break;
    case LBM_FIELD_SV: need = (size_t)nh * N; break;
    case LBM_FIELD_C1: case LBM_FIELD_C2: case LBM_FIELD_C3: case LBM_FIELD_RHO: case LBM_FIELD_P:
    case LBM_FIELD_UX: case LBM_FIELD_UY: case LBM_FIELD_TAU: case LBM_FIELD_MU1: case LBM_FIELD_MU2:
    case LBM_FIELD_MU3: case LBM_FIELD_SHEAR: need = N; break;
    default: return h->fail(LBM_E_INVAL, "unknown field id");
  }
  if (n < need) return h->fail(LBM_E_INVAL, "output buffer too small");
  const size_t pf = h->L.plane_bytes / sizeof(float);
  cudaError_t e = cudaSuccess;
  switch (id) {
    case LBM_FIELD_G: {
      const float *g32 = fp32_populations(h, &e);
      if (e == cudaSuccess) e = download_pops(h, g32, out, 9);
      break;
    }
    case LBM_FIELD_H:
      if (h->prm.collapse_h) return h->fail(LBM_E_STATE, "the collapsed state form stores no h populations");
      e = download_pops(h, h->h[h->cur], out, 9 * nh);
      break;
    case LBM_FIELD_TAU: e = download_planes(h, h->tau[h->cur], out, 1); break;
    case LBM_FIELD_SHEAR: e = download_planes(h, h->shear, out, 1); break;
    case LBM_FIELD_SV: e = download_planes(h, h->SV, out, nh); break;
    default: {
      lbm_status st = compute_macros(h);
      if (st != LBM_OK) return st;
      const float *Cp = h->buffers(h->cur).C;
      if (id == LBM_FIELD_C1) e = download_planes(h, Cp, out, 1);
      else if (id == LBM_FIELD_C2) {
        if (nh == 2) e = download_planes(h, Cp + pf, out, 1);
        else std::memset(out, 0, N * sizeof(double));
      } else if (id == LBM_FIELD_C3 || id == LBM_FIELD_RHO) {
        std::vector<double> c(2 * N, 0.0);
        e = download_planes(h, Cp, c.data(), nh);
        if (e == cudaSuccess)
          for (size_t k = 0; k < N; ++k) {
            // C3 = 1 - C1 - C2 (Eq. 1); rho by the clipped mixture law (R1)
            const double C1 = (float)c[k], C2 = nh == 2 ? (float)c[N + k] : 0.0;
            const double C3 = (double)(1.0f - (float)C1 - (float)C2);
            if (id == LBM_FIELD_C3) {
              out[k] = C3;
            } else {
              double w[3] = {C1, C2, C3}, s = 0;
              for (double &v : w) { v = v < 0 ? 0 : (v > 1 ? 1 : v); s += v; }
              out[k] = (w[0] * h->prm.rho[0] + w[1] * h->prm.rho[1] + w[2] * h->prm.rho[2]) / s;
            }
          }
      } else if (id == LBM_FIELD_P) e = download_planes(h, h->p, out, 1);
      else if (id == LBM_FIELD_UX) e = download_planes(h, h->ux, out, 1);
      else if (id == LBM_FIELD_UY) e = download_planes(h, h->uy, out, 1);
      else e = download_planes(h, h->mu + (size_t)(id - LBM_FIELD_MU1) * pf, out, 1);
    }
  }
  if (e != cudaSuccess) return h->cuda_fail(e, "lbm_get_field");
  return LBM_OK;
}

lbm_status lbm_save(lbm_handle *h, const char *path) {
  if (!h || !path) return LBM_E_INVAL;
  if (!h->initialized) return h->fail(LBM_E_STATE, "save before initial fields");
  const int nh = h->prm.ncomp - 1;
  const size_t pf = h->L.plane_bytes / sizeof(float);
  const int hp = (h->prm.collapse_h ? 1 : 9) * nh;
  const int nplanes = 9 + hp + 1;
  std::vector<float> buf((size_t)nplanes * pf);
  cudaError_t e = cudaMemcpyAsync(buf.data(), h->g[h->cur], 9 * pf * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(buf.data() + 9 * pf, h->h[h->cur], hp * pf * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(buf.data() + (size_t)(9 + hp) * pf, h->tau[h->cur], pf * sizeof(float),
                        cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "lbm_save");
  FILE *f = std::fopen(path, "wb");
  if (!f) return h->fail(LBM_E_IO, std::string("cannot open ") + path);
  long long hdr[2] = {h->step, (long long)buf.size()};
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&h->prm, sizeof(lbm_params), 1, f) == 1 &&
            std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
            std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return h->fail(LBM_E_IO, "short write");
  return LBM_OK;
}

lbm_status lbm_load(lbm_handle *h, const char *path) {
  if (!h || !path) return LBM_E_INVAL;
  FILE *f = std::fopen(path, "rb");
  if (!f) return h->fail(LBM_E_IO, std::string("cannot open ") + path);
  char magic[8];
  lbm_params prm;
  long long hdr[2];
  const int nh = h->prm.ncomp - 1;
  const size_t pf = h->L.plane_bytes / sizeof(float);
  const int hp = (h->prm.collapse_h ? 1 : 9) * nh;
  const size_t count = (size_t)(9 + hp + 1) * pf;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
            std::fread(&prm, sizeof(prm), 1, f) == 1 && std::fread(hdr, sizeof(hdr), 1, f) == 1;
  if (ok && (std::memcmp(&prm, &h->prm, sizeof(prm)) != 0 || hdr[1] != (long long)count)) {
    std::fclose(f);
    return h->fail(LBM_E_INVAL, "checkpoint parameters differ from the handle's");
  }
  std::vector<float> buf(count);
  ok = ok && std::fread(buf.data(), sizeof(float), count, f) == count;
  std::fclose(f);
  if (!ok) return h->fail(LBM_E_IO, "truncated or foreign checkpoint");
  cudaError_t e = cudaMemcpyAsync(h->g[0], buf.data(), 9 * pf * sizeof(float), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h[0], buf.data() + 9 * pf, hp * pf * sizeof(float), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->tau[0], buf.data() + (size_t)(9 + hp) * pf, pf * sizeof(float),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return h->cuda_fail(e, "lbm_load");
  h->cur = 0;
  h->step = hdr[0];
  h->initialized = true;
  h->have_prev = false;
  return LBM_OK;
}

int lbm_kernels_per_step(const lbm_handle *h) { return h ? h->kernels_per_step() : 0; }

const char *lbm_kernel_name(const lbm_handle *h, int i) {
  static const char *names[lbm::kSplitKernels] = {"k_moments", "k_fields", "k_sources", "k_collide"};
  if (!h || i < 0 || i >= h->kernels_per_step()) return "";
  if (!h->fused()) return names[i];
  lbm_handle *m = const_cast<lbm_handle *>(h);
  const bool sweep = h->variant < lbm::sweep_variant_count(h->dp);
  m->kname = std::string(sweep ? "k_step_sweep[" : "k_step_fused[") + lbm::fused_variant_name(h->dp, h->variant) + "]";
  return m->kname.c_str();
}

int lbm_kernel_config_count(const lbm_handle *h) {
  if (!h) return 0;
  return h->fused() ? lbm::fused_variant_count(h->dp) : 1;
}

lbm_status lbm_set_kernel_config(lbm_handle *h, int config) {
  if (!h) return LBM_E_INVAL;
  if (config < 0 || config >= lbm_kernel_config_count(h)) return h->fail(LBM_E_INVAL, "no such kernel configuration");
  h->variant = h->fused() ? config : 0;
  return LBM_OK;
}

lbm_status lbm_autotune(lbm_handle *h, int reps, int *chosen) {
  if (!h || reps < 1) return LBM_E_INVAL;
  if (!h->initialized) return h->fail(LBM_E_STATE, "autotune before initial fields");
  if (!h->fused()) {
    if (chosen) *chosen = 0;
    return LBM_OK;
  }
  const int nv = lbm::fused_variant_count(h->dp);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return h->fail(LBM_E_CUDA, "cudaEventCreate");
  // every candidate runs from the current state into the spare buffer; the
  // state itself is not advanced
  const lbm::FusedBuffers B = h->fused_buffers(h->cur, false);
  int best = 0;
  float best_ms = 0.f;
  cudaError_t err = cudaSuccess;
  for (int v = 0; v < nv && err == cudaSuccess; ++v) {
    err = lbm::launch_fused_step(h->dp, B, h->stream, v);  // warm-up and attribute set-up
    if (err != cudaSuccess) break;
    cudaEventRecord(e0, h->stream);
    for (int r = 0; r < reps; ++r) lbm::launch_fused_step(h->dp, B, h->stream, v);
    cudaEventRecord(e1, h->stream);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && (v == 0 || ms < best_ms)) {
      best = v;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return h->cuda_fail(err, "lbm_autotune");
  h->variant = best;
  if (chosen) *chosen = best;
  return LBM_OK;
}

lbm_status lbm_profile_step(lbm_handle *h, long long nsteps, double *ms_per_kernel, int nkernels) {
  if (!h || !ms_per_kernel || nsteps < 1) return LBM_E_INVAL;
  if (!h->initialized) return h->fail(LBM_E_STATE, "profile before initial fields");
  const int K = h->kernels_per_step();
  if (nkernels < K) return h->fail(LBM_E_INVAL, "ms_per_kernel too small");
  std::vector<cudaEvent_t> ev((size_t)(K + 1) * nsteps);
  for (auto &e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return h->fail(LBM_E_CUDA, "cudaEventCreate");
  for (long long t = 0; t < nsteps; ++t) h->launch_step(false, ev.data() + t * (K + 1));
  cudaError_t e = cudaStreamSynchronize(h->stream);
  for (int i = 0; i < K; ++i) ms_per_kernel[i] = 0.0;
  for (long long t = 0; t < nsteps && e == cudaSuccess; ++t)
    for (int i = 0; i < K; ++i) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[t * (K + 1) + i], ev[t * (K + 1) + i + 1]);
      ms_per_kernel[i] += ms / (double)nsteps;
    }
  for (auto &x : ev) cudaEventDestroy(x);
  if (e != cudaSuccess) return h->cuda_fail(e, "lbm_profile_step");
  h->step += nsteps;
  return LBM_OK;
}

void lbm_destroy(lbm_handle *h) { delete h; }

const char *lbm_last_error(const lbm_handle *h) { return h ? h->last_error.c_str() : "NULL handle"; }

}  // extern "C"
