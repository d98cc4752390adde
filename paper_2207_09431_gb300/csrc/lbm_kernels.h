// Launchers shared between the C-ABI host code and the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "lbm_devparams.h"

namespace lbm {

// Population arrays (g, and h in the population state form) keep their nq
// planes interleaved in blocks of 32 columns: element q of node
// k = y * pitch + x (pitch a multiple of 32) is at
// ((k / 32) * nq + q) * 32 + k % 32, so the planes of a node are 128 bytes
// apart, a constant the step kernels fold into their loads and stores.  Every
// other array (tau, C, mu, p, u, ...) is planar: element i of node k at
// i * plane + k.
__host__ __device__ constexpr long long pop_index(long long k, int q, int nq) {
  return ((k >> 5) * nq + q) * 32 + (k & 31);
}

// Device buffers of one step.  *_in are the current state, *_out the next one;
// the remaining planes are scratch fields.
struct StepBuffers {
  const float *g_in, *h_in, *tau_in;
  float *g_out, *h_out, *tau_out;
  float *C, *mu, *p, *ux, *uy, *shear, *SV;
  unsigned *err;
};

// Launches one step; if ev is non-null, records ev[i] before kernel i and
// ev[nkernels] after the last one.
constexpr int kSplitKernels = 4;
void launch_split_step(const DevParams &P, const StepBuffers &B, cudaStream_t s, cudaEvent_t *ev = nullptr);
// Buffers of the fused single-kernel step.  shear and SV may be null (no
// diagnostics written).
struct FusedBuffers {
  const float *g_in, *h_in, *tau_in;
  float *g_out, *h_out, *tau_out;
  float *shear, *SV;
  unsigned *err;
};

// One lattice of a batch: its parameters and both buffer sets; buffer set
// base_parity ^ parity is the input of the step launched with `parity`.
struct BatchCase {
  DevParams P;
  FusedBuffers B[2];
  int base_parity;
};
// One CTA of a batched step: a case and the origin of one of its tiles.
struct WorkItem {
  int case_id, x0, y0, y1;  // y1: end row of a sweep segment (unused by tiles)
};

// Grid-wide barrier state of the persistent batched step: arrivals of the
// current barrier, the barrier generation, and the status word (bit 0: a wait
// ran out of its iteration limit).  Zeroed by the host before each launch.
struct GridSync {
  unsigned count, gen, status, pad;
  unsigned next[2];  // work-item counters of even and odd steps (dynamic assignment)
  unsigned pad2[2];
};
constexpr unsigned kSyncTimeout = 1u;

bool fused_supported(const DevParams &P);
// Configurations of the batched step: sweeps (work items (case, strip,
// segment)) first, then tiles (work items (case, tile)).
int batched_variant_count(int nh);
bool batched_variant_is_sweep(int nh, int v);
void batched_variant_tile(int nh, int v, int *tx, int *ty);
int sweep_batched_count(int nh);
void sweep_batched_shape(int nh, int v, int *tx, int *rows);
// form: 0 populations g, h; 1 g and C (collapse_h); 2 FP16 g deviations and C
cudaError_t launch_sweep_batched(int nh, int form, const BatchCase *cases, const WorkItem *work, int nwork,
                                 int parity, cudaStream_t s, int v);
cudaError_t launch_batched_step(int nh, int form, const BatchCase *cases, const WorkItem *work, int nwork,
                                int parity, cudaStream_t s, int v);
// nsteps time steps of every work item in one persistent cooperative launch
// (sweep configurations v < sweep_batched_count(nh) only): the CTAs that fit
// on the device at once share the items of a step and meet at a grid barrier
// between steps; a barrier wait gives up after spin_limit polls, sets
// kSyncTimeout in sync->status and the kernel returns.  *grid = CTAs launched.
cudaError_t launch_sweep_persistent(int nh, int form, const BatchCase *cases, const WorkItem *work, int nwork,
                                    int parity0, int nsteps, GridSync *sync, long long spin_limit, cudaStream_t s,
                                    int v, int *grid);
// Launch configurations of the fused step: row sweeps (strip width, rows per
// pipeline step, threads, CTAs per SM), then tiles (tile, threads, CTAs per SM).
int sweep_variant_count(const DevParams &P);
const char *sweep_variant_name(const DevParams &P, int v);
// Configuration a handle starts with: the sweep that measured fastest on the
// 2048 x 4096 rising bubble (60 x 2 strips, 160 threads, 3 CTAs per SM).
int sweep_default_variant(const DevParams &P);
cudaError_t launch_sweep_step(const DevParams &P, const FusedBuffers &B, cudaStream_t s, int v);
int fused_variant_count(const DevParams &P);
const char *fused_variant_name(const DevParams &P, int v);
cudaError_t launch_fused_step(const DevParams &P, const FusedBuffers &B, cudaStream_t s, int v);
// FP16 storage (P.g16): g32 holds 9 FP32 planes, g16 the same space as 9 half
// planes followed by the FP32 plane of the per-node reference sum_a g_a.
cudaError_t launch_g16_encode(const DevParams &P, const float *g32, float *g16, cudaStream_t s);
cudaError_t launch_g16_decode(const DevParams &P, const float *g16, float *g32, cudaStream_t s);

void launch_macros(const DevParams &P, const StepBuffers &B, cudaStream_t s);
void launch_init(const DevParams &P, const StepBuffers &B, cudaStream_t s);
// nplanes dense FP64 planes (ny x nx each, device) into pitched FP32 planes
// (plane stride P.plane floats).
cudaError_t launch_planes_from_f64(const DevParams &P, const double *src, float *dst, int nplanes, cudaStream_t s);

}  // namespace lbm
