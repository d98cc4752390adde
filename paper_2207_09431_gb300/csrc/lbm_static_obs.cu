// Observables of a lattice state held in caller buffers, without any device
// allocation: the reduction scratch is a fixed file-scope device array.
//
// Who needs this: a caller that owns all device memory itself (for example an
// application that reserves its whole device budget at start-up and hands out
// fixed buffers, so any later cudaMalloc would fail or is forbidden by its
// memory policy) cannot give lbm_create an arena for a short query, and cannot
// let the library allocate one.  It still holds the populations of its lattice
// and wants the masses, centroid and rise velocity of that state.
//
// The per-block partial sums live in `g_static_scratch`, which every GPU that
// loads this library keeps for the life of the process (LBM_STATIC_MAX_NODES
// nodes, 416 KB).  Host code must not pass the array's name to a kernel: on the
// host it is only a stand-in symbol, so the device address is looked up once
// per device with cudaGetSymbolAddress and cached.  Every call overwrites the
// rows it uses, so nothing has to be cleared between calls; two calls that
// overlap on the GPU (different streams, or different host threads) race on
// the same array.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "lbm.h"
#include "lbm_device.cuh"

namespace lbm {
namespace {

constexpr int kBlockNodes = 256;  // 32 x 8 nodes per block
constexpr int kMaxBlocks = LBM_STATIC_MAX_NODES / kBlockNodes;
constexpr int kSums = 11;          // M1..3, M1..3 above 0.5, A, sum Cx, sum Cy, sum C ux, sum C uy
constexpr int kExt = 4;            // xmin, -xmax, ymin, -ymax

struct StaticScratch {
  double partial[kMaxBlocks][kSums];
  int ext[kMaxBlocks][kExt];
  double total[kSums];
  int ext_total[kExt];
};

__device__ __align__(256) StaticScratch g_static_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
StaticScratch *g_scratch_ptr[kMaxDevices] = {};

// C_1..C_3 at node k from the populations (Eq. 22) or from the stored C.
__device__ __forceinline__ void order_params(const DevParams &P, const float *hc, int collapse, long long k,
                                             float C[3]) {
  C[0] = C[1] = 0.f;
  for (int i = 0; i < P.nh; ++i) {
    float acc = 0.f;
    if (collapse) {
      acc = hc[(long long)i * P.plane + k];
    } else {
      for (int a = 0; a < 9; ++a) acc += hc[((long long)i * 9 + a) * P.plane + k];
    }
    C[i] = acc;
  }
  C[2] = 1.0f - C[0] - C[1];
}

// One block per 32 x 8 nodes: C, u (Eq. 23, with mu from Eq. 5) and the
// block's partial sums, written to its own row of the scratch array.
__global__ void k_obs_partial(DevParams P, const float *__restrict__ g, const float *__restrict__ hc, int collapse,
                              int gas_comp, StaticScratch *scr) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  const int blk = blockIdx.y * gridDim.x + blockIdx.x;
  double v[kSums];
  for (int q = 0; q < kSums; ++q) v[q] = 0.0;
  int e[kExt] = {0x7fffffff, 0x7fffffff, 0x7fffffff, 0x7fffffff};
  if (x < P.nx && y < P.ny) {
    const long long k = (long long)y * P.pitch + x;
    float Cn[9][3], rn[9];
    for (int a = 0; a < 9; ++a) {
      const int xs = wrap_x(x + ex(a), P.nx), ys = wrap_y(y + ey(a), P.ny, P.periodic_y);
      order_params(P, hc, collapse, (long long)ys * P.pitch + xs, Cn[a]);
      rn[a] = rho_of(P, Cn[a][0], Cn[a][1], Cn[a][2]);
    }
    float lap[3], gx[3], gy[3], mu[3], rx = 0.f, ry = 0.f;
    for (int j = 0; j < 3; ++j) {
      float sx = 0.f, sy = 0.f, lp = 0.f;
      for (int a = 0; a < 9; ++a) {
        sx += wt(a) * ex(a) * Cn[a][j];
        sy += wt(a) * ey(a) * Cn[a][j];
        lp += wt(a) * (Cn[a][j] - Cn[0][j]);
      }
      gx[j] = 3.0f * sx;
      gy[j] = 3.0f * sy;
      lap[j] = 6.0f * lp;
    }
    for (int a = 0; a < 9; ++a) {
      rx += wt(a) * ex(a) * rn[a];
      ry += wt(a) * ey(a) * rn[a];
    }
    chem_potentials(P, Cn[0], lap, mu);
    const float Fsx = mu[0] * gx[0] + mu[1] * gx[1] + mu[2] * gx[2];
    const float Fsy = mu[0] * gy[0] + mu[1] * gy[1] + mu[2] * gy[2];
    const float rho = rn[0];
    float mx = 0.f, my = 0.f;
    for (int a = 0; a < 9; ++a) {
      const float ga = g[(long long)a * P.plane + k];
      mx += ex(a) * ga;
      my += ey(a) * ga;
    }
    const float ux = (3.0f * mx + 0.5f * (Fsx + P.force_x)) / rho;
    const float uy = (3.0f * my + 0.5f * (Fsy - rho * P.gravity)) / rho;
    for (int i = 0; i < 3; ++i) {
      v[i] = Cn[0][i];
      v[3 + i] = Cn[0][i] > 0.5f ? (double)Cn[0][i] : 0.0;
    }
    const double cg = Cn[0][gas_comp - 1];
    v[6] = cg;
    v[7] = cg * x;
    v[8] = cg * y;
    v[9] = cg * ux;
    v[10] = cg * uy;
    if (Cn[0][gas_comp - 1] > 0.5f) {
      e[0] = x;
      e[1] = -x;
      e[2] = y;
      e[3] = -y;
    }
  }
  // fixed-order reduction: warp shuffles, then the 8 warp results in order
  __shared__ double ws[8][kSums];
  __shared__ int we[8][kExt];
  for (int off = 16; off > 0; off >>= 1) {
    for (int q = 0; q < kSums; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
    for (int q = 0; q < kExt; ++q) e[q] = min(e[q], __shfl_down_sync(0xffffffffu, e[q], off));
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < kSums; ++q) ws[threadIdx.y][q] = v[q];
    for (int q = 0; q < kExt; ++q) we[threadIdx.y][q] = e[q];
  }
  __syncthreads();
  if (threadIdx.y == 0 && threadIdx.x < kSums) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += ws[w][threadIdx.x];
    scr->partial[blk][threadIdx.x] = s;
  }
  if (threadIdx.y == 1 && threadIdx.x < kExt) {
    int m = 0x7fffffff;
    for (int w = 0; w < 8; ++w) m = min(m, we[w][threadIdx.x]);
    scr->ext[blk][threadIdx.x] = m;
  }
}

// One block folds the partial rows in a fixed order.
__global__ void k_obs_total(int nblocks, StaticScratch *scr) {
  __shared__ double red[256];
  __shared__ int rede[256];
  for (int q = 0; q < kSums + kExt; ++q) {
    double s = 0.0;
    int m = 0x7fffffff;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
      if (q < kSums) s += scr->partial[b][q];
      else m = min(m, scr->ext[b][q - kSums]);
    }
    red[threadIdx.x] = s;
    rede[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        red[threadIdx.x] += red[threadIdx.x + w];
        rede[threadIdx.x] = min(rede[threadIdx.x], rede[threadIdx.x + w]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (q < kSums) scr->total[q] = red[0];
      else scr->ext_total[q - kSums] = rede[0];
    }
    __syncthreads();
  }
}

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does it; make that first call before
// any stream capture on the device).
cudaError_t scratch_on_current_device(StaticScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<StaticScratch *>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace lbm

extern "C" lbm_status lbm_observables_static(const lbm_params *p, const float *g, const float *hc, int pitch,
                                             long long plane_stride, double raw_out[15], void *cuda_stream) {
  if (!p || !g || !hc || !raw_out) return LBM_E_INVAL;
  if (p->nx < 1 || p->ny < 3 || (p->ncomp != 2 && p->ncomp != 3) || (p->gas_comp != 2 && p->gas_comp != 3))
    return LBM_E_INVAL;
  if (pitch < p->nx || plane_stride < (long long)pitch * p->ny) return LBM_E_INVAL;
  if ((long long)p->nx * p->ny > LBM_STATIC_MAX_NODES) return LBM_E_RANGE;
  const int bx = (p->nx + 31) / 32, by = (p->ny + 7) / 8;
  if (bx * by > lbm::kMaxBlocks) return LBM_E_RANGE;
  lbm::DevParams d{};
  d.nx = p->nx;
  d.ny = p->ny;
  d.pitch = pitch;
  d.ncomp = p->ncomp;
  d.nh = p->ncomp - 1;
  d.periodic_y = p->periodic_y ? 1 : 0;
  for (int i = 0; i < 3; ++i) d.rho[i] = (float)p->rho[i];
  d.sig12 = (float)p->sigma12;
  d.sig13 = (float)p->sigma13;
  d.sig23 = (float)p->sigma23;
  d.Lambda = (float)p->Lambda;
  const double S1 = p->sigma12 + p->sigma13 - p->sigma23;
  const double S2 = p->sigma12 + p->sigma23 - p->sigma13;
  const double S3 = p->sigma13 + p->sigma23 - p->sigma12;
  if (!(S1 > 0 && S2 > 0 && S3 > 0) || !(p->xi > 0)) return LBM_E_INVAL;
  d.Sig[0] = (float)S1;
  d.Sig[1] = (float)S2;
  d.Sig[2] = (float)S3;
  d.SigT = (float)(3.0 / (1.0 / S1 + 1.0 / S2 + 1.0 / S3));
  d.xi = (float)p->xi;
  const double Sg[3] = {S1, S2, S3};
  for (int i = 0; i < 3; ++i) {
    d.inv_sig[i] = (float)(1.0 / Sg[i]);
    d.grad_coef[i] = (float)(0.75 * p->xi * Sg[i]);
  }
  d.mu_pre = (float)(4.0 * (3.0 / (1.0 / S1 + 1.0 / S2 + 1.0 / S3)) / p->xi);
  d.gravity = (float)p->gravity;
  d.force_x = (float)p->force_x;
  d.plane = plane_stride;
  lbm::StaticScratch *scr = nullptr;
  if (lbm::scratch_on_current_device(&scr) != cudaSuccess) return LBM_E_CUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  lbm::k_obs_partial<<<dim3(bx, by), dim3(32, 8), 0, s>>>(d, g, hc, p->collapse_h ? 1 : 0, p->gas_comp, scr);
  lbm::k_obs_total<<<1, 256, 0, s>>>(bx * by, scr);
  double total[lbm::kSums];
  int ext[lbm::kExt];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(total, scr->total, sizeof(total), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ext, scr->ext_total, sizeof(ext), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return LBM_E_CUDA;
  for (int q = 0; q < lbm::kSums; ++q) raw_out[q] = total[q];
  const bool any = ext[0] != 0x7fffffff;
  raw_out[11] = any ? ext[0] : -1.0;
  raw_out[12] = any ? -ext[1] : -1.0;
  raw_out[13] = any ? ext[2] : -1.0;
  raw_out[14] = any ? -ext[3] : -1.0;
  return LBM_OK;
}
