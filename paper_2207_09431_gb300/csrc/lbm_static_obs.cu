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
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kBlockNodes = 256;  // 256 consecutive nodes (row-major, x fastest) per block
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

// Column seen at x for offsets of one column: periodic, or (open x) the
// mirror ghost columns beyond the inlet and outlet, as the step kernels see it.
__device__ __forceinline__ int column_at(const DevParams &P, int x) {
  if (!P.open_x) return wrap_x(x, P.nx);
  return x < 0 ? -1 - x : (x >= P.nx ? 2 * P.nx - 1 - x : x);
}

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

// One block per 256 consecutive nodes of the row-major order (so that
// ceil(nx ny / 256) rows of the scratch array suffice for any shape): C, u
// (Eq. 23, with mu from Eq. 5) and the block's partial sums, written to its
// own row of the scratch array.
__global__ void k_obs_partial(DevParams P, const float *__restrict__ g, const float *__restrict__ hc, int collapse,
                              int gas_comp, StaticScratch *scr) {
  const long long node = (long long)blockIdx.x * kBlockNodes + threadIdx.x;
  const int blk = blockIdx.x;
  double v[kSums];
  for (int q = 0; q < kSums; ++q) v[q] = 0.0;
  int e[kExt] = {0x7fffffff, 0x7fffffff, 0x7fffffff, 0x7fffffff};
  if (node < (long long)P.nx * P.ny) {
    const int x = (int)(node % P.nx), y = (int)(node / P.nx);
    const long long k = (long long)y * P.pitch + x;
    float Cn[9][3], rn[9];
    for (int a = 0; a < 9; ++a) {
      const int xs = column_at(P, x + ex(a)), ys = wrap_y(y + ey(a), P.ny, P.periodic_y);
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
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    for (int q = 0; q < kSums; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], off);
    for (int q = 0; q < kExt; ++q) e[q] = min(e[q], __shfl_down_sync(0xffffffffu, e[q], off));
  }
  if (lane == 0) {
    for (int q = 0; q < kSums; ++q) ws[warp][q] = v[q];
    for (int q = 0; q < kExt; ++q) we[warp][q] = e[q];
  }
  __syncthreads();
  if (warp == 0 && lane < kSums) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += ws[w][lane];
    scr->partial[blk][lane] = s;
  }
  if (warp == 1 && lane < kExt) {
    int m = 0x7fffffff;
    for (int w = 0; w < 8; ++w) m = min(m, we[w][lane]);
    scr->ext[blk][lane] = m;
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
// per device by the first call made on it.
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
  if (validate(p)) return LBM_E_INVAL;
  if (p->storage != 0) return LBM_E_INVAL;  // g is read as FP32 planes
  if (pitch < p->nx || plane_stride < (long long)pitch * p->ny) return LBM_E_INVAL;
  if ((long long)p->nx * p->ny > LBM_STATIC_MAX_NODES) return LBM_E_RANGE;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  {
    // the call reads its results back and waits for the stream, which a
    // capturing stream does not allow
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return LBM_E_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return LBM_E_INVAL;
  }
  const int nblocks = (int)(((long long)p->nx * p->ny + lbm::kBlockNodes - 1) / lbm::kBlockNodes);
  lbm::DevParams d = dev_params(*p);
  d.pitch = pitch;
  d.plane = plane_stride;
  lbm::StaticScratch *scr = nullptr;
  if (lbm::scratch_on_current_device(&scr) != cudaSuccess) return LBM_E_CUDA;
  lbm::k_obs_partial<<<nblocks, lbm::kBlockNodes, 0, s>>>(d, g, hc, p->collapse_h ? 1 : 0, p->gas_comp, scr);
  lbm::k_obs_total<<<1, 256, 0, s>>>(nblocks, scr);
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
