// Surrogate network for the rising-bubble ensemble: an MLP 5 -> 128 -> 128 ->
// 128 -> 2 (tanh hidden layers) mapping (n, Eo, log10 Mo, density ratio,
// viscosity ratio) to (log terminal velocity, log drag coefficient), with BF16
// weights and FP32 accumulation on the tensor cores.  An ensemble of members
// trained from different initial weights gives a spread; inputs outside the
// box spanned by the training inputs, or with a spread above a threshold, are
// flagged so that the caller runs the lattice Boltzmann solve instead.
//
// Kernels: a small GEMM on mma.sync m16n8k16 (BF16 operands, FP32 accumulator)
// with operands read through row/column strides (so transposes cost nothing)
// and fused epilogues (bias + tanh, bias, tanh derivative), bias gradients,
// the loss gradient, and Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "lbm.h"

namespace surr {

constexpr int kLayers = 4;
constexpr int kSize[kLayers + 1] = {5, 128, 128, 128, 2};

constexpr int param_count() {
  int n = 0;
  for (int l = 0; l < kLayers; ++l) n += kSize[l + 1] * kSize[l] + kSize[l + 1];
  return n;
}
constexpr int kParams = param_count();

// Offset of W_l (out x in, row-major) and b_l in the flat parameter vector.
constexpr int w_off(int l) {
  int o = 0;
  for (int i = 0; i < l; ++i) o += kSize[i + 1] * kSize[i] + kSize[i + 1];
  return o;
}
constexpr int b_off(int l) { return w_off(l) + kSize[l + 1] * kSize[l]; }

enum Epilogue { kStore = 0, kBiasTanh = 1, kBias = 2, kTanhGrad = 3 };

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat16 l = __float2bfloat16_rn(lo), h = __float2bfloat16_rn(hi);
  return (uint32_t)__bfloat16_as_ushort(l) | ((uint32_t)__bfloat16_as_ushort(h) << 16);
}

// C (M x N) = A (M x K) B (K x N) with A(m, k) = A[m * as + k * ak] and
// B(k, n) = B[k * bk + n * bs], FP32 inputs rounded to BF16, FP32 accumulation.
// One warp per 16 x 8 output tile.  Epilogue on element (m, n):
//   kStore     C = acc
//   kBiasTanh  C = tanh(acc + bias[n])
//   kBias      C = acc + bias[n]
//   kTanhGrad  C = acc * (1 - aux[m * N + n]^2)   (aux: the layer's tanh output)
template <int EPI>
__global__ void k_gemm_bf16(int M, int N, int K, const float *__restrict__ A, long as, long ak,
                            const float *__restrict__ B, long bk, long bs, float *__restrict__ C,
                            const float *__restrict__ bias, const float *__restrict__ aux) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int tiles_n = (N + 7) / 8;
  const int tm = warp / tiles_n, tn = warp % tiles_n;
  if (tm * 16 >= M) return;  // whole warp leaves together
  const int gid = lane >> 2, tig = lane & 3;
  const int m0 = tm * 16 + gid, m1 = m0 + 8, n0 = tn * 8 + gid;
  auto a_at = [&](int m, int k) { return (m < M && k < K) ? A[m * as + k * ak] : 0.0f; };
  auto b_at = [&](int k, int n) { return (k < K && n < N) ? B[k * bk + n * bs] : 0.0f; };
  float d[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int ka = k0 + tig * 2, kb = ka + 8;
    uint32_t a[4], b[2];
    a[0] = pack_bf16(a_at(m0, ka), a_at(m0, ka + 1));
    a[1] = pack_bf16(a_at(m1, ka), a_at(m1, ka + 1));
    a[2] = pack_bf16(a_at(m0, kb), a_at(m0, kb + 1));
    a[3] = pack_bf16(a_at(m1, kb), a_at(m1, kb + 1));
    b[0] = pack_bf16(b_at(ka, n0), b_at(ka + 1, n0));
    b[1] = pack_bf16(b_at(kb, n0), b_at(kb + 1, n0));
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
  }
  const int cn = tn * 8 + tig * 2;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int m = (q < 2) ? m0 : m1, n = cn + (q & 1);
    if (m >= M || n >= N) continue;
    float v = d[q];
    if constexpr (EPI == kBiasTanh) v = tanhf(v + bias[n]);
    if constexpr (EPI == kBias) v = v + bias[n];
    if constexpr (EPI == kTanhGrad) {
      const float h = aux[(long)m * N + n];
      v = v * (1.0f - h * h);
    }
    C[(long)m * N + n] = v;
  }
}

template <int EPI>
cudaError_t gemm(int M, int N, int K, const float *A, long as, long ak, const float *B, long bk, long bs, float *C,
                 const float *bias, const float *aux, cudaStream_t s) {
  const int warps = ((M + 15) / 16) * ((N + 7) / 8);
  const int threads = 128;
  const int blocks = (warps * 32 + threads - 1) / threads;
  k_gemm_bf16<EPI><<<blocks, threads, 0, s>>>(M, N, K, A, as, ak, B, bk, bs, C, bias, aux);
  return cudaGetLastError();
}

// dZ = (Y - T) / B; loss partial sums per block (fixed order on the host).
__global__ void k_loss_grad(int n, const float *Y, const float *T, float *dZ, float *partial) {
  __shared__ float red[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < n * 2) {
    const float r = Y[i] - T[i];
    dZ[i] = r / (float)n;
    l = 0.5f * r * r;
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// db[j] = sum over rows of dZ[:, j].
__global__ void k_bias_grad(int rows, int cols, const float *dZ, float *db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += dZ[(long)r * cols + j];
  db[j] = s;
}

// Adam (Kingma and Ba 2015) on the FP32 master parameters.
__global__ void k_adam(int n, float *w, const float *g, float *m, float *v, float lr, float b1, float b2, float c1,
                       float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Row gather for mini-batches: out[r] = in[idx[r]] (rows of `cols` floats).
__global__ void k_gather(int rows, int cols, const int *idx, const float *in, float *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int r = i / cols, c = i % cols;
  out[i] = in[(long)idx[r] * cols + c];
}

}  // namespace surr

using namespace surr;

struct surr_net {
  int members = 1, max_batch = 0, max_rows = 0;
  cudaStream_t stream = nullptr;
  // device buffers (carved from the caller's arena)
  float *w = nullptr;        // members x kParams master weights
  float *g = nullptr;        // kParams gradients
  float *m = nullptr, *v = nullptr;  // members x kParams Adam moments
  float *act[kLayers + 1] = {};      // activations, max_batch rows each
  float *dz[kLayers] = {};           // pre-activation gradients
  float *X = nullptr, *T = nullptr;  // training set (max_rows x 5, x 2), normalised
  float *Xb = nullptr, *Tb = nullptr;
  int *idx = nullptr;
  float *partial = nullptr;
  // host state
  double in_mean[5] = {0}, in_std[5] = {1, 1, 1, 1, 1}, out_mean[2] = {0}, out_std[2] = {1, 1};
  double lo[5] = {0}, hi[5] = {0};
  bool trained = false;
  // out-of-fold residuals of the training rows (surr_train_cv) and the
  // local-trust bound of surr_answer
  std::vector<double> cv_x, cv_res;
  int trust_k = 0;
  double trust_max = 0.0;
  long long adam_t[16] = {0};
  std::string last_error;

  lbm_status cuda_fail(cudaError_t e, const char *where) {
    last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return LBM_E_CUDA;
  }

  // Forward pass of member `mem` on `rows` rows of act[0].
  cudaError_t forward(int mem, int rows) {
    const float *W = w + (long)mem * kParams;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
      const int in = kSize[l], out = kSize[l + 1];
      if (l < kLayers - 1)
        e = gemm<kBiasTanh>(rows, out, in, act[l], in, 1, W + w_off(l), 1, in, act[l + 1], W + b_off(l), nullptr,
                            stream);
      else
        e = gemm<kBias>(rows, out, in, act[l], in, 1, W + w_off(l), 1, in, act[l + 1], W + b_off(l), nullptr,
                        stream);
    }
    return e;
  }

  // Gradients of member `mem` into g for targets T (rows x 2); loss partials.
  cudaError_t backward(int mem, int rows, const float *Tt) {
    const float *W = w + (long)mem * kParams;
    const int nb = (rows * 2 + 255) / 256;
    k_loss_grad<<<nb, 256, 0, stream>>>(rows, act[kLayers], Tt, dz[kLayers - 1], partial);
    cudaError_t e = cudaGetLastError();
    for (int l = kLayers - 1; l >= 0 && e == cudaSuccess; --l) {
      const int in = kSize[l], out = kSize[l + 1];
      // dW_l (out x in) = dz_l^T (out x rows) act_l (rows x in)
      e = gemm<kStore>(out, in, rows, dz[l], 1, out, act[l], in, 1, g + w_off(l), nullptr, nullptr, stream);
      if (e != cudaSuccess) break;
      k_bias_grad<<<(out + 127) / 128, 128, 0, stream>>>(rows, out, dz[l], g + b_off(l));
      e = cudaGetLastError();
      if (e != cudaSuccess || l == 0) break;
      // dz_{l-1} (rows x in) = (dz_l (rows x out) W_l (out x in)) * (1 - act_l^2)
      e = gemm<kTanhGrad>(rows, in, out, dz[l], out, 1, W + w_off(l), in, 1, dz[l - 1], nullptr, act[l], stream);
    }
    return e;
  }
};

static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

static size_t layout(int members, int max_batch, int max_rows, surr_net *n, char *base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char * {
    char *p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  float *w = (float *)take((size_t)members * kParams * 4);
  float *g = (float *)take((size_t)kParams * 4);
  float *m = (float *)take((size_t)members * kParams * 4);
  float *v = (float *)take((size_t)members * kParams * 4);
  float *act[kLayers + 1], *dz[kLayers];
  for (int l = 0; l <= kLayers; ++l) act[l] = (float *)take((size_t)max_batch * kSize[l] * 4);
  for (int l = 0; l < kLayers; ++l) dz[l] = (float *)take((size_t)max_batch * kSize[l + 1] * 4);
  float *X = (float *)take((size_t)max_rows * 5 * 4);
  float *T = (float *)take((size_t)max_rows * 2 * 4);
  float *Tb = (float *)take((size_t)max_batch * 2 * 4);
  int *idx = (int *)take((size_t)max_batch * 4);
  float *partial = (float *)take((size_t)(max_batch * 2 / 256 + 2) * 4);
  if (n) {
    n->w = w;
    n->g = g;
    n->m = m;
    n->v = v;
    for (int l = 0; l <= kLayers; ++l) n->act[l] = act[l];
    for (int l = 0; l < kLayers; ++l) n->dz[l] = dz[l];
    n->X = X;
    n->T = T;
    n->Xb = act[0];
    n->Tb = Tb;
    n->idx = idx;
    n->partial = partial;
  }
  return off;
}

// SplitMix64 step for the host-side shuffles.
static uint64_t sm64(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

extern "C" {

int surr_param_count(void) { return kParams; }

size_t surr_required_bytes(int members, int max_batch, int max_rows) {
  if (members < 1 || members > 16 || max_batch < 1 || max_rows < 1) return 0;
  return layout(members, max_batch, max_rows, nullptr, nullptr);
}

lbm_status surr_create(int members, int max_batch, int max_rows, const double *init_weights, void *dev_arena,
                       size_t arena_bytes, void *cuda_stream, surr_net **out) {
  if (!out || !init_weights || !dev_arena) return LBM_E_INVAL;
  *out = nullptr;
  const size_t need = surr_required_bytes(members, max_batch, max_rows);
  if (need == 0 || ((uintptr_t)dev_arena % 256) != 0) return LBM_E_INVAL;
  if (arena_bytes < need) return LBM_E_NOMEM;
  surr_net *n = new (std::nothrow) surr_net();
  if (!n) return LBM_E_NOMEM;
  n->members = members;
  n->max_batch = max_batch;
  n->max_rows = max_rows;
  n->stream = (cudaStream_t)cuda_stream;
  layout(members, max_batch, max_rows, n, (char *)dev_arena);
  std::vector<float> w((size_t)members * kParams);
  for (size_t i = 0; i < w.size(); ++i) w[i] = (float)init_weights[i];
  cudaError_t e = cudaMemcpyAsync(n->w, w.data(), w.size() * 4, cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, w.size() * 4, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, w.size() * 4, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) {
    delete n;
    return LBM_E_CUDA;
  }
  *out = n;
  return LBM_OK;
}

void surr_destroy(surr_net *n) { delete n; }

const char *surr_last_error(const surr_net *n) { return n ? n->last_error.c_str() : "NULL network"; }

lbm_status surr_get_weights(surr_net *n, int member, double *out) {
  if (!n || !out || member < 0 || member >= n->members) return LBM_E_INVAL;
  std::vector<float> w(kParams);
  cudaError_t e = cudaMemcpyAsync(w.data(), n->w + (long)member * kParams, kParams * 4, cudaMemcpyDeviceToHost,
                                  n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return n->cuda_fail(e, "surr_get_weights");
  for (int i = 0; i < kParams; ++i) out[i] = w[i];
  return LBM_OK;
}

// Raw network (no normalisation): outputs for rows of X, optionally the loss
// and the gradients against targets T (rows x 2).  rows <= max_batch.
lbm_status surr_forward_backward(surr_net *n, int member, const double *X, const double *T, int rows, double *Y,
                                 double *loss, double *grads) {
  if (!n || !X || member < 0 || member >= n->members || rows < 1 || rows > n->max_batch) return LBM_E_INVAL;
  std::vector<float> x((size_t)rows * 5), t((size_t)rows * 2, 0.f);
  for (size_t i = 0; i < x.size(); ++i) x[i] = (float)X[i];
  if (T)
    for (size_t i = 0; i < t.size(); ++i) t[i] = (float)T[i];
  cudaError_t e = cudaMemcpyAsync(n->act[0], x.data(), x.size() * 4, cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(n->Tb, t.data(), t.size() * 4, cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) e = n->forward(member, rows);
  if (e == cudaSuccess && T) e = n->backward(member, rows, n->Tb);
  std::vector<float> y((size_t)rows * 2), g(kParams), part((rows * 2 + 255) / 256);
  if (e == cudaSuccess) e = cudaMemcpyAsync(y.data(), n->act[kLayers], y.size() * 4, cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess && T) e = cudaMemcpyAsync(g.data(), n->g, kParams * 4, cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess && T)
    e = cudaMemcpyAsync(part.data(), n->partial, part.size() * 4, cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return n->cuda_fail(e, "surr_forward_backward");
  if (Y)
    for (size_t i = 0; i < y.size(); ++i) Y[i] = y[i];
  if (T && grads)
    for (int i = 0; i < kParams; ++i) grads[i] = g[i];
  if (T && loss) {
    double s = 0;
    for (float p : part) s += p;
    *loss = s / rows;
  }
  return LBM_OK;
}

// Trains every member with Adam on mini-batches of the normalised set.
// X: rows x 5 raw inputs, Y: rows x 2 raw targets (taken as given: the caller
// passes log terminal velocity and log drag coefficient).  Normalisation (mean,
// std per column) and the input box are taken from this set.  batch >= rows
// means full-batch steps in the given order.
lbm_status surr_train(surr_net *n, const double *X, const double *Y, int rows, int epochs, int batch, double lr,
                      unsigned long long seed, double *final_loss) {
  if (!n || !X || !Y || rows < 1 || rows > n->max_rows || epochs < 0 || batch < 1 || !(lr > 0))
    return LBM_E_INVAL;
  batch = batch > rows ? rows : batch;
  if (batch > n->max_batch) return LBM_E_INVAL;
  n->cv_x.clear();  // out-of-fold residuals belong to the set they were computed on
  n->cv_res.clear();
  for (int c = 0; c < 5; ++c) {
    double s = 0, s2 = 0, lo = X[c], hi = X[c];
    for (int r = 0; r < rows; ++r) {
      const double v = X[r * 5 + c];
      s += v;
      s2 += v * v;
      lo = v < lo ? v : lo;
      hi = v > hi ? v : hi;
    }
    n->in_mean[c] = s / rows;
    const double var = s2 / rows - n->in_mean[c] * n->in_mean[c];
    n->in_std[c] = var > 1e-24 ? std::sqrt(var) : 1.0;
    n->lo[c] = lo;
    n->hi[c] = hi;
  }
  for (int c = 0; c < 2; ++c) {
    double s = 0, s2 = 0;
    for (int r = 0; r < rows; ++r) {
      s += Y[r * 2 + c];
      s2 += Y[r * 2 + c] * Y[r * 2 + c];
    }
    n->out_mean[c] = s / rows;
    const double var = s2 / rows - n->out_mean[c] * n->out_mean[c];
    n->out_std[c] = var > 1e-24 ? std::sqrt(var) : 1.0;
  }
  std::vector<float> xs((size_t)rows * 5), ys((size_t)rows * 2);
  for (int r = 0; r < rows; ++r) {
    for (int c = 0; c < 5; ++c) xs[r * 5 + c] = (float)((X[r * 5 + c] - n->in_mean[c]) / n->in_std[c]);
    for (int c = 0; c < 2; ++c) ys[r * 2 + c] = (float)((Y[r * 2 + c] - n->out_mean[c]) / n->out_std[c]);
  }
  cudaError_t e = cudaMemcpyAsync(n->X, xs.data(), xs.size() * 4, cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(n->T, ys.data(), ys.size() * 4, cudaMemcpyHostToDevice, n->stream);
  if (e != cudaSuccess) return n->cuda_fail(e, "surr_train upload");
  std::vector<int> perm(rows);
  double last = 0;
  for (int mem = 0; mem < n->members; ++mem) {
    uint64_t st = seed + 0x1234567ULL * (mem + 1);
    float *wm = n->w + (long)mem * kParams, *mm = n->m + (long)mem * kParams, *vm = n->v + (long)mem * kParams;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
      for (int r = 0; r < rows; ++r) perm[r] = r;
      if (batch < rows)
        for (int r = rows - 1; r > 0; --r) std::swap(perm[r], perm[(int)(sm64(st) % (uint64_t)(r + 1))]);
      for (int b0 = 0; b0 + batch <= rows && e == cudaSuccess; b0 += batch) {
        e = cudaMemcpyAsync(n->idx, perm.data() + b0, batch * 4, cudaMemcpyHostToDevice, n->stream);
        if (e != cudaSuccess) break;
        k_gather<<<(batch * 5 + 255) / 256, 256, 0, n->stream>>>(batch, 5, n->idx, n->X, n->act[0]);
        k_gather<<<(batch * 2 + 255) / 256, 256, 0, n->stream>>>(batch, 2, n->idx, n->T, n->Tb);
        e = n->forward(mem, batch);
        if (e == cudaSuccess) e = n->backward(mem, batch, n->Tb);
        if (e != cudaSuccess) break;
        const long long t = ++n->adam_t[mem];
        const float c1 = (float)(1.0 - std::pow(0.9, (double)t)), c2 = (float)(1.0 - std::pow(0.999, (double)t));
        k_adam<<<(kParams + 255) / 256, 256, 0, n->stream>>>(kParams, wm, n->g, mm, vm, (float)lr, 0.9f, 0.999f, c1,
                                                            c2, 1e-8f);
        e = cudaGetLastError();
      }
      // the copies above read `perm` from the host: finish before reshuffling
      if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    }
    if (e == cudaSuccess && final_loss) {
      // loss of the last mini-batch of this member
      std::vector<float> part((batch * 2 + 255) / 256);
      e = cudaMemcpyAsync(part.data(), n->partial, part.size() * 4, cudaMemcpyDeviceToHost, n->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
      double s = 0;
      for (float p : part) s += p;
      last = s / batch;
    }
  }
  if (e != cudaSuccess) return n->cuda_fail(e, "surr_train");
  n->trained = true;
  if (final_loss) *final_loss = last;
  return LBM_OK;
}

// Restores the initial weights of every member and restarts Adam.
static lbm_status surr_reset(surr_net *n, const double *init_weights) {
  std::vector<float> w((size_t)n->members * kParams);
  for (size_t i = 0; i < w.size(); ++i) w[i] = (float)init_weights[i];
  cudaError_t e = cudaMemcpyAsync(n->w, w.data(), w.size() * 4, cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, w.size() * 4, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, w.size() * 4, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return n->cuda_fail(e, "surr_reset");
  for (long long &t : n->adam_t) t = 0;
  n->trained = false;
  return LBM_OK;
}

static lbm_status train_cv(surr_net *n, const double *X, const double *Y, int rows, int folds, int epochs, int batch,
                           double lr, unsigned long long seed, const double *init_weights, double *final_loss);

lbm_status surr_train_cv(surr_net *n, const double *X, const double *Y, int rows, int folds, int epochs, int batch,
                         double lr, unsigned long long seed, const double *init_weights, double *final_loss) {
  if (!n || !X || !Y || !init_weights || rows < folds || folds < 2 || folds > 16 || rows > n->max_rows)
    return LBM_E_INVAL;
  const lbm_status s = train_cv(n, X, Y, rows, folds, epochs, batch, lr, seed, init_weights, final_loss);
  if (s != LBM_OK) {
    // the weights are those of an interrupted fold: not a usable ensemble
    n->trained = false;
    n->cv_x.clear();
    n->cv_res.clear();
  }
  return s;
}

static lbm_status train_cv(surr_net *n, const double *X, const double *Y, int rows, int folds, int epochs, int batch,
                           double lr, unsigned long long seed, const double *init_weights, double *final_loss) {
  // fold of each row: position in a seeded permutation, modulo folds
  std::vector<int> perm(rows), fold(rows);
  for (int r = 0; r < rows; ++r) perm[r] = r;
  uint64_t st = seed ^ 0x5DEECE66DULL;
  for (int r = rows - 1; r > 0; --r) std::swap(perm[r], perm[(int)(sm64(st) % (uint64_t)(r + 1))]);
  for (int i = 0; i < rows; ++i) fold[perm[i]] = i % folds;
  std::vector<double> res(rows, 0.0);
  for (int f = 0; f < folds; ++f) {
    std::vector<double> xt, yt, xv;
    std::vector<int> rv;
    for (int r = 0; r < rows; ++r) {
      if (fold[r] == f) {
        rv.push_back(r);
        xv.insert(xv.end(), X + 5 * r, X + 5 * r + 5);
      } else {
        xt.insert(xt.end(), X + 5 * r, X + 5 * r + 5);
        yt.insert(yt.end(), Y + 2 * r, Y + 2 * r + 2);
      }
    }
    lbm_status s = surr_reset(n, init_weights);
    if (s == LBM_OK) s = surr_train(n, xt.data(), yt.data(), (int)(xt.size() / 5), epochs, batch, lr, seed + f + 1, nullptr);
    if (s != LBM_OK) return s;
    const int nv = (int)rv.size();
    std::vector<double> mean((size_t)nv * 2);
    for (int r0 = 0; r0 < nv; r0 += n->max_batch) {
      const int m = nv - r0 < n->max_batch ? nv - r0 : n->max_batch;
      s = surr_predict(n, xv.data() + 5 * r0, m, mean.data() + 2 * r0, nullptr, nullptr);
      if (s != LBM_OK) return s;
    }
    for (int i = 0; i < nv; ++i) {
      const int r = rv[i];
      res[r] = std::fmax(std::fabs(mean[2 * i] - Y[2 * r]), std::fabs(mean[2 * i + 1] - Y[2 * r + 1]));
    }
  }
  lbm_status s = surr_reset(n, init_weights);
  if (s == LBM_OK) s = surr_train(n, X, Y, rows, epochs, batch, lr, seed, final_loss);
  if (s != LBM_OK) return s;
  n->cv_x.assign(X, X + 5 * (size_t)rows);
  n->cv_res = res;
  return LBM_OK;
}

lbm_status surr_local_residual(surr_net *n, const double *X, int rows, int k, double *local) {
  if (!n || !X || !local || rows < 0) return LBM_E_INVAL;
  const int nt = (int)n->cv_res.size();
  if (nt == 0 || !n->trained) {
    n->last_error = "surr_local_residual before surr_train_cv";
    return LBM_E_STATE;
  }
  if (k < 1 || k > nt) return LBM_E_INVAL;
  std::vector<std::pair<double, int>> d(nt);
  for (int r = 0; r < rows; ++r) {
    for (int t = 0; t < nt; ++t) {
      double s = 0.0;
      for (int c = 0; c < 5; ++c) {
        const double z = (X[5 * r + c] - n->cv_x[5 * (size_t)t + c]) / n->in_std[c];
        s += z * z;
      }
      d[t] = {s, t};
    }
    std::partial_sort(d.begin(), d.begin() + k, d.end());
    double m = 0.0;
    for (int i = 0; i < k; ++i) m = std::fmax(m, n->cv_res[d[i].second]);
    local[r] = m;
  }
  return LBM_OK;
}

lbm_status surr_set_local_trust(surr_net *n, int k, double max_residual) {
  if (!n || k < 1) return LBM_E_INVAL;
  n->trust_k = k;
  n->trust_max = max_residual;
  return LBM_OK;
}

// Ensemble prediction: mean and disagreement (largest deviation of a member
// from the mean) of the two outputs in raw units, and flags for inputs outside
// the training box.
lbm_status surr_predict(surr_net *n, const double *X, int rows, double *y_mean, double *y_spread, int *outside) {
  if (!n || !X || !y_mean || rows < 1 || rows > n->max_batch) return LBM_E_INVAL;
  if (!n->trained) {
    n->last_error = "surr_predict before surr_train";
    return LBM_E_STATE;
  }
  std::vector<float> xs((size_t)rows * 5), y((size_t)rows * 2);
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < 5; ++c) xs[r * 5 + c] = (float)((X[r * 5 + c] - n->in_mean[c]) / n->in_std[c]);
  std::vector<double> val((size_t)n->members * rows * 2), sum((size_t)rows * 2, 0.0);
  cudaError_t e = cudaSuccess;
  for (int mem = 0; mem < n->members && e == cudaSuccess; ++mem) {
    e = cudaMemcpyAsync(n->act[0], xs.data(), xs.size() * 4, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = n->forward(mem, rows);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y.data(), n->act[kLayers], y.size() * 4, cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    for (int i = 0; e == cudaSuccess && i < rows * 2; ++i) {
      const double v = y[i] * n->out_std[i % 2] + n->out_mean[i % 2];
      val[(size_t)mem * rows * 2 + i] = v;
      sum[i] += v;
    }
  }
  if (e != cudaSuccess) return n->cuda_fail(e, "surr_predict");
  for (int i = 0; i < rows * 2; ++i) {
    y_mean[i] = sum[i] / n->members;
    double dev = 0.0;
    for (int mem = 0; mem < n->members; ++mem)
      dev = std::fmax(dev, std::fabs(val[(size_t)mem * rows * 2 + i] - y_mean[i]));
    if (y_spread) y_spread[i] = dev;
  }
  if (outside)
    for (int r = 0; r < rows; ++r) {
      int o = 0;
      for (int c = 0; c < 5; ++c) o |= (X[r * 5 + c] < n->lo[c] || X[r * 5 + c] > n->hi[c]);
      outside[r] = o;
    }
  return LBM_OK;
}

// Terminal states from the network where it is trusted, from the lattice
// Boltzmann solver elsewhere (one batch of the untrusted cases in the caller's
// arena, run by lbm_batch_run).
lbm_status surr_answer(surr_net *n, const double *X, const lbm_params *cases, const lbm_bubble *bubbles, int rows,
                       double max_spread, double noise_amp, const lbm_run_opts *opts, void *dev_arena,
                       size_t arena_bytes, double *y_out, int *used_fallback, int *fallback_outcome) {
  if (!n || !X || !cases || !bubbles || !opts || !y_out || !used_fallback || rows < 1 || !(max_spread > 0))
    return LBM_E_INVAL;
  std::vector<double> mean((size_t)rows * 2), spread((size_t)rows * 2);
  std::vector<int> outside(rows);
  lbm_status st = surr_predict(n, X, rows, mean.data(), spread.data(), outside.data());
  if (st != LBM_OK) return st;
  const bool local_test = n->trust_max > 0.0;
  std::vector<double> local(rows, 0.0);
  if (local_test) {
    st = surr_local_residual(n, X, rows, n->trust_k, local.data());
    if (st != LBM_OK) return st;
  }
  std::vector<int> fb;
  for (int r = 0; r < rows; ++r) {
    const bool trusted = !outside[r] && spread[2 * r] < max_spread && spread[2 * r + 1] < max_spread &&
                         (!local_test || local[r] < n->trust_max);
    used_fallback[r] = trusted ? 0 : 1;
    if (fallback_outcome) fallback_outcome[r] = LBM_RUN_SKIPPED;
    // the network is trained on (log U_t, log C_D)
    y_out[2 * r] = trusted ? std::exp(mean[2 * r]) : NAN;
    y_out[2 * r + 1] = trusted ? std::exp(mean[2 * r + 1]) : NAN;
    if (!trusted) fb.push_back(r);
  }
  if (fb.empty()) return LBM_OK;
  std::vector<lbm_params> sub;
  for (int r : fb) sub.push_back(cases[r]);
  const size_t need = lbm_batch_required_bytes(sub.data(), (int)sub.size());
  if (need == 0) {
    n->last_error = "surr_answer: a fallback case's parameters are not valid for a batch";
    return LBM_E_INVAL;
  }
  if (!dev_arena || arena_bytes < need) {
    n->last_error = "surr_answer: the arena is smaller than lbm_batch_required_bytes of the fallback cases";
    return LBM_E_NOMEM;
  }
  lbm_batch *b = nullptr;
  st = lbm_batch_create(sub.data(), (int)sub.size(), dev_arena, arena_bytes, n->stream, &b);
  if (st != LBM_OK) {
    n->last_error = "surr_answer: lbm_batch_create failed";
    return st;
  }
  for (size_t k = 0; k < fb.size() && st == LBM_OK; ++k)
    st = lbm_init_bubbles(lbm_batch_case(b, (int)k), &bubbles[fb[k]], 1, (unsigned long long)fb[k], noise_amp);
  std::vector<lbm_obs> obs(fb.size());
  std::vector<int> outc(fb.size());
  if (st == LBM_OK) st = lbm_batch_run(b, opts, obs.data(), outc.data(), nullptr);
  if (st != LBM_OK) {
    n->last_error = std::string("surr_answer: ") + lbm_batch_last_error(b);
    lbm_batch_destroy(b);
    return st;
  }
  for (size_t k = 0; k < fb.size(); ++k) {
    const int r = fb[k];
    const bool ok = outc[k] != LBM_RUN_DIVERGED;
    y_out[2 * r] = ok ? obs[k].rise_velocity : NAN;
    y_out[2 * r + 1] = ok ? obs[k].drag_coefficient : NAN;
    if (fallback_outcome) fallback_outcome[r] = outc[k];
  }
  lbm_batch_destroy(b);
  return LBM_OK;
}

}  // extern "C"
