// Batched ensemble of lattices (many rising-bubble cases of different sizes
// and parameters): every active case advances in one kernel launch per time
// step over a work list of (case, tile) items, and runs of steps are replayed
// from a captured CUDA graph; or (persistent mode) in one cooperative launch
// for thousands of steps, whose CTAs share each step's work items and meet at
// a bounded grid barrier between steps, replayed from a captured graph too.  Each case is an ordinary lbm_handle carved from
// the batch arena, so initial conditions, observables, fields and checkpoints
// use the single-lattice calls on lbm_batch_case(b, i).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int kGraphSteps = 16;  // time steps per captured graph (even: parity returns)
// time steps per persistent launch (even); about 2 s for 128 cases of up to
// 300 x 600, so a launch stays short and a run of steps is a few graph replays
constexpr int kPersistSteps = 4096;
// polls of a grid-barrier wait before it gives up (each poll sleeps ~64 ns and
// reads two words from L2: well over a second, against microseconds expected)
constexpr long long kDefaultSpinLimit = 1LL << 22;

size_t batch_table_bytes(int n) { return align_up((size_t)n * sizeof(lbm::BatchCase), kAlign); }
size_t batch_err_bytes(int n) { return align_up((size_t)n * sizeof(unsigned), kAlign); }
size_t batch_sync_bytes() { return align_up(sizeof(lbm::GridSync), kAlign); }

// Upper bound of work items: tiles of the smallest tile shape.
size_t max_work(const lbm_params *cases, int n) {
  size_t w = 0;
  for (int i = 0; i < n; ++i) w += (size_t)((cases[i].nx + 31) / 32) * ((cases[i].ny + 7) / 8);
  return w;
}

}  // namespace

struct lbm_batch {
  int n = 0;
  cudaStream_t stream = nullptr;
  std::vector<lbm_handle *> h;
  std::vector<char> active;
  lbm::BatchCase *d_cases = nullptr;
  lbm::WorkItem *d_work = nullptr;
  unsigned *d_err = nullptr;
  lbm::GridSync *d_sync = nullptr;
  bool persistent = false;
  long long spin_limit = kDefaultSpinLimit;
  cudaGraphExec_t pgraph = nullptr;  // one persistent launch of kPersistSteps steps
  int pgraph_nwork = -1, pgraph_variant = -1;
  long long pgraph_limit = -1;
  size_t work_cap = 0;
  int nwork = 0;
  int variant = 0;
  int nh = 1;
  int form = 0;  // 0 populations, 1 C state (collapse_h), 2 FP16 g and C (storage 1)
  bool work_valid = false;
  cudaGraphExec_t graph = nullptr;
  int graph_nwork = -1, graph_variant = -1;
  std::string last_error;

  lbm_status fail(lbm_status s, const std::string &m) {
    last_error = m;
    return s;
  }
  lbm_status cuda_fail(cudaError_t e, const char *where) {
    last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return LBM_E_CUDA;
  }
  ~lbm_batch() {
    if (graph) cudaGraphExecDestroy(graph);
    if (pgraph) cudaGraphExecDestroy(pgraph);
    for (auto *x : h) delete x;
  }

  // Work list of the active, initialised cases for configuration v (tiles, or
  // strips x row segments of a sweep); uploads it.
  cudaError_t build_work(int v, int *count) {
    std::vector<lbm::WorkItem> w;
    for (int i = 0; i < n; ++i) {
      if (!active[i] || !h[i]->initialized) continue;
      int tx = 32, ty = 8;
      lbm::batched_variant_tile(nh, v, &tx, &ty);
      const int ny = h[i]->dp.ny;
      if (lbm::batched_variant_is_sweep(nh, v)) {
        // sweep segments: the rows of a strip split evenly (an even number of
        // rows each, as the two-row pipeline steps take them), so that no
        // short last segment pays a whole pipeline fill for a few rows
        const int nseg = (ny + ty - 1) / ty;
        int len = (ny + nseg - 1) / nseg;
        len += len & 1;
        for (int y0 = 0; y0 < ny; y0 += len)
          for (int x0 = 0; x0 < h[i]->dp.nx; x0 += tx) w.push_back({i, x0, y0, y0 + len < ny ? y0 + len : ny});
      } else {
        for (int y0 = 0; y0 < ny; y0 += ty)
          for (int x0 = 0; x0 < h[i]->dp.nx; x0 += tx) w.push_back({i, x0, y0, y0 + ty < ny ? y0 + ty : ny});
      }
    }
    // longest items first: the CTAs take items in order (one launch per step,
    // or from a counter in the persistent launch), which then approximates the
    // longest-processing-time schedule
    std::stable_sort(w.begin(), w.end(), [](const lbm::WorkItem &a, const lbm::WorkItem &b) {
      return a.y1 - a.y0 > b.y1 - b.y0;
    });
    if (w.size() > work_cap) return cudaErrorInvalidValue;  // the arena's work list is sized for 32 x 8 items
    *count = (int)w.size();
    if (w.empty()) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(d_work, w.data(), w.size() * sizeof(lbm::WorkItem), cudaMemcpyHostToDevice,
                                    stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    return e;
  }

  // Case table with every case's parameters, both buffer sets and current parity.
  cudaError_t upload_table() {
    std::vector<lbm::BatchCase> t(n);
    for (int i = 0; i < n; ++i) {
      t[i].P = h[i]->dp;
      t[i].B[0] = h[i]->fused_buffers(0, false);
      t[i].B[1] = h[i]->fused_buffers(1, false);
      t[i].B[0].err = t[i].B[1].err = d_err + i;
      t[i].base_parity = h[i]->cur;
    }
    cudaError_t e = cudaMemcpyAsync(d_cases, t.data(), t.size() * sizeof(lbm::BatchCase), cudaMemcpyHostToDevice,
                                    stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    return e;
  }
};

// Persistent mode of lbm_batch_step: whole launches of kPersistSteps steps
// replayed from a captured graph (barrier state reset, then the launch), the
// remainder in one direct launch; then the error words and the barrier status.
static lbm_status persistent_steps(lbm_batch *b, long long nsteps) {
  if (!lbm::batched_variant_is_sweep(b->nh, b->variant))
    return b->fail(LBM_E_STATE, "persistent mode runs sweep configurations (autotune in persistent mode)");
  cudaError_t e = cudaSuccess;
  int grid = 0;
  auto one_launch = [&](int steps) {
    cudaError_t r = cudaMemsetAsync(b->d_sync, 0, sizeof(lbm::GridSync), b->stream);
    if (r == cudaSuccess)
      r = lbm::launch_sweep_persistent(b->nh, b->form, b->d_cases, b->d_work, b->nwork, 0, steps, b->d_sync,
                                       b->spin_limit, b->stream, b->variant, &grid);
    return r;
  };
  const bool capturable = b->stream != nullptr && b->stream != cudaStreamLegacy && b->stream != cudaStreamPerThread;
  const long long full = capturable ? nsteps / kPersistSteps : 0;
  if (full > 0 && (!b->pgraph || b->pgraph_nwork != b->nwork || b->pgraph_variant != b->variant ||
                   b->pgraph_limit != b->spin_limit)) {
    // kernel attributes and occupancy are queried outside the capture
    e = lbm::launch_sweep_persistent(b->nh, b->form, b->d_cases, b->d_work, b->nwork, 0, 0, b->d_sync,
                                     b->spin_limit, b->stream, b->variant, &grid);
    if (e != cudaSuccess) return b->cuda_fail(e, "lbm_batch_step persistent prepare");
    if (b->pgraph) cudaGraphExecDestroy(b->pgraph);
    b->pgraph = nullptr;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = one_launch(kPersistSteps);
    cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = ec;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->pgraph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return b->cuda_fail(e, "lbm_batch_step persistent graph capture");
    b->pgraph_nwork = b->nwork;
    b->pgraph_variant = b->variant;
    b->pgraph_limit = b->spin_limit;
  }
  std::vector<unsigned> err(b->n);
  lbm::GridSync sync{};
  long long done = 0;
  // one replay or launch at a time, each checked, so that a wait that ran out
  // stops the run at that launch
  while (done < nsteps && e == cudaSuccess) {
    const long long left = nsteps - done;
    int steps;
    if (done < full * (long long)kPersistSteps) {
      steps = kPersistSteps;
      e = cudaGraphLaunch(b->pgraph, b->stream);
    } else {
      steps = (int)(left < kPersistSteps ? left : kPersistSteps);
      e = one_launch(steps);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&sync, b->d_sync, sizeof(sync), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) break;
    if (sync.status & lbm::kSyncTimeout) {
      // the launch stopped part-way: no case holds a whole time step
      for (int i = 0; i < b->n; ++i)
        if (b->active[i]) b->h[i]->initialized = false;
      b->work_valid = false;
      return b->fail(LBM_E_TIMEOUT, "a grid-barrier wait of the persistent step ran out after " +
                                        std::to_string(b->spin_limit) + " polls (" + std::to_string(grid) +
                                        " CTAs); the active cases must be set again");
    }
    done += steps;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(err.data(), b->d_err, err.size() * sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return b->cuda_fail(e, "lbm_batch_step persistent launch");
  std::string diverged;
  for (int i = 0; i < b->n; ++i) {
    if (!b->active[i] || !b->h[i]->initialized) continue;
    if (nsteps & 1) b->h[i]->cur = 1 - b->h[i]->cur;
    b->h[i]->step += nsteps;
    if (err[i]) {
      diverged += " " + std::to_string(i);
      b->active[i] = 0;
      b->work_valid = false;
    }
  }
  if (!diverged.empty()) return b->fail(LBM_E_DIVERGED, "non-finite values in case(s)" + diverged + "; deactivated");
  return LBM_OK;
}

extern "C" {

size_t lbm_batch_required_bytes(const lbm_params *cases, int ncases) {
  if (!cases || ncases < 1) return 0;
  size_t total = 0;
  for (int i = 0; i < ncases; ++i) {
    const size_t b = lbm_required_bytes(&cases[i]);
    if (b == 0 || cases[i].open_x) return 0;  // periodic x only
    total += align_up(b, kAlign);
  }
  total += batch_table_bytes(ncases) + batch_err_bytes(ncases) + batch_sync_bytes();
  total += align_up(max_work(cases, ncases) * sizeof(lbm::WorkItem), kAlign);
  return total;
}

lbm_status lbm_batch_create(const lbm_params *cases, int ncases, void *dev_arena, size_t arena_bytes,
                            void *cuda_stream, lbm_batch **out) {
  if (!out) return LBM_E_INVAL;
  *out = nullptr;
  const size_t need = lbm_batch_required_bytes(cases, ncases);
  if (need == 0) return LBM_E_INVAL;
  if (!dev_arena || ((uintptr_t)dev_arena % kAlign) != 0) return LBM_E_INVAL;
  if (arena_bytes < need) return LBM_E_NOMEM;
  for (int i = 0; i < ncases; ++i) {
    if (cases[i].ncomp != cases[0].ncomp || cases[i].collapse_h != cases[0].collapse_h || cases[i].fd_scheme != 0 ||
        cases[i].storage != cases[0].storage)
      return LBM_E_INVAL;  // one kernel: same component count and state form, central differences
  }
  lbm_batch *b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_E_NOMEM;
  b->n = ncases;
  b->stream = (cudaStream_t)cuda_stream;
  b->nh = cases[0].ncomp - 1;
  b->form = cases[0].storage == 1 ? 2 : (cases[0].collapse_h ? 1 : 0);
  b->active.assign(ncases, 1);
  char *base = (char *)dev_arena;
  size_t off = 0;
  for (int i = 0; i < ncases; ++i) {
    const size_t bytes = align_up(lbm_required_bytes(&cases[i]), kAlign);
    lbm_handle *hi = nullptr;
    lbm_status st = lbm_create(&cases[i], base + off, bytes, cuda_stream, &hi);
    if (st != LBM_OK) {
      delete b;
      return st;
    }
    b->h.push_back(hi);
    off += bytes;
  }
  b->d_cases = (lbm::BatchCase *)(base + off);
  off += batch_table_bytes(ncases);
  b->d_err = (unsigned *)(base + off);
  off += batch_err_bytes(ncases);
  b->d_sync = (lbm::GridSync *)(base + off);
  off += batch_sync_bytes();
  b->d_work = (lbm::WorkItem *)(base + off);
  b->work_cap = max_work(cases, ncases);
  *out = b;
  return LBM_OK;
}

lbm_handle *lbm_batch_case(lbm_batch *b, int i) { return (b && i >= 0 && i < b->n) ? b->h[i] : nullptr; }

lbm_status lbm_batch_set_active(lbm_batch *b, int i, int active) {
  if (!b || i < 0 || i >= b->n) return LBM_E_INVAL;
  b->active[i] = active ? 1 : 0;
  b->work_valid = false;
  return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch *b, int reps, int *chosen) {
  if (!b || reps < 1) return LBM_E_INVAL;
  cudaError_t e = b->upload_table();
  if (e != cudaSuccess) return b->cuda_fail(e, "lbm_batch_autotune table");
  // the persistent launch runs the sweep configurations only
  const int nv = b->persistent ? lbm::sweep_batched_count(b->nh) : lbm::batched_variant_count(b->nh);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return b->fail(LBM_E_CUDA, "cudaEventCreate");
  int best = 0;
  float best_ms = 0.f;
  for (int v = 0; v < nv && e == cudaSuccess; ++v) {
    int nw = 0;
    e = b->build_work(v, &nw);
    if (e != cudaSuccess || nw == 0) break;
    // parity 0 reads every case's current state and writes its spare buffers
    e = lbm::launch_batched_step(b->nh, b->form, b->d_cases, b->d_work, nw, 0, b->stream, v);
    if (e != cudaSuccess) break;
    cudaEventRecord(e0, b->stream);
    for (int r = 0; r < reps; ++r) lbm::launch_batched_step(b->nh, b->form, b->d_cases, b->d_work, nw, 0, b->stream, v);
    cudaEventRecord(e1, b->stream);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (v == 0 || ms < best_ms)) {
      best = v;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return b->cuda_fail(e, "lbm_batch_autotune");
  b->variant = best;
  b->work_valid = false;
  if (chosen) *chosen = best;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch *b, long long nsteps) {
  if (!b || nsteps < 0) return LBM_E_INVAL;
  if (nsteps == 0) return LBM_OK;
  cudaError_t e = cudaSuccess;
  if (!b->work_valid) {
    e = b->build_work(b->variant, &b->nwork);
    if (e != cudaSuccess) return b->cuda_fail(e, "lbm_batch_step work list");
    b->work_valid = true;
  }
  if (b->nwork == 0) return b->fail(LBM_E_STATE, "no active, initialised case");
  e = b->upload_table();
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, (size_t)b->n * sizeof(unsigned), b->stream);
  if (e != cudaSuccess) return b->cuda_fail(e, "lbm_batch_step table");
  if (b->persistent) return persistent_steps(b, nsteps);
  // graphs need a capturable stream: not the legacy or per-thread default stream
  const bool capturable = b->stream != nullptr && b->stream != cudaStreamLegacy && b->stream != cudaStreamPerThread;
  const long long graphs = capturable ? nsteps / kGraphSteps : 0;
  if (graphs > 0 && (!b->graph || b->graph_nwork != b->nwork || b->graph_variant != b->variant)) {
    // kernel attributes are set outside the capture
    e = lbm::launch_batched_step(b->nh, b->form, b->d_cases, b->d_work, 0, 0, b->stream, b->variant);
    if (e != cudaSuccess) return b->cuda_fail(e, "lbm_batch_step prepare");
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    for (int t = 0; t < kGraphSteps && e == cudaSuccess; ++t)
      e = lbm::launch_batched_step(b->nh, b->form, b->d_cases, b->d_work, b->nwork, t & 1, b->stream, b->variant);
    cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = ec;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return b->cuda_fail(e, "lbm_batch_step graph capture");
    b->graph_nwork = b->nwork;
    b->graph_variant = b->variant;
  }
  for (long long r = 0; r < graphs && e == cudaSuccess; ++r) e = cudaGraphLaunch(b->graph, b->stream);
  for (long long t = graphs * kGraphSteps; t < nsteps && e == cudaSuccess; ++t)
    e = lbm::launch_batched_step(b->nh, b->form, b->d_cases, b->d_work, b->nwork, (int)(t & 1), b->stream,
                                 b->variant);
  if (e != cudaSuccess) return b->cuda_fail(e, "lbm_batch_step launch");
  std::vector<unsigned> err(b->n);
  e = cudaMemcpyAsync(err.data(), b->d_err, err.size() * sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return b->cuda_fail(e, "lbm_batch_step");
  std::string diverged;
  for (int i = 0; i < b->n; ++i) {
    if (!b->active[i] || !b->h[i]->initialized) continue;
    if (nsteps & 1) b->h[i]->cur = 1 - b->h[i]->cur;
    b->h[i]->step += nsteps;
    if (err[i]) {
      diverged += " " + std::to_string(i);
      b->active[i] = 0;
      b->work_valid = false;
    }
  }
  if (!diverged.empty()) return b->fail(LBM_E_DIVERGED, "non-finite values in case(s)" + diverged + "; deactivated");
  return LBM_OK;
}

lbm_status lbm_batch_set_persistent(lbm_batch *b, int on, long long spin_limit) {
  if (!b || (on != 0 && on != 1) || spin_limit < 0) return LBM_E_INVAL;
  b->persistent = on != 0;
  b->spin_limit = spin_limit == 0 ? kDefaultSpinLimit : spin_limit;
  if (b->persistent && !lbm::batched_variant_is_sweep(b->nh, b->variant)) b->variant = 0;
  b->work_valid = false;
  return LBM_OK;
}

lbm_status lbm_batch_run(lbm_batch *b, const lbm_run_opts *opts, lbm_obs *out, int *outcome, long long *steps) {
  if (!b || !opts || !out || !outcome) return LBM_E_INVAL;
  if (opts->window < 1 || !(opts->rtol > 0) || opts->max_steps < opts->window || !(opts->top_margin >= 0))
    return b->fail(LBM_E_INVAL, "lbm_batch_run: need window >= 1, rtol > 0, max_steps >= window, top_margin >= 0");
  const int n = b->n;
  std::vector<std::vector<double>> ys(n);
  std::vector<double> top(n, 0.0);
  std::vector<long long> ran(n, 0);
  std::vector<char> running(n, 0);
  int left = 0;
  for (int i = 0; i < n; ++i) {
    outcome[i] = LBM_RUN_SKIPPED;
    if (steps) steps[i] = 0;
    if (!b->active[i] || !b->h[i]->initialized) continue;
    lbm_obs o{};
    lbm_status st = lbm_observables(b->h[i], &o);
    if (st != LBM_OK) return b->fail(st, std::string("lbm_batch_run: ") + lbm_last_error(b->h[i]));
    ys[i].push_back(o.centroid[1]);
    top[i] = (double)(b->h[i]->prm.ny - 1) - opts->top_margin * o.d_eq;
    running[i] = 1;
    ++left;
  }
  // window-averaged rise velocities of case i so far
  auto velocities = [&](int i) {
    std::vector<double> u;
    for (size_t k = 1; k < ys[i].size(); ++k) u.push_back((ys[i][k] - ys[i][k - 1]) / (double)opts->window);
    return u;
  };
  auto finish = [&](int i, int result, const lbm_obs &o) {
    const std::vector<double> u = velocities(i);
    const double U = u.empty() ? 0.0 : u.back();
    double raw[15];
    for (int q = 0; q < 15; ++q) raw[q] = o.raw[q];
    raw[10] = U * raw[6];
    lbm_postprocess(&b->h[i]->prm, raw, &out[i]);
    out[i].step = o.step;
    out[i].y_integrated = o.y_integrated;
    outcome[i] = result;
    if (steps) steps[i] = ran[i];
    running[i] = 0;
    b->active[i] = 0;
    b->work_valid = false;
    --left;
  };
  int tuned_for = -1;  // running cases when the launch configuration was last tuned
  while (left > 0) {
    if (left != tuned_for) {
      // the work list changed: pick the launch configuration for the cases
      // still running (timed without advancing them)
      lbm_status st = lbm_batch_autotune(b, 1, nullptr);
      if (st != LBM_OK) return st;
      tuned_for = left;
    }
    lbm_status st = lbm_batch_step(b, opts->window);
    if (st != LBM_OK && st != LBM_E_DIVERGED) return st;
    for (int i = 0; i < n; ++i) {
      if (!running[i]) continue;
      ran[i] += opts->window;
      lbm_obs o{};
      if (!b->active[i]) {  // deactivated by lbm_batch_step: non-finite values
        lbm_observables(b->h[i], &o);
        finish(i, LBM_RUN_DIVERGED, o);
        continue;
      }
      st = lbm_observables(b->h[i], &o);
      if (st != LBM_OK) return b->fail(st, std::string("lbm_batch_run: ") + lbm_last_error(b->h[i]));
      if (!std::isfinite(o.centroid[1]) || !std::isfinite(o.rise_velocity)) {
        finish(i, LBM_RUN_DIVERGED, o);
        continue;
      }
      ys[i].push_back(o.centroid[1]);
      const std::vector<double> u = velocities(i);
      const size_t m = u.size();
      bool steady = m >= 3;
      for (size_t j = 1; steady && j <= 2; ++j)
        steady = std::fabs(u[m - j] - u[m - j - 1]) < opts->rtol * std::fabs(u[m - j]);
      if (steady) finish(i, LBM_RUN_TERMINAL, o);
      else if (o.centroid[1] > top[i]) finish(i, LBM_RUN_TOP, o);
      else if (ran[i] >= opts->max_steps) finish(i, LBM_RUN_MAX_STEPS, o);
    }
  }
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b) { delete b; }

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->last_error.c_str() : "NULL batch"; }

}  // extern "C"
