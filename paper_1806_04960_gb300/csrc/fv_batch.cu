// Batched ensemble of independent domains (C ABI declared in include/fv.h).
//
// Every domain has its own grid, equation of state, boundaries, level
// detector, dt and time.  One step of the ensemble is one launch of
// batch_strip_kernel over the column strips of all domains (a persistent grid
// of the resident CTAs striding over them, or one CTA per strip, as
// fv_batch_tune measures fastest) followed by one per-domain finalize launch.
// n steps are captured once into a CUDA graph on an internal stream and
// replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "fv.h"
#include "fv_kernels.cuh"

using namespace fv;

namespace {

fv_status bfail(fv_status s, const std::string& m) {
  fv::set_last_error(m.c_str());
  return s;
}

#define BV_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return bfail(FV_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct fv_batch {
  int ndom = 0;
  fv_prec prec = FV_FP64;
  cudaStream_t user = nullptr;
  cudaStream_t inner = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<BatchDomainDesc> desc;
  std::vector<fv_grid> grids;
  std::vector<fv_eos> eos;
  unsigned char* pool = nullptr;  // all per-domain device buffers
  void* d_table = nullptr;
  int4* d_tiles = nullptr;
  int ntiles = 0;
  double* d_stage = nullptr;       // double staging for set/get (largest domain)
  double* d_partial = nullptr;
  double* d_mass = nullptr;
  int cur = 0;
  int strip_h = BATCH_STRIP_H;     // rows per strip of the work list
  int order = 0;                   // work order (batch_work)
  bool persistent = true;          // launch form of the step kernel
  std::vector<char> has_state;
  std::map<std::tuple<int, double, int>, cudaGraphExec_t> graphs;
};

static void batch_release(fv_batch* b) {
  if (!b) return;
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  cudaFree(b->pool);
  cudaFree(b->d_table);
  cudaFree(b->d_tiles);
  cudaFree(b->d_stage);
  cudaFree(b->d_partial);
  cudaFree(b->d_mass);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->inner) cudaStreamDestroy(b->inner);
  delete b;
}

// Work list of the batch kernel: every domain cut into strips of 32 columns x
// H rows (the last strip of a column shorter).  order 0: domain by domain;
// order 1: longest strips first (stable), which balances uneven domains in
// both launch forms (round-robin over a persistent grid; CTAs handed out by
// the block scheduler).
static std::vector<int4> batch_work(const std::vector<fv_grid>& grids, int H, int order) {
  std::vector<int4> w;
  for (int k = 0; k < (int)grids.size(); ++k) {
    const int sx = (grids[k].nx + 31) / 32, sy = (grids[k].ny + H - 1) / H;
    for (int j = 0; j < sy; ++j)
      for (int i = 0; i < sx; ++i) w.push_back(make_int4(k, i, j, H));
  }
  if (order == 1) {
    auto rows = [&](const int4& t) { return std::min(t.w, grids[t.x].ny - t.z * t.w); };
    std::stable_sort(w.begin(), w.end(), [&](const int4& a, const int4& b) { return rows(a) > rows(b); });
  }
  return w;
}

// Make (H, order, persistent) the batch's step launch: a new work list when H
// or the order changes; the cached step graphs are dropped on any change.
static fv_status batch_apply(fv_batch* b, int H, int order, bool persistent, const char* who) {
  if (H == b->strip_h && order == b->order && persistent == b->persistent) return FV_OK;
  if (H != b->strip_h || order != b->order) {
    const std::vector<int4> w = batch_work(b->grids, H, order);
    int4* d_new = nullptr;
    cudaError_t e = cudaMalloc((void**)&d_new, w.size() * sizeof(int4));
    if (e == cudaSuccess)
      e = cudaMemcpy(d_new, w.data(), w.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(d_new);
      return bfail(FV_ECUDA, std::string(who) + ": " + cudaGetErrorString(e));
    }
    cudaFree(b->d_tiles);
    b->d_tiles = d_new;
    b->ntiles = (int)w.size();
    b->strip_h = H;
    b->order = order;
  }
  b->persistent = persistent;
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
  return FV_OK;
}

static StepParams bparams(const fv_grid& g, const fv_eos& e, const int32_t side[4], double cfl) {
  StepParams p;
  p.nx = g.nx;
  p.ny = g.ny;
  p.dx = g.dx;
  p.dy = g.dy;
  p.rho0 = e.rho0;
  p.k0 = e.k0;
  p.g = e.g;
  p.eps = e.eps_gas;
  p.c2 = e.k0 / e.rho0;
  p.c = std::sqrt(p.c2);
  p.kappa = e.g * e.rho0 / e.k0;
  for (int s = 0; s < 4; ++s) p.side[s] = side[s];
  p.cfl = cfl;
  return p;
}

extern "C" {

fv_status fv_batch_create(int32_t ndom, const fv_grid* grids, const fv_eos* eos, const fv_bc* bcs,
                          fv_prec prec, void* cuda_stream, fv_batch** out) {
  if (ndom < 1 || !grids || !eos || !bcs || !out) return bfail(FV_EINVAL, "fv_batch_create: bad arguments");
  if (prec != FV_FP64 && prec != FV_FP32_DEV) return bfail(FV_EINVAL, "fv_batch_create: bad precision");
  for (int k = 0; k < ndom; ++k) {
    const fv_grid& g = grids[k];
    const fv_eos& e = eos[k];
    if (g.nx < 1 || g.ny < 1 || (long long)g.nx * g.ny > 2147483647LL || !(g.dx > 0.0) || !(g.dy > 0.0))
      return bfail(FV_EINVAL, "fv_batch_create: bad grid of domain " + std::to_string(k));
    if (e.gamma != 1.0 || !(e.rho0 > 0.0) || !(e.k0 > 0.0) || !(e.g >= 0.0) || !(e.eps_gas > 0.0) ||
        !(e.eps_gas < 0.1))
      return bfail(FV_EINVAL, "fv_batch_create: bad equation of state of domain " + std::to_string(k));
    for (int s = 0; s < 4; ++s)
      if (bcs[k].side[s] != FV_BC_WALL && bcs[k].side[s] != FV_BC_TRANSMISSIVE)
        return bfail(FV_EINVAL, "fv_batch_create: bad boundary of domain " + std::to_string(k));
  }
  fv_batch* b = new (std::nothrow) fv_batch();
  if (!b) return bfail(FV_ENOMEM, "fv_batch_create: host allocation");
  b->ndom = ndom;
  b->prec = prec;
  b->user = (cudaStream_t)cuda_stream;
  b->grids.assign(grids, grids + ndom);
  b->eos.assign(eos, eos + ndom);
  b->has_state.assign(ndom, 0);
  const bool f64 = prec == FV_FP64;
  const size_t elem = f64 ? sizeof(double) : sizeof(float);
  // one pool for every domain's buffers
  std::vector<size_t> off(ndom);
  size_t total = 0, maxN = 0;
  for (int k = 0; k < ndom; ++k) {
    const size_t N = (size_t)grids[k].nx * grids[k].ny, nx = grids[k].nx, ny = grids[k].ny;
    maxN = N > maxN ? N : maxN;
    off[k] = total;
    total += 2 * up256(4 * N * elem) + up256(N) + 2 * up256(nx * 4) + up256(nx * 8) +
             up256(sizeof(DevScalars)) + up256((4 * ny + 1) * 8) + up256((4 * ny + 1) * 4);
  }
  cudaError_t e = cudaMalloc((void**)&b->pool, total);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_table, batch_table_bytes(ndom, f64));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_stage, 4 * maxN * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_partial, 1024 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_mass, sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->inner, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_release(b);
    return bfail(FV_ENOMEM, std::string("fv_batch_create: ") + cudaGetErrorString(e));
  }
  batch_grid_size(f64);  // kernel attributes and occupancy, outside any capture
  std::vector<int4> tiles;
  b->desc.resize(ndom);
  for (int k = 0; k < ndom; ++k) {
    const fv_grid& g = grids[k];
    const size_t N = (size_t)g.nx * g.ny, nx = g.nx, ny = g.ny;
    unsigned char* p = b->pool + off[k];
    BatchDomainDesc& d = b->desc[k];
    d.p = bparams(g, eos[k], bcs[k].side, 0.9);
    d.q[0] = p; p += up256(4 * N * elem);
    d.q[1] = p; p += up256(4 * N * elem);
    unsigned char* solid = p; p += up256(N);
    d.solid = solid;
    d.Kref = (int32_t*)p; p += up256(nx * 4);
    d.Kcur = (int32_t*)p; p += up256(nx * 4);
    d.colsum = (unsigned long long*)p; p += up256(nx * 8);
    d.sc = (DevScalars*)p; p += up256(sizeof(DevScalars));
    double* rt = (double*)p; p += up256((4 * ny + 1) * 8);
    float* rtf = (float*)p;
    d.rhoE_d = rt;
    d.rhoE_f = rtf;
    std::vector<uint8_t> hs(N, 0);
    if (bcs[k].solid)
      for (size_t c = 0; c < N; ++c) hs[c] = bcs[k].solid[c] ? 1 : 0;
    std::vector<double> ht(4 * ny + 1);
    std::vector<float> hf(4 * ny + 1);
    const double kappa = eos[k].g * eos[k].rho0 / eos[k].k0;
    for (long h2 = -2L * (long)ny; h2 <= 2L * (long)ny; ++h2) {
      const double val = eos[k].rho0 * std::exp(-kappa * (0.5 * (double)h2) * g.dy);
      ht[h2 + 2L * ny] = val;
      hf[h2 + 2L * ny] = (float)val;
    }
    e = cudaMemcpy(solid, hs.data(), N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(rt, ht.data(), ht.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(rtf, hf.data(), hf.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d.colsum, 0, nx * 8);
    if (e == cudaSuccess) e = cudaMemset(d.sc, 0, sizeof(DevScalars));
    if (e == cudaSuccess) e = cudaMemset(d.Kref, 0, nx * 4);
    if (e == cudaSuccess) e = cudaMemset(d.Kcur, 0, nx * 4);
    if (e == cudaSuccess) e = cudaMemset(d.q[0], 0, 4 * N * elem);
    if (e == cudaSuccess) e = cudaMemset(d.q[1], 0, 4 * N * elem);
    if (e != cudaSuccess) {
      batch_release(b);
      return bfail(FV_ECUDA, std::string("fv_batch_create: ") + cudaGetErrorString(e));
    }
  }
  tiles = batch_work(b->grids, b->strip_h, b->order);
  std::vector<unsigned char> table(batch_table_bytes(ndom, f64));
  batch_fill_table(b->desc.data(), ndom, f64, table.data());
  b->ntiles = (int)tiles.size();
  e = cudaMemcpy(b->d_table, table.data(), table.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_tiles, tiles.size() * sizeof(int4));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    batch_release(b);
    return bfail(FV_ECUDA, std::string("fv_batch_create: ") + cudaGetErrorString(e));
  }
  *out = b;
  return FV_OK;
}

fv_status fv_batch_set_state(fv_batch* b, int32_t dom, const double* q, int on_device) {
  if (!b || !q || dom < 0 || dom >= b->ndom) return bfail(FV_EINVAL, "fv_batch_set_state: bad arguments");
  const BatchDomainDesc& d = b->desc[dom];
  const size_t N = (size_t)d.p.nx * d.p.ny;
  const StepParams& p = d.p;
  const bool f64 = b->prec == FV_FP64;
  double* target = f64 ? (double*)d.q[b->cur] : b->d_stage;
  cudaStream_t st = b->inner;
  BV_CUDA(cudaEventRecord(b->ev_in, b->user));
  BV_CUDA(cudaStreamWaitEvent(st, b->ev_in, 0));
  BV_CUDA(cudaMemcpyAsync(target, q, 4 * N * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  launch_zero_solid(p, target, d.solid, st);
  BV_CUDA(cudaMemsetAsync(d.sc, 0, sizeof(DevScalars), st));
  BV_CUDA(cudaMemsetAsync(d.colsum, 0, p.nx * sizeof(unsigned long long), st));
  launch_prologue_f64(p, target, d.solid, d.colsum, d.sc, st);
  launch_finalize(p, d.Kref, d.Kcur, d.colsum, d.sc, 0, st);
  BV_CUDA(cudaMemcpyAsync(d.Kref, d.Kcur, p.nx * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  if (!f64) {
    Tables tb{d.rhoE_d, d.rhoE_f};
    launch_to_dev(p, b->d_stage, d.solid, d.Kcur, tb, (float*)d.q[b->cur], st);
  }
  BV_CUDA(cudaGetLastError());
  DevScalars sc;
  BV_CUDA(cudaMemcpyAsync(&sc, d.sc, sizeof(sc), cudaMemcpyDeviceToHost, st));
  BV_CUDA(cudaStreamSynchronize(st));
  if (sc.status) {
    BV_CUDA(cudaMemset(d.sc, 0, sizeof(DevScalars)));
    b->has_state[dom] = 0;
    return bfail(FV_EINVAL, "fv_batch_set_state: non-admissible fluid cell in domain " + std::to_string(dom));
  }
  b->has_state[dom] = 1;
  return FV_OK;
}

static fv_status batch_run(fv_batch* b, int32_t n, double cfl, double* total_ms) {
  if (!b) return bfail(FV_EINVAL, "fv_batch_step: null batch");
  if (n < 0) return bfail(FV_EINVAL, "fv_batch_step: n must be >= 0");
  if (!(cfl > 0.0) || !(cfl <= 1.0)) return bfail(FV_EINVAL, "fv_batch_step: cfl must be in (0, 1]");
  for (int k = 0; k < b->ndom; ++k)
    if (!b->has_state[k]) return bfail(FV_EINVAL, "fv_batch_step: domain " + std::to_string(k) + " has no state");
  if (n == 0) return FV_OK;
  const bool f64 = b->prec == FV_FP64;
  const auto key = std::make_tuple((int)n, cfl, b->cur);
  cudaGraphExec_t exec = nullptr;
  auto it = b->graphs.find(key);
  if (it != b->graphs.end()) {
    exec = it->second;
  } else {
    cudaGraph_t graph = nullptr;
    BV_CUDA(cudaStreamBeginCapture(b->inner, cudaStreamCaptureModeThreadLocal));
    launch_batch_prepare(f64, b->d_table, b->ndom, cfl, b->inner);
    int par = b->cur;
    for (int32_t k = 0; k < n; ++k) {
      launch_batch_step(f64, b->d_table, b->d_tiles, b->ntiles, par, b->persistent, b->inner);
      launch_batch_finalize(f64, b->d_table, b->ndom, cfl, 1, b->inner);
      par ^= 1;
    }
    cudaError_t e = cudaStreamEndCapture(b->inner, &graph);
    if (e != cudaSuccess) return bfail(FV_ECUDA, std::string("fv_batch_step: capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(FV_ECUDA, std::string("fv_batch_step: instantiate: ") + cudaGetErrorString(e));
    if (b->graphs.size() > 16) {
      for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
      b->graphs.clear();
    }
    b->graphs[key] = exec;
  }
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (total_ms) {
    BV_CUDA(cudaEventCreate(&t0));
    BV_CUDA(cudaEventCreate(&t1));
  }
  BV_CUDA(cudaEventRecord(b->ev_in, b->user));
  BV_CUDA(cudaStreamWaitEvent(b->inner, b->ev_in, 0));
  if (total_ms) BV_CUDA(cudaEventRecord(t0, b->inner));
  BV_CUDA(cudaGraphLaunch(exec, b->inner));
  if (total_ms) BV_CUDA(cudaEventRecord(t1, b->inner));
  BV_CUDA(cudaEventRecord(b->ev_out, b->inner));
  BV_CUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
  b->cur ^= (n & 1);
  if (total_ms) {
    BV_CUDA(cudaEventSynchronize(t1));
    float ms = 0.f;
    BV_CUDA(cudaEventElapsedTime(&ms, t0, t1));
    *total_ms = ms;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
  }
  return FV_OK;
}

fv_status fv_batch_step(fv_batch* b, int32_t n, double cfl) { return batch_run(b, n, cfl, nullptr); }

fv_status fv_batch_step_timed(fv_batch* b, int32_t n, double cfl, double* total_ms) {
  if (!total_ms) return bfail(FV_EINVAL, "fv_batch_step_timed: null total_ms");
  return batch_run(b, n, cfl, total_ms);
}

fv_status fv_batch_set_launch(fv_batch* b, int32_t rows, int32_t order, int32_t persistent) {
  if (!b) return bfail(FV_EINVAL, "fv_batch_set_launch: null batch");
  if (rows < 8 || rows % 8 != 0 || rows > (1 << 20) || (order != 0 && order != 1) ||
      (persistent != 0 && persistent != 1))
    return bfail(FV_EINVAL, "fv_batch_set_launch: rows a positive multiple of 8, order and "
                            "persistent 0 or 1");
  return batch_apply(b, rows, order, persistent == 1, "fv_batch_set_launch");
}

fv_status fv_batch_tune(fv_batch* b, double cfl, int32_t* rows_out, int32_t* order_out,
                        int32_t* persistent_out) {
  if (!b) return bfail(FV_EINVAL, "fv_batch_tune: null batch");
  if (!(cfl > 0.0) || !(cfl <= 1.0)) return bfail(FV_EINVAL, "fv_batch_tune: cfl must be in (0, 1]");
  for (int k = 0; k < b->ndom; ++k)
    if (!b->has_state[k]) return bfail(FV_EINVAL, "fv_batch_tune: domain " + std::to_string(k) + " has no state");
  const bool f64 = b->prec == FV_FP64;
  cudaStream_t st = b->inner;
  BV_CUDA(cudaEventRecord(b->ev_in, b->user));
  BV_CUDA(cudaStreamWaitEvent(st, b->ev_in, 0));
  // the trial launches accumulate into each domain's scalars and column sums:
  // keep the scalars, zero the sums afterwards (they are zero between steps)
  std::vector<DevScalars> saved(b->ndom);
  for (int k = 0; k < b->ndom; ++k)
    BV_CUDA(cudaMemcpyAsync(&saved[k], b->desc[k].sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st));
  BV_CUDA(cudaStreamSynchronize(st));
  const int cand_h[] = {32, 48, 64, 96, 128, 160, 192, 256};
  size_t most = 0;
  for (int H : cand_h) most = std::max(most, batch_work(b->grids, H, 0).size());
  int4* d_try = nullptr;
  BV_CUDA(cudaMalloc((void**)&d_try, most * sizeof(int4)));
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best = 3.4e38f;
  int best_h = b->strip_h, best_o = b->order;
  bool best_p = b->persistent;
  launch_batch_prepare(f64, b->d_table, b->ndom, cfl, st);
  for (int H : cand_h) {
    for (int order = 0; order < 2 && e == cudaSuccess; ++order) {
      const std::vector<int4> w = batch_work(b->grids, H, order);
      e = cudaMemcpyAsync(d_try, w.data(), w.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
      for (int form = 0; form < 2 && e == cudaSuccess; ++form) {
        const bool pers = form == 0;
        launch_batch_step(f64, b->d_table, d_try, (int)w.size(), b->cur, pers, st);   // warm-up
        e = cudaEventRecord(t0, st);
        for (int r = 0; r < 3 && e == cudaSuccess; ++r)
          launch_batch_step(f64, b->d_table, d_try, (int)w.size(), b->cur, pers, st);
        if (e == cudaSuccess) e = cudaEventRecord(t1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && ms < best) {
          best = ms;
          best_h = H;
          best_o = order;
          best_p = pers;
        }
      }
    }
  }
  // restore: scalars as they were, column sums zero
  for (int k = 0; k < b->ndom && e == cudaSuccess; ++k) {
    e = cudaMemcpyAsync(b->desc[k].sc, &saved[k], sizeof(DevScalars), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(b->desc[k].colsum, 0, b->desc[k].p.nx * sizeof(unsigned long long), st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(d_try);
  if (e != cudaSuccess) return bfail(FV_ECUDA, std::string("fv_batch_tune: ") + cudaGetErrorString(e));
  const fv_status st_apply = batch_apply(b, best_h, best_o, best_p, "fv_batch_tune");
  if (st_apply != FV_OK) return st_apply;
  if (rows_out) *rows_out = b->strip_h;
  if (order_out) *order_out = b->order;
  if (persistent_out) *persistent_out = b->persistent ? 1 : 0;
  BV_CUDA(cudaEventRecord(b->ev_out, st));
  BV_CUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
  return FV_OK;
}

fv_status fv_batch_get_state(fv_batch* b, int32_t dom, double* q, int on_device) {
  if (!b || !q || dom < 0 || dom >= b->ndom) return bfail(FV_EINVAL, "fv_batch_get_state: bad arguments");
  if (!b->has_state[dom]) return bfail(FV_EINVAL, "fv_batch_get_state: no state");
  const BatchDomainDesc& d = b->desc[dom];
  const size_t N = (size_t)d.p.nx * d.p.ny;
  cudaStream_t st = b->inner;
  BV_CUDA(cudaEventRecord(b->ev_in, b->user));
  BV_CUDA(cudaStreamWaitEvent(st, b->ev_in, 0));
  const double* src = (const double*)d.q[b->cur];
  if (b->prec == FV_FP32_DEV) {
    Tables tb{d.rhoE_d, d.rhoE_f};
    launch_from_dev(d.p, (const float*)d.q[b->cur], d.solid, d.Kref, tb, b->d_stage, st);
    src = b->d_stage;
  }
  BV_CUDA(cudaMemcpyAsync(q, src, 4 * N * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  BV_CUDA(cudaStreamSynchronize(st));
  return FV_OK;
}

fv_status fv_batch_get_diag(fv_batch* b, int32_t dom, fv_diag* out) {
  if (!b || !out || dom < 0 || dom >= b->ndom) return bfail(FV_EINVAL, "fv_batch_get_diag: bad arguments");
  if (!b->has_state[dom]) return bfail(FV_EINVAL, "fv_batch_get_diag: no state");
  const BatchDomainDesc& d = b->desc[dom];
  cudaStream_t st = b->inner;
  BV_CUDA(cudaEventRecord(b->ev_in, b->user));
  BV_CUDA(cudaStreamWaitEvent(st, b->ev_in, 0));
  const double* src = (const double*)d.q[b->cur];
  if (b->prec == FV_FP32_DEV) {
    Tables tb{d.rhoE_d, d.rhoE_f};
    launch_from_dev(d.p, (const float*)d.q[b->cur], d.solid, d.Kref, tb, b->d_stage, st);
    src = b->d_stage;
  }
  launch_mass(d.p, src, d.solid, b->d_partial, 1024, b->d_mass, st);
  BV_CUDA(cudaGetLastError());
  DevScalars sc;
  double mass = 0.0;
  BV_CUDA(cudaMemcpyAsync(&sc, d.sc, sizeof(sc), cudaMemcpyDeviceToHost, st));
  BV_CUDA(cudaMemcpyAsync(&mass, b->d_mass, sizeof(double), cudaMemcpyDeviceToHost, st));
  BV_CUDA(cudaStreamSynchronize(st));
  out->t = sc.t;
  out->steps = sc.steps;
  out->dt_next = sc.dt_cur;
  out->mass = mass;
  out->status = sc.status ? FV_ENONFINITE : FV_OK;
  return FV_OK;
}

int32_t fv_batch_size(const fv_batch* b) { return b ? b->ndom : 0; }

void fv_batch_destroy(fv_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->inner);
  batch_release(b);
}

}  // extern "C"
