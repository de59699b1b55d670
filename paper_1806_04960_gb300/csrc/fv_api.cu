// C ABI of libfv (declared in include/fv.h): handle, device memory, tables and
// the host side of one time step.  All device work is enqueued on the
// handle's stream; nothing here computes the scheme.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fv.h"
#include "fv_handle.cuh"
#include "fv_kernels.cuh"

using namespace fv;

namespace {

thread_local std::string g_err;

fv_status fail(fv_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

fv_status cuda_fail(cudaError_t e, const char* where) {
  return fail(FV_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define FV_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

}  // namespace

void fv::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

static void release(fv_handle* h) {
  if (!h) return;
  cudaFree(h->d_solid);
  cudaFree(h->d_Kref);
  cudaFree(h->d_Kcur);
  cudaFree(h->d_colsum);
  cudaFree(h->d_sc);
  cudaFree(h->d_rhoE);
  cudaFree(h->d_rhoE_f);
  cudaFree(h->d_rq);
  cudaFree(h->d_pq);
  cudaFree(h->d_rq_f);
  cudaFree(h->d_pq_f);
  cudaFree(h->d_q[0]);
  cudaFree(h->d_q[1]);
  cudaFree(h->d_stage);
  cudaFree(h->d_partial);
  cudaFree(h->d_mass);
  delete h;
}

// One step of the handle's scheme from d_q[a] to d_q[b] (no finalize).
static void launch_one_step(fv_handle* h, const StepParams& p, int a, int b) {
  Tables tb{h->d_rhoE, h->d_rhoE_f};
  QuarterTables tq{h->d_rq, h->d_pq, h->d_rq_f, h->d_pq_f};
  const bool orx = h->xface == FV_XFACE_OR;
  if (h->prec == FV_FP64) {
    StateF64 s{(const double*)h->d_q[a], (double*)h->d_q[b]};
    if (h->order == 1)
      launch_step_o1_f64(p, s, h->d_solid, h->d_Kcur, h->d_colsum, h->d_sc, tb, tq, h->stream, orx);
    else
      launch_step_f64(p, s, h->d_solid, h->d_Kcur, h->d_colsum, h->d_sc, tb, h->stream, orx,
                      h->tiling, h->strip_h);
  } else {
    StateF32 s{(const float*)h->d_q[a], (float*)h->d_q[b]};
    if (h->order == 1)
      launch_step_o1_f32(p, s, h->d_solid, h->d_Kref, h->d_Kcur, h->d_colsum, h->d_sc, tb, tq,
                         h->stream, orx);
    else
      launch_step_f32(p, s, h->d_solid, h->d_Kref, h->d_Kcur, h->d_colsum, h->d_sc, tb, h->stream,
                      orx, h->tiling, h->strip_h);
  }
}

extern "C" {

const char* fv_last_error(void) { return g_err.c_str(); }

const char* fv_version(void) { return "libfv 0.1 (sm_103a)"; }

fv_status fv_create(const fv_grid* grid, const fv_eos* eos, const fv_bc* bc, fv_prec prec,
                    void* cuda_stream, fv_handle** out) {
  if (!grid || !eos || !bc || !out) return fail(FV_EINVAL, "fv_create: null argument");
  if (grid->nx < 1 || grid->ny < 1) return fail(FV_EINVAL, "fv_create: nx, ny must be >= 1");
  if ((long long)grid->nx * grid->ny > 2147483647LL)
    return fail(FV_EINVAL, "fv_create: nx*ny exceeds 2^31-1");
  if (!(grid->dx > 0.0) || !(grid->dy > 0.0) || !std::isfinite(grid->dx) || !std::isfinite(grid->dy))
    return fail(FV_EINVAL, "fv_create: dx, dy must be finite and > 0");
  if (eos->gamma != 1.0) return fail(FV_EINVAL, "fv_create: only gamma = 1 is supported");
  if (!(eos->rho0 > 0.0) || !(eos->k0 > 0.0) || !(eos->g >= 0.0) || !(eos->eps_gas > 0.0) ||
      !(eos->eps_gas < 0.1))
    return fail(FV_EINVAL, "fv_create: need rho0 > 0, k0 > 0, g >= 0, 0 < eps_gas < 0.1");
  for (int s = 0; s < 4; ++s)
    if (bc->side[s] != FV_BC_WALL && bc->side[s] != FV_BC_TRANSMISSIVE)
      return fail(FV_EINVAL, "fv_create: side must be FV_BC_WALL or FV_BC_TRANSMISSIVE");
  if (prec != FV_FP64 && prec != FV_FP32_DEV) return fail(FV_EINVAL, "fv_create: bad precision");

  fv_handle* h = new (std::nothrow) fv_handle();
  if (!h) return fail(FV_ENOMEM, "fv_create: host allocation");
  h->grid = *grid;
  h->eos = *eos;
  for (int s = 0; s < 4; ++s) h->side[s] = bc->side[s];
  h->prec = prec;
  h->stream = (cudaStream_t)cuda_stream;
  h->ncell = (size_t)grid->nx * grid->ny;
  const size_t N = h->ncell;
  const int nx = grid->nx, ny = grid->ny;
  const size_t elem = prec == FV_FP64 ? sizeof(double) : sizeof(float);
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  h->mass_blocks = 1024;
  bool ok = alloc((void**)&h->d_solid, N) && alloc((void**)&h->d_Kref, nx * sizeof(int32_t)) &&
            alloc((void**)&h->d_Kcur, nx * sizeof(int32_t)) &&
            alloc((void**)&h->d_colsum, nx * sizeof(unsigned long long)) &&
            alloc((void**)&h->d_sc, sizeof(DevScalars)) &&
            alloc((void**)&h->d_rhoE, (4 * (size_t)ny + 1) * sizeof(double)) &&
            alloc((void**)&h->d_rhoE_f, (4 * (size_t)ny + 1) * sizeof(float)) &&
            alloc((void**)&h->d_rq, (8 * (size_t)ny + 1) * sizeof(double)) &&
            alloc((void**)&h->d_pq, (8 * (size_t)ny + 1) * sizeof(double)) &&
            alloc((void**)&h->d_rq_f, (8 * (size_t)ny + 1) * sizeof(float)) &&
            alloc((void**)&h->d_pq_f, (8 * (size_t)ny + 1) * sizeof(float)) &&
            alloc(&h->d_q[0], 4 * N * elem) && alloc(&h->d_q[1], 4 * N * elem) &&
            alloc((void**)&h->d_partial, h->mass_blocks * sizeof(double)) &&
            alloc((void**)&h->d_mass, sizeof(double));
  if (ok && prec == FV_FP32_DEV) ok = alloc((void**)&h->d_stage, 4 * N * sizeof(double));
  if (!ok) {
    release(h);
    return fail(FV_ENOMEM, "fv_create: device allocation failed");
  }
  // Solid mask.
  std::vector<uint8_t> solid(N, 0);
  if (bc->solid)
    for (size_t c = 0; c < N; ++c) solid[c] = bc->solid[c] ? 1 : 0;
  // Equilibrium table rho^E(h dy/2 above the level), h in [-2 ny, 2 ny] (Eq. (BNs_eq3)).
  std::vector<double> rt(4 * (size_t)ny + 1);
  std::vector<float> rtf(rt.size());
  const double kappa = eos->g * eos->rho0 / eos->k0;
  for (long h2 = -2L * ny; h2 <= 2L * ny; ++h2) {
    const double val = eos->rho0 * std::exp(-kappa * (0.5 * (double)h2) * grid->dy);
    rt[h2 + 2L * ny] = val;
    rtf[h2 + 2L * ny] = (float)val;
  }
  // the same at quarter-cell heights, with p^E = k0 (rho^E / rho0 - 1)
  std::vector<double> rq(8 * (size_t)ny + 1), pq(rq.size());
  std::vector<float> rqf(rq.size()), pqf(rq.size());
  for (long q4 = -4L * ny; q4 <= 4L * ny; ++q4) {
    const double r = eos->rho0 * std::exp(-kappa * (0.25 * (double)q4) * grid->dy);
    const size_t k = (size_t)(q4 + 4L * ny);
    rq[k] = r;
    pq[k] = eos->k0 * (r / eos->rho0 - 1.0);
    rqf[k] = (float)r;
    pqf[k] = (float)pq[k];
  }
  cudaError_t e = cudaMemcpyAsync(h->d_solid, solid.data(), N, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_rq, rq.data(), rq.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_pq, pq.data(), pq.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_rq_f, rqf.data(), rqf.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_pq_f, pqf.data(), pqf.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_rhoE, rt.data(), rt.size() * sizeof(double), cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_rhoE_f, rtf.data(), rtf.size() * sizeof(float),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_colsum, 0, nx * sizeof(unsigned long long), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_sc, 0, sizeof(DevScalars), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_Kcur, 0, nx * sizeof(int32_t), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_Kref, 0, nx * sizeof(int32_t), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    release(h);
    return cuda_fail(e, "fv_create");
  }
  *out = h;
  return FV_OK;
}

fv_status fv_set_state(fv_handle* h, const double* q, int on_device) {
  if (!h || !q) return fail(FV_EINVAL, "fv_set_state: null argument");
  const size_t N = h->ncell;
  const StepParams p = params_of(h, h->cfl);
  double* target = h->prec == FV_FP64 ? (double*)h->d_q[0] : h->d_stage;
  FV_CUDA(cudaMemcpyAsync(target, q, 4 * N * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  launch_zero_solid(p, target, h->d_solid, h->stream);
  FV_CUDA(cudaMemsetAsync(h->d_sc, 0, sizeof(DevScalars), h->stream));
  FV_CUDA(cudaMemsetAsync(h->d_colsum, 0, h->grid.nx * sizeof(unsigned long long), h->stream));
  launch_prologue_f64(p, target, h->d_solid, h->d_colsum, h->d_sc, h->stream);
  launch_finalize(p, h->d_Kref, h->d_Kcur, h->d_colsum, h->d_sc, 0, h->stream);
  FV_CUDA(cudaMemcpyAsync(h->d_Kref, h->d_Kcur, h->grid.nx * sizeof(int32_t),
                          cudaMemcpyDeviceToDevice, h->stream));
  if (h->prec == FV_FP32_DEV) {
    Tables tb{h->d_rhoE, h->d_rhoE_f};
    launch_to_dev(p, h->d_stage, h->d_solid, h->d_Kcur, tb, (float*)h->d_q[0], h->stream);
  }
  h->cur = 0;
  FV_CUDA(cudaGetLastError());
  DevScalars sc;
  FV_CUDA(cudaMemcpyAsync(&sc, h->d_sc, sizeof(sc), cudaMemcpyDeviceToHost, h->stream));
  FV_CUDA(cudaStreamSynchronize(h->stream));
  h->has_state = true;
  if (sc.status) {
    FV_CUDA(cudaMemsetAsync(h->d_sc, 0, sizeof(DevScalars), h->stream));
    h->has_state = false;
    return fail(FV_EINVAL, "fv_set_state: a fluid cell has alpha <= 0, alpha*rho <= 0 or a non-finite value");
  }
  return FV_OK;
}

fv_status fv_step(fv_handle* h, int32_t n, double cfl, double* t_out) {
  if (!h) return fail(FV_EINVAL, "fv_step: null handle");
  if (n < 0) return fail(FV_EINVAL, "fv_step: n must be >= 0");
  if (!(cfl > 0.0) || !(cfl <= 1.0)) return fail(FV_EINVAL, "fv_step: cfl must be in (0, 1]");
  if (!h->has_state) return fail(FV_EINVAL, "fv_step: no state (call fv_set_state first)");
  if (h->own_hi > 0 && n > 1)
    return fail(FV_EINVAL, "fv_step: a strip of a partitioned domain advances one step per call");
  h->cfl = cfl;
  const StepParams p = params_of(h, cfl);
  if (n > 0) launch_prepare(cfl, h->d_sc, h->stream);
  for (int32_t k = 0; k < n; ++k) {
    const int a = h->cur, b = 1 - h->cur;
    launch_one_step(h, p, a, b);
    launch_finalize(p, h->d_Kref, h->d_Kcur, h->d_colsum, h->d_sc, 1, h->stream);
    h->cur = b;
  }
  FV_CUDA(cudaGetLastError());
  if (t_out) {
    DevScalars sc;
    FV_CUDA(cudaMemcpyAsync(&sc, h->d_sc, sizeof(sc), cudaMemcpyDeviceToHost, h->stream));
    FV_CUDA(cudaStreamSynchronize(h->stream));
    *t_out = sc.t;
    if (sc.status) return fail(FV_ENONFINITE, "fv_step: a step produced a non-admissible state");
  }
  return FV_OK;
}

fv_status fv_step_timed(fv_handle* h, int32_t n, double cfl, double* kernel_ms,
                        double* total_ms) {
  if (!h) return fail(FV_EINVAL, "fv_step_timed: null handle");
  if (n < 0) return fail(FV_EINVAL, "fv_step_timed: n must be >= 0");
  if (!(cfl > 0.0) || !(cfl <= 1.0)) return fail(FV_EINVAL, "fv_step_timed: cfl must be in (0, 1]");
  if (!h->has_state) return fail(FV_EINVAL, "fv_step_timed: no state (call fv_set_state first)");
  if (h->own_hi > 0 && n > 1)
    return fail(FV_EINVAL, "fv_step_timed: a strip of a partitioned domain advances one step per call");
  h->cfl = cfl;
  const StepParams p = params_of(h, cfl);
  std::vector<cudaEvent_t> ev(2 * (size_t)n + 2);
  for (auto& e : ev) FV_CUDA(cudaEventCreate(&e));
  fv_status st = FV_OK;
  if (n > 0) launch_prepare(cfl, h->d_sc, h->stream);
  cudaError_t err = cudaEventRecord(ev[2 * n], h->stream);
  for (int32_t k = 0; k < n && err == cudaSuccess; ++k) {
    const int a = h->cur, b = 1 - h->cur;
    err = cudaEventRecord(ev[2 * k], h->stream);
    launch_one_step(h, p, a, b);
    if (err == cudaSuccess) err = cudaEventRecord(ev[2 * k + 1], h->stream);
    launch_finalize(p, h->d_Kref, h->d_Kcur, h->d_colsum, h->d_sc, 1, h->stream);
    h->cur = b;
  }
  if (err == cudaSuccess) err = cudaEventRecord(ev[2 * n + 1], h->stream);
  if (err == cudaSuccess) err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
  double ksum = 0.0, tot = 0.0;
  for (int32_t k = 0; k < n && err == cudaSuccess; ++k) {
    float ms = 0.f;
    err = cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]);
    ksum += ms;
  }
  if (err == cudaSuccess) {
    float ms = 0.f;
    err = cudaEventElapsedTime(&ms, ev[2 * n], ev[2 * n + 1]);
    tot = ms;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (err != cudaSuccess) return cuda_fail(err, "fv_step_timed");
  if (kernel_ms) *kernel_ms = ksum;
  if (total_ms) *total_ms = tot;
  DevScalars sc;
  FV_CUDA(cudaMemcpy(&sc, h->d_sc, sizeof(sc), cudaMemcpyDeviceToHost));
  if (sc.status) st = fail(FV_ENONFINITE, "fv_step_timed: a step produced a non-admissible state");
  return st;
}

fv_status fv_set_order(fv_handle* h, int32_t order) {
  if (!h) return fail(FV_EINVAL, "fv_set_order: null handle");
  if (order != 1 && order != 2) return fail(FV_EINVAL, "fv_set_order: order must be 1 or 2");
  h->order = order;
  return FV_OK;
}

fv_status fv_set_xface(fv_handle* h, int32_t solver) {
  if (!h) return fail(FV_EINVAL, "fv_set_xface: null handle");
  if (solver != FV_XFACE_GL && solver != FV_XFACE_OR)
    return fail(FV_EINVAL, "fv_set_xface: solver must be FV_XFACE_GL or FV_XFACE_OR");
  h->xface = solver;
  return FV_OK;
}

fv_status fv_set_tiling(fv_handle* h, int32_t tiling) {
  if (!h) return fail(FV_EINVAL, "fv_set_tiling: null handle");
  if (tiling != FV_TILING_AUTO && tiling != FV_TILING_TILE && tiling != FV_TILING_STRIP)
    return fail(FV_EINVAL, "fv_set_tiling: tiling must be FV_TILING_AUTO, _TILE or _STRIP");
  h->tiling = tiling;
  return FV_OK;
}

fv_status fv_set_strip_height(fv_handle* h, int32_t rows) {
  if (!h) return fail(FV_EINVAL, "fv_set_strip_height: null handle");
  if (rows < 0 || rows % 8 != 0)
    return fail(FV_EINVAL, "fv_set_strip_height: rows must be 0 or a positive multiple of 8");
  h->strip_h = rows;
  return FV_OK;
}

fv_status fv_tune(fv_handle* h, int32_t* rows_out) {
  if (!h) return fail(FV_EINVAL, "fv_tune: null handle");
  if (!h->has_state) return fail(FV_EINVAL, "fv_tune: no state (call fv_set_state first)");
  if (h->order != 2 || h->tiling == FV_TILING_TILE) {
    if (rows_out) *rows_out = h->strip_h;
    return FV_OK;  // nothing to tune: the step does not stage by strips
  }
  // Trial launches read the current state and write the other buffer, which
  // the next step overwrites; the accumulators they touch are put back.
  DevScalars saved;
  FV_CUDA(cudaMemcpyAsync(&saved, h->d_sc, sizeof(saved), cudaMemcpyDeviceToHost, h->stream));
  FV_CUDA(cudaStreamSynchronize(h->stream));
  const StepParams p = params_of(h, h->cfl > 0.0 ? h->cfl : 0.9);
  const int hmax = ((h->grid.ny + 7) / 8) * 8;
  static const int cand[] = {32, 48, 64, 96, 128, 160, 192, 256};
  const int keep = h->strip_h;
  int best = keep;
  float best_ms = 1e30f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  for (int c : cand) {
    if (err != cudaSuccess) break;
    if (c > hmax && c != cand[0]) continue;
    h->strip_h = c;
    const int a = h->cur, b = 1 - h->cur;
    launch_one_step(h, p, a, b);  // warm-up
    err = cudaEventRecord(e0, h->stream);
    for (int k = 0; k < 3 && err == cudaSuccess; ++k) launch_one_step(h, p, a, b);
    if (err == cudaSuccess) err = cudaEventRecord(e1, h->stream);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  h->strip_h = err == cudaSuccess ? best : keep;
  if (err == cudaSuccess) err = cudaMemsetAsync(h->d_colsum, 0, sizeof(unsigned long long) * h->grid.nx, h->stream);
  if (err == cudaSuccess) err = cudaMemcpyAsync(h->d_sc, &saved, sizeof(saved), cudaMemcpyHostToDevice, h->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
  if (err != cudaSuccess) return cuda_fail(err, "fv_tune");
  if (rows_out) *rows_out = h->strip_h;
  return FV_OK;
}

fv_status fv_get_state(fv_handle* h, double* q, int on_device) {
  if (!h || !q) return fail(FV_EINVAL, "fv_get_state: null argument");
  if (!h->has_state) return fail(FV_EINVAL, "fv_get_state: no state");
  const size_t N = h->ncell;
  const double* src = (const double*)h->d_q[h->cur];
  if (h->prec == FV_FP32_DEV) {
    const StepParams p = params_of(h, h->cfl);
    Tables tb{h->d_rhoE, h->d_rhoE_f};
    launch_from_dev(p, (const float*)h->d_q[h->cur], h->d_solid, h->d_Kref, tb, h->d_stage,
                    h->stream);
    FV_CUDA(cudaGetLastError());
    src = h->d_stage;
  }
  FV_CUDA(cudaMemcpyAsync(q, src, 4 * N * sizeof(double),
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  FV_CUDA(cudaStreamSynchronize(h->stream));
  return FV_OK;
}

fv_status fv_get_levels(fv_handle* h, int32_t* K) {
  if (!h || !K) return fail(FV_EINVAL, "fv_get_levels: null argument");
  FV_CUDA(cudaMemcpyAsync(K, h->d_Kcur, h->grid.nx * sizeof(int32_t), cudaMemcpyDeviceToHost,
                          h->stream));
  FV_CUDA(cudaStreamSynchronize(h->stream));
  return FV_OK;
}

fv_status fv_get_diag(fv_handle* h, fv_diag* d) {
  if (!h || !d) return fail(FV_EINVAL, "fv_get_diag: null argument");
  if (!h->has_state) return fail(FV_EINVAL, "fv_get_diag: no state");
  const StepParams p = params_of(h, h->cfl);
  const double* src = (const double*)h->d_q[h->cur];
  if (h->prec == FV_FP32_DEV) {
    Tables tb{h->d_rhoE, h->d_rhoE_f};
    launch_from_dev(p, (const float*)h->d_q[h->cur], h->d_solid, h->d_Kref, tb, h->d_stage,
                    h->stream);
    src = h->d_stage;
  }
  launch_mass(p, src, h->d_solid, h->d_partial, h->mass_blocks, h->d_mass, h->stream);
  FV_CUDA(cudaGetLastError());
  DevScalars sc;
  double mass = 0.0;
  FV_CUDA(cudaMemcpyAsync(&sc, h->d_sc, sizeof(sc), cudaMemcpyDeviceToHost, h->stream));
  FV_CUDA(cudaMemcpyAsync(&mass, h->d_mass, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  FV_CUDA(cudaStreamSynchronize(h->stream));
  d->t = sc.t;
  d->steps = sc.steps;
  d->dt_next = sc.rate_cur > 0.0 ? h->cfl / sc.rate_cur : 0.0;
  d->mass = mass;
  d->status = sc.status ? FV_ENONFINITE : FV_OK;
  return FV_OK;
}

void fv_destroy(fv_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  release(h);
}

}  // extern "C"
