// Handle of libfv (opaque to callers: include/fv.h declares it incomplete).
// Internal header shared by the C ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "fv.h"
#include "fv_kernels.cuh"

struct fv_handle {
  fv_grid grid;
  fv_eos eos;
  int side[4];
  fv_prec prec;
  cudaStream_t stream;
  size_t ncell;
  uint8_t* d_solid = nullptr;
  int32_t* d_Kref = nullptr;
  int32_t* d_Kcur = nullptr;
  unsigned long long* d_colsum = nullptr;
  fv::DevScalars* d_sc = nullptr;
  double* d_rhoE = nullptr;
  float* d_rhoE_f = nullptr;
  double* d_rq = nullptr;       // quarter-cell rho^E and p^E (first-order y faces)
  double* d_pq = nullptr;
  float* d_rq_f = nullptr;
  float* d_pq_f = nullptr;
  int order = 2;                // scheme of fv_step: 2 (Eq. (Scheme)) or 1 (Sections 3.2-3.3)
  int xface = FV_XFACE_GL;      // x-face viscosity (fv_set_xface)
  int tiling = FV_TILING_AUTO;  // step-kernel staging (fv_set_tiling)
  int strip_h = 0;              // strip height in rows, 0 = heuristic (fv_set_strip_height, fv_tune)
  void* d_q[2] = {nullptr, nullptr};
  int cur = 0;
  double* d_stage = nullptr;    // FP32 path: double staging buffer
  double* d_partial = nullptr;  // mass partials
  double* d_mass = nullptr;
  int mass_blocks = 0;
  bool has_state = false;
  double cfl = 0.9;
  int own_lo = 0;               // owned columns of a partitioned domain (fv_set_partition)
  int own_hi = 0;               // 0 = the whole grid
};

inline fv::StepParams params_of(const fv_handle* h, double cfl) {
  fv::StepParams p;
  p.nx = h->grid.nx;
  p.ny = h->grid.ny;
  p.dx = h->grid.dx;
  p.dy = h->grid.dy;
  p.rho0 = h->eos.rho0;
  p.k0 = h->eos.k0;
  p.g = h->eos.g;
  p.eps = h->eos.eps_gas;
  p.c2 = h->eos.k0 / h->eos.rho0;
  p.c = std::sqrt(p.c2);
  p.kappa = h->eos.g * h->eos.rho0 / h->eos.k0;
  for (int s = 0; s < 4; ++s) p.side[s] = h->side[s];
  p.cfl = cfl;
  if (h->own_hi > 0) {
    p.own_lo = h->own_lo;
    p.own_hi = h->own_hi;
  }
  return p;
}

