// Per-precision constants of one step, built on the host from StepParams, and
// the equilibrium-density table lookup.  Internal header shared by the step
// and adjoint kernels.
#pragma once

#include <cmath>

#include "fv_kernels.cuh"
#include "fv_model.cuh"

namespace fv {

// Per-precision constants, built once on the host.
template <typename T>
struct KConsts {
  Phys<T> P;
  ReconConsts<T> R;  // half_dt is filled in the kernel
  T dx, dy, eps, inv_dx, inv_dy, inv_1meps;
};

template <typename T>
inline KConsts<T> make_consts(const StepParams& p) {
  KConsts<T> k;
  k.P.c = (T)p.c;
  k.P.c2 = (T)p.c2;
  k.P.inv_c = (T)(1.0 / p.c);
  k.P.rho0 = (T)p.rho0;
  k.P.k0 = (T)p.k0;
  k.P.g = (T)p.g;
  k.P.kappa = (T)p.kappa;
  k.R.half_dx = (T)(0.5 * p.dx);
  k.R.half_dy = (T)(0.5 * p.dy);
  k.R.inv_2dx = (T)(1.0 / (2.0 * p.dx));
  k.R.inv_2dy = (T)(1.0 / (2.0 * p.dy));
  k.R.ten_eps = (T)(10.0 * p.eps);
  k.R.half_dt = (T)0;
  // limiter ramp scales: 2^-20 rho0, 2^-10 rho0 c (momenta), 2^-20 (alpha)
  const double eta[4] = {std::ldexp(p.rho0, -20), std::ldexp(p.rho0 * p.c, -10),
                         std::ldexp(p.rho0 * p.c, -10), std::ldexp(1.0, -20)};
  for (int v = 0; v < 4; ++v) {
    k.R.eta[v] = (T)eta[v];
    k.R.inv_eta[v] = (T)(1.0 / eta[v]);
  }
  k.dx = (T)p.dx;
  k.dy = (T)p.dy;
  k.eps = (T)p.eps;
  k.inv_dx = (T)(1.0 / p.dx);
  k.inv_dy = (T)(1.0 / p.dy);
  k.inv_1meps = (T)(1.0 / (1.0 - p.eps));
  return k;
}

template <typename T>
__host__ __device__ __forceinline__ T tab(const T* rt, int h, int ny) {
  return rt[h + 2 * ny];
}

}  // namespace fv
