// Per-precision constants of one step, built on the host from StepParams, the
// equilibrium-density table lookup and the epilogue every step kernel ends
// with.  Internal header shared by the step, first-order and adjoint kernels.
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

// Product rounded on its own (never fused into an FMA): a difference of two
// such products of equal factors is then exactly zero, which keeps equal
// neighbouring rest states exactly balanced when both products are formed in
// the same expression.
template <typename T>
__device__ __forceinline__ T mul_rn(T a, T b);
template <>
__device__ __forceinline__ float mul_rn<float>(float a, float b) {
  return __fmul_rn(a, b);
}
template <>
__device__ __forceinline__ double mul_rn<double>(double a, double b) {
  return __dmul_rn(a, b);
}

// Detected level K = round(column sum) of Eq. (Free_surf_detector) from the
// 2^-32 fixed-point sum, half away from zero; at most ny (a column of ny cells),
// so that every table lookup stays in range whatever the state.
__device__ __forceinline__ int32_t level_of(unsigned long long colsum, int ny) {
  const unsigned long long k = (colsum + (1ull << 31)) >> 32;
  return k > (unsigned long long)ny ? ny : (int32_t)k;
}

// FP64 signal rate (reading R-cfl) and detector weight of Eq.
// (Free_surf_detector) on the 2^-32 fixed-point scale of one fluid cell with
// state (m, mu, mv, a); bad = not admissible.  The same function of the
// state for the prologue of a state that is set and for the epilogue of a
// step, so that dt does not depend on where it was formed.  Reciprocals and
// products in place of divisions (the FP64 pipe bounds the step kernels):
// the rate is within an ulp or two of (|u| + c)/dx + (|v| + c)/dy.  inv_dx,
// inv_dy, inv_1meps: 1/dx, 1/dy, 1/(1 - eps), each rounded once.
__device__ __forceinline__ void rate_weight_f64(const StepParams& p, double inv_dx, double inv_dy,
                                                double inv_1meps, double m, double mu, double mv,
                                                double a, double& rate, unsigned long long& w,
                                                bool& bad) {
  const double r = rcp(m);
  const double u = mu * r, v = mv * r;
  bad = !gtz(m) || !gtz(a) || !isfinite(u) || !isfinite(v) || !isfinite(a);
  rate = (tabs(u) + p.c) * inv_dx + (tabs(v) + p.c) * inv_dy;
  double x = (a - p.eps) * inv_1meps;
  x = x >= 0.0 ? (x > 1.0 ? 1.0 : x) : 0.0;  // NaN -> 0 (the status flag reports it)
  w = (unsigned long long)__double2ll_rn(x * 4294967296.0);
}

// Per-cell epilogue of a step on the new state qn (stored form) with full
// alpha rho m_full: admissibility, the signal rate of the next dt (reading
// R-cfl) and the detector weight of Eq. (Free_surf_detector) on the common
// 2^-32 fixed-point scale.  own = false (a halo column of a partitioned
// domain, whose new values are replaced by its owner's): the cell adds no rate
// and no status.
template <typename T, bool DEV>
__device__ __forceinline__ void cell_epilogue(const StepParams& p, const KConsts<T>& kc,
                                              const T qn[4], T m_full, T& my_rate,
                                              unsigned long long& my_w, bool& bad,
                                              bool own = true) {
  if (DEV) {
    // float path: in float; the max is taken in double by the reduction
    const T r = rcp(m_full);
    const T u = qn[1] * r, v = qn[2] * r;
    if (own && (!(m_full > T(0)) || !(qn[3] > T(0)) || !isfinite(u) || !isfinite(v) ||
                !isfinite(qn[3])))
      bad = true;
    const T rt_ = (tabs(u) + kc.P.c) * kc.inv_dx + (tabs(v) + kc.P.c) * kc.inv_dy;
    my_rate = own && rt_ >= T(0) ? rt_ : T(0);
    T w = (qn[3] - kc.eps) * kc.inv_1meps;
    w = w >= T(0) ? (w > T(1) ? T(1) : w) : T(0);  // NaN -> 0 (the status flag reports it)
    // 2^-24 resolution in float, placed on the common 2^-32 fixed-point scale
    my_w = (unsigned long long)__float2uint_rn((float)w * 16777216.0f) << 8;
  } else {
    double rd;
    bool b = false;
    rate_weight_f64(p, (double)kc.inv_dx, (double)kc.inv_dy, (double)kc.inv_1meps, (double)m_full,
                    (double)qn[1], (double)qn[2], (double)qn[3], rd, my_w, b);
    if (own && b) bad = true;
    my_rate = own && rd >= 0.0 ? (T)rd : T(0);
  }
}

// Block part of the epilogue for a CTA of TX x TY threads (called by all of
// them): the status flag, one 64-bit atomicAdd per column of the tile into the
// detector's column sums and one atomicMax of the tile's largest rate.  col
// and wmax are shared scratch of TY x TX and TX*TY/32 entries.
template <typename T, int TX, int TY>
__device__ __forceinline__ void block_epilogue(T my_rate, unsigned long long my_w, bool bad,
                                               bool inside, int gi, unsigned long long (*col)[TX],
                                               double* wmax, unsigned long long* colsum,
                                               DevScalars* sc) {
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  if (bad) atomicOr(&sc->status, 1);
  col[ty][tx] = my_w;
  // rate max (in T; one double per warp)
  T r_t = my_rate;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r_t = fmax(r_t, __shfl_xor_sync(0xffffffffu, r_t, o));
  if ((tid & 31) == 0) wmax[tid >> 5] = (double)r_t;
  __syncthreads();
  if (ty == 0 && inside) {
    unsigned long long s = 0;
#pragma unroll
    for (int r = 0; r < TY; ++r) s += col[r][tx];
    if (s) atomicAdd(&colsum[gi], s);
  }
  if (tid == 0) {
    double mrate = 0.0;
#pragma unroll
    for (int k = 0; k < TX * TY / 32; ++k) mrate = fmax(mrate, wmax[k]);
    if (mrate > 0.0) atomicMax(&sc->rate_acc, (unsigned long long)__double_as_longlong(mrate));
  }
}

}  // namespace fv
