// Device model of the reduced Baer-Nunziato system and the two face solvers of
// the well-balanced path-conservative scheme (Gaburro, Castro, Dumbser,
// Section 3).  Templated on the arithmetic type T (double or float).
//
// State q = (m, mu, mv, a) = (alpha rho, alpha rho u, alpha rho v, alpha); the
// gravity potential y is static and never enters a difference (both states of
// a face sit at the same height at second order).  Tait law with gamma = 1
// (Eq. (TaitLaw)): alpha p = c2 (m - rho0 a), c2 = k0/rho0 constant, so that
// rho c^2 - p = k0 and k0 / c2 = rho0 in the printed eigenvectors.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <type_traits>

namespace fv {

template <typename T>
struct Phys {
  T c, c2, inv_c, rho0, k0, g, kappa;  // kappa = g rho0 / k0
};

template <typename T>
__host__ __device__ __forceinline__ T sgn(T x) {
  return x > T(0) ? T(1) : (x < T(0) ? T(-1) : T(0));
}

template <typename T>
__host__ __device__ __forceinline__ T tabs(T x) {
  return x < T(0) ? -x : x;
}

// FP64 device code: sign, magnitude and comparisons with zero on the integer
// pipe (the FP64 pipe runs at 1/64 of the FP32 rate on this part).  A double's
// bits, read as a signed 64-bit integer, are > 0 exactly for the values > 0,
// and < 0 for the values < 0 and -0 (NaN aside: non-admissible anyway).
#ifdef __CUDA_ARCH__
template <>
__device__ __forceinline__ double sgn<double>(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 ? 1.0 : (b < 0 && (b << 1) != 0 ? -1.0 : 0.0);
}
template <>
__device__ __forceinline__ double tabs<double>(double x) {
  return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffLL);
}
#endif
// sgn(s) x.  In FP64 device code on the integer pipe: the sign bit of s
// applied to x (a zero s gives the zero 0 x of the sign of x; x finite).
template <typename T>
__host__ __device__ __forceinline__ T sgn_mul(T s, T x) {
  return sgn(s) * x;
}
#ifdef __CUDA_ARCH__
template <>
__device__ __forceinline__ double sgn_mul<double>(double s, double x) {
  const long long bs = __double_as_longlong(s), bx = __double_as_longlong(x);
  const long long sign = (long long)0x8000000000000000ULL;
  return __longlong_as_double((bs << 1) == 0 ? (bx & sign) : (bx ^ (bs & sign)));
}
#endif
// x > 0, and |x| > y for y >= 0 (the same integer reading in FP64 device code).
template <typename T>
__host__ __device__ __forceinline__ bool gtz(T x) {
  return x > T(0);
}
template <typename T>
__host__ __device__ __forceinline__ bool abs_gt(T x, T y) {
  return tabs(x) > y;
}
template <typename T>
__host__ __device__ __forceinline__ bool abs_lt(T x, T y) {
  return tabs(x) < y;
}
#ifdef __CUDA_ARCH__
template <>
__device__ __forceinline__ bool gtz<double>(double x) {
  return __double_as_longlong(x) > 0;
}
template <>
__device__ __forceinline__ bool abs_gt<double>(double x, double y) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) > __double_as_longlong(y);
}
template <>
__device__ __forceinline__ bool abs_lt<double>(double x, double y) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) < __double_as_longlong(y);
}
#endif

// The smaller of two values >= 0 (or -0).  In FP64 device code on the
// integer pipe: the bits of doubles >= +0, read as signed 64-bit integers,
// order as the values do (-0 reads as the smallest, and equals +0 in every
// later use).
template <typename T>
__host__ __device__ __forceinline__ T min_nonneg(T a, T b) {
  return fmin(a, b);
}
#ifdef __CUDA_ARCH__
template <>
__device__ __forceinline__ double min_nonneg<double>(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return ia <= ib ? a : b;
}
#endif

// A face state: full conserved state q plus the exact jump to the other side
// is formed by the caller.  Velocities from 1/m.
template <typename T>
struct Vel {
  T u, v;
};

// Reciprocal: IEEE division on the host; on the device the refined hardware
// approximation below in double and the fast hardware reciprocal in float
// (relative error ~1e-7, inside the float path's stated tolerance).
template <typename T>
__host__ __device__ __forceinline__ T rcp(T x) {
  return T(1) / x;
}
// Double on the device: the hardware's approximate reciprocal r
// (rcp.approx.f64) refined by the series 1/x = r / (1 - e) = r (1 + e + e^2 +
// ...) with e = 1 - x r, truncated after e^2 (relative error e^3, below the
// last rounding for the approximation's |e|), rounded once by the last fused
// multiply-add: within one ulp of 1/x (tests/test_gpu_parity.py checks it
// against CUDA's division) in three FP64-pipe instructions, where two steps
// of Newton's iteration take four and IEEE division more; that pipe bounds
// the FP64 step.
template <>
__host__ __device__ __forceinline__ double rcp<double>(double x) {
#ifdef __CUDA_ARCH__
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
#else
  return 1.0 / x;
#endif
}
template <>
__host__ __device__ __forceinline__ float rcp<float>(float x) {
#ifdef __CUDA_ARCH__
  return __fdividef(1.0f, x);
#else
  return 1.0f / x;
#endif
}

template <typename T>
__host__ __device__ __forceinline__ Vel<T> velocity(T m, T mu, T mv) {
  const T r = rcp(m);
  return {mu * r, mv * r};
}

// The momentum fluxes of a face state: (mu u, mu v) across an x face and
// (mu v, mv v) across a y face.  In FP64 device code each product is rounded
// on its own (never fused into a neighbouring add), so that a flux formed
// once per cell and stored gives the same bits as one formed where it is
// used: the face solvers and the interior integral take the same four face
// states of a cell.
template <typename T>
__host__ __device__ __forceinline__ T prod(T a, T b) {
  return a * b;
}
#ifdef __CUDA_ARCH__
template <>
__device__ __forceinline__ double prod<double>(double a, double b) {
  return __dmul_rn(a, b);
}
#endif
template <typename T>
__host__ __device__ __forceinline__ void xflux(T m, T mu, T mv, T f[2]) {
  const Vel<T> w = velocity(m, mu, mv);
  f[0] = prod(mu, w.u);
  f[1] = prod(mu, w.v);
}
template <typename T>
__host__ __device__ __forceinline__ void yflux(T m, T mu, T mv, T g[2]) {
  const Vel<T> w = velocity(m, mu, mv);
  g[0] = prod(mu, w.v);
  g[1] = prod(mv, w.v);
}

// Paired FP32 forms of the face solvers (two evaluations of the same
// arithmetic in the two lanes of float2, one instruction per pair on sm_100
// and later); defined at the end of this file, used by xface and yface in
// FP32 device code.
__host__ __device__ __forceinline__ void xface_f2(const float qm[4], const float qp[4],
                                                  const float dq[4], const Phys<float>& P,
                                                  float Dm[4], float Dp[4]);
__host__ __device__ __forceinline__ void yface_f2(const float qm[4], const float qp[4],
                                                  const float dq[4], float dap,
                                                  const Phys<float>& P, float Dm[4], float Dp[4]);

// ---------------------------------------------------------------------------
// x faces: Osher viscosity, Eq. (OsherMatrixFormal_approx): 3-point
// Gauss-Legendre quadrature of |A1(Psi(s))| dq on the segment path, with
// |A1| = R1 |Lambda1| R1^-1 applied in closed form; b4x = u_bar Delta alpha with
// u_bar the same quadrature of u along the path.  D+- of Eq.
// (FIrstOrderDgeneric_x).  qm, qp: full states; dq: qp - qm formed exactly by
// the caller.
// ---------------------------------------------------------------------------
// fm, fp: the x fluxes (xflux) of qm and qp.
template <typename T>
__host__ __device__ __forceinline__ void xface_fx(const T qm[4], const T dq[4], const T fm[2],
                                                  const T fp[2], const Phys<T>& P, T Dm[4],
                                                  T Dp[4]) {
  const T s_gl[3] = {T(0.5 - 0.38729833462074168852), T(0.5), T(0.5 + 0.38729833462074168852)};
  // half the Gauss-Legendre weights (5/18, 8/18, 5/18): the sums below are
  // then half of V and of u_bar, exactly (a power-of-two scale), and so
  // D-+ = (F -+ V) / 2 takes one subtraction or addition per component
  const T w_gl[3] = {T(5.0 / 36.0), T(8.0 / 36.0), T(5.0 / 36.0)};
  T V0 = 0, V1 = 0, V2 = 0, lbar = 0, ubar = 0;
  const T dr = dq[0] - P.rho0 * dq[3];  // d1 - rho0 d4
  const T cdr = P.c * dr, B = P.rho0 * dq[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T m = qm[0] + s_gl[k] * dq[0];
    const T mu = qm[1] + s_gl[k] * dq[1];
    const T mv = qm[2] + s_gl[k] * dq[2];
    const Vel<T> w = velocity(m, mu, mv);
    const T la = tabs(w.u);
    const T w2 = dq[2] - w.v * dr;
    T Pk, amd;  // a1 + a5 and a5 - a1
    if (abs_lt(w.u, P.c)) {
      // |u| < c: |u - c| = c - u, |u + c| = c + u, so the two acoustic terms
      // combine to c dr + u e / c and e + u dr, e = d2 - u d1
      const T e = dq[1] - w.u * dq[0];
      Pk = cdr + (w.u * P.inv_c) * e;
      amd = e + w.u * dr;
    } else {
      const T uc = w.u * P.inv_c;
      // R1^-1 dq (rows 1, 2, 5; row 3 is d4 / c2)
      const T w1 = T(0.5) * ((T(1) + uc) * dq[0] - dq[1] * P.inv_c - B);
      const T w5 = T(0.5) * ((T(1) - uc) * dq[0] + dq[1] * P.inv_c - B);
      const T a1 = tabs(w.u - P.c) * w1, a5 = tabs(w.u + P.c) * w5;
      Pk = a1 + a5;
      amd = a5 - a1;
    }
    const T r0 = Pk + la * B;
    V0 += w_gl[k] * r0;
    V1 += w_gl[k] * (w.u * r0 + P.c * amd);
    V2 += w_gl[k] * (w.v * Pk + la * w2);
    lbar += w_gl[k] * la;  // V3 = lbar d4
    ubar += w_gl[k] * w.u;
  }
  const T V3 = lbar * dq[3];
  // F / 2
  const T F0 = T(0.5) * dq[1];
  const T F1 = T(0.5) * (fp[0] - fm[0]) + (T(0.5) * P.c2) * dr;
  const T F2 = T(0.5) * (fp[1] - fm[1]);
  const T F3 = ubar * dq[3];
  Dm[0] = F0 - V0;
  Dp[0] = F0 + V0;
  Dm[1] = F1 - V1;
  Dp[1] = F1 + V1;
  Dm[2] = F2 - V2;
  Dp[2] = F2 + V2;
  Dm[3] = F3 - V3;
  Dp[3] = F3 + V3;
}

template <typename T>
__host__ __device__ __forceinline__ void xface_scalar(const T qm[4], const T qp[4], const T dq[4],
                                                      const Phys<T>& P, T Dm[4], T Dp[4]) {
  T fm[2], fp[2];
  xflux(qm[0], qm[1], qm[2], fm);
  xflux(qp[0], qp[1], qp[2], fp);
  xface_fx(qm, dq, fm, fp, P, Dm, Dp);
}

// sign(A1(q)) r = R1 sign(Lambda1) R1^-1 r for r with zero 5th entry: the
// closed form of |A1| in xface with each |lambda| replaced by sign(lambda).
template <typename T>
__host__ __device__ __forceinline__ void sign_A1(T u, T v, const T r[4], const Phys<T>& P,
                                                 T out[4]) {
  const T uc = u * P.inv_c;
  const T w1 = T(0.5) * ((T(1) + uc) * r[0] - r[1] * P.inv_c - P.rho0 * r[3]);
  const T w5 = T(0.5) * ((T(1) - uc) * r[0] + r[1] * P.inv_c - P.rho0 * r[3]);
  const T w2 = r[2] - v * (r[0] - P.rho0 * r[3]);
  const T s1 = sgn(u - P.c), s5 = sgn(u + P.c), s3 = sgn(u);
  const T a1 = s1 * w1, a5 = s5 * w5;
  const T Pk = a1 + a5;
  const T r0 = Pk + s3 * P.rho0 * r[3];
  out[0] = r0;
  out[1] = u * r0 + P.c * (a5 - a1);
  out[2] = v * Pk + s3 * w2;
  out[3] = s3 * r[3];
}

// x faces with the conservative Osher-Romberg viscosity of Eq. (OR_cons): the
// Romberg sum over the segment path of sign(A1(Psi(s_k))) times the flux
// difference across the sub-segment, completed by b4x = u(Psi(s_k)) Delta
// alpha; the face's own b4x uses the Romberg average of the node velocities.
// Arguments as for xface.
template <typename T>
__host__ __device__ __forceinline__ void xface_or(const T qm[4], const T qp[4], const T dq[4],
                                                  const Phys<T>& P, T Dm[4], T Dp[4]) {
  // nodes s = 0, 1/4, 1/2, 3/4, 1 (interior nodes on the path, exact endpoints)
  T mu_[5], u_[5], v_[5];
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    const T s = T(0.25 * k);
    const T m = qm[0] + s * dq[0];
    mu_[k] = qm[1] + s * dq[1];
    const Vel<T> w = velocity(m, mu_[k], qm[2] + s * dq[2]);
    u_[k] = w.u;
    v_[k] = w.v;
  }
  {
    const Vel<T> a = velocity(qm[0], qm[1], qm[2]);
    const Vel<T> b = velocity(qp[0], qp[1], qp[2]);
    mu_[0] = qm[1];
    u_[0] = a.u;
    v_[0] = a.v;
    mu_[4] = qp[1];
    u_[4] = b.u;
    v_[4] = b.v;
  }
  // f components at nodes 0, 2, 4: (mu, mu u + alpha p, mu v); alpha p is
  // linear in q, so its jump over a sub-segment of length l is c2 l dr
  const T f1_0 = mu_[0] * u_[0], f2_0 = mu_[0] * v_[0];
  const T f1_2 = mu_[2] * u_[2], f2_2 = mu_[2] * v_[2];
  const T f1_4 = mu_[4] * u_[4], f2_4 = mu_[4] * v_[4];
  const T dr = dq[0] - P.rho0 * dq[3];
  T V[4] = {0, 0, 0, 0};
  {  // [0, 1/2], node 1/4, weight 4/3
    const T r[4] = {mu_[2] - mu_[0], f1_2 - f1_0 + T(0.5) * P.c2 * dr, f2_2 - f2_0,
                    T(0.5) * u_[1] * dq[3]};
    T o[4];
    sign_A1(u_[1], v_[1], r, P, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) V[c] += T(4.0 / 3.0) * o[c];
  }
  {  // [1/2, 1], node 3/4, weight 4/3
    const T r[4] = {mu_[4] - mu_[2], f1_4 - f1_2 + T(0.5) * P.c2 * dr, f2_4 - f2_2,
                    T(0.5) * u_[3] * dq[3]};
    T o[4];
    sign_A1(u_[3], v_[3], r, P, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) V[c] += T(4.0 / 3.0) * o[c];
  }
  {  // [0, 1], node 1/2, weight -1/3
    const T r[4] = {dq[1], f1_4 - f1_0 + P.c2 * dr, f2_4 - f2_0, u_[2] * dq[3]};
    T o[4];
    sign_A1(u_[2], v_[2], r, P, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) V[c] -= T(1.0 / 3.0) * o[c];
  }
  const T ubar = T(2.0 / 3.0) * (u_[1] + u_[3]) - T(1.0 / 3.0) * u_[2];
  const T F[4] = {dq[1], f1_4 - f1_0 + P.c2 * dr, f2_4 - f2_0, ubar * dq[3]};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    Dm[c] = T(0.5) * (F[c] - V[c]);
    Dp[c] = T(0.5) * (F[c] + V[c]);
  }
}

// sign(A2(q)) r = R2 sign(Lambda2) R2^-1 r for r with zero 5th entry, closed form
// of the printed eigenstructure; the eigenvalue-0 mode has sign 0.
template <typename T>
__host__ __device__ __forceinline__ void sign_A2(T u, T v, const T r[4], const Phys<T>& P,
                                                 T out[4]) {
  if (abs_lt(v, P.c)) {
    // |v| < c: the acoustic eigenvalues v - c < 0 < v + c, so the two acoustic
    // terms combine to (w5 - w1) = (r2 - v r0) / c and (w5 + w1) = r0 - rho0 r3
    const T rr = P.rho0 * r[3];
    const T D = r[0] - rr;
    const T Pk = (r[2] - v * r[0]) * P.inv_c;
    const T o0 = Pk + sgn_mul(v, rr);
    out[0] = o0;
    out[1] = u * Pk + sgn_mul(v, r[1] - u * D);
    out[2] = v * o0 + P.c * D;
    out[3] = sgn_mul(v, r[3]);
    return;
  }
  const T s3 = sgn(v);
  const T vc = v * P.inv_c;
  const T w1 = T(0.5) * ((T(1) + vc) * r[0] - r[2] * P.inv_c - P.rho0 * r[3]);
  const T w5 = T(0.5) * ((T(1) - vc) * r[0] + r[2] * P.inv_c - P.rho0 * r[3]);
  const T w2 = r[1] - u * (r[0] - P.rho0 * r[3]);
  const T s1 = sgn(v - P.c), s5 = sgn(v + P.c);
  const T a1 = s1 * w1, a5 = s5 * w5;
  const T Pk = a1 + a5;
  const T srho = s3 * P.rho0 * r[3];
  out[0] = Pk + srho;
  out[1] = u * Pk + s3 * w2;
  out[2] = v * (Pk + srho) + P.c * (a5 - a1);
  out[3] = s3 * r[3];
}

// ---------------------------------------------------------------------------
// y faces: well-balanced Osher-Romberg scheme, Eq. (ViscosityOR), for two
// states at the same height.  The path Phi = Phi^E + Phi^f (Eq. (path)) is
// linear in the conserved variables, so node states are qm + s dq.  R_k uses
// the flux difference g(Phi(s_k+e_k)) - g(Phi(s_k-e_k)) plus B_Phi: b3 is the
// path integral of d(alpha p) (exact for gamma = 1, equilibrium part included),
// b4 = v(Phi(s_k)) Delta alpha on the sub-interval; the face's own b4 uses the
// Romberg combination of the node velocities.  D+- of Eq.
// (FIrstOrderDgeneric_y).
// ---------------------------------------------------------------------------
// dap: jump of alpha p = c2 (m - rho0 alpha) from qm to qp, formed by the
// caller so that it is exactly zero between two states of one rest profile.
// gm, gp: the y fluxes (yflux) of qm and qp.
template <typename T>
__host__ __device__ __forceinline__ void yface_fx(const T qm[4], const T dq[4], const T gm[2],
                                                  const T gp[2], T dap, const Phys<T>& P, T Dm[4],
                                                  T Dp[4]) {
  // interior nodes s = 1/4, 1/2, 3/4 on the path
  T u_[4], v_[4];
  T mu2 = T(0), mv2 = T(0);
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    const T s = T(0.25 * k);
    const T m = qm[0] + s * dq[0];
    const T mu = qm[1] + s * dq[1];
    const T mv = qm[2] + s * dq[2];
    const Vel<T> w = velocity(m, mu, mv);
    u_[k] = w.u;
    v_[k] = w.v;
    if (k == 2) {
      mu2 = mu;
      mv2 = mv;
    }
  }
  // g components at nodes 0, 2, 4: (mv, mu v, mv v)
  const T g1_0 = gm[0], g2_0 = gm[1];
  const T g1_2 = mu2 * v_[2], g2_2 = mv2 * v_[2];
  const T g1_4 = gp[0], g2_4 = gp[1];
  // the Romberg weights 4/3, 4/3, -1/3 halved: V and v_bar below are half
  // of the sums, exactly, so that D-+ = G/2 -+ V/2
  T V[4] = {0, 0, 0, 0};
  {  // k = 1: [0, 1/2], node 1/4, weight 4/3
    const T r[4] = {T(0.5) * dq[2], g1_2 - g1_0, g2_2 - g2_0 + T(0.5) * dap,
                    T(0.5) * v_[1] * dq[3]};
    T o[4];
    sign_A2(u_[1], v_[1], r, P, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) V[c] += T(2.0 / 3.0) * o[c];
  }
  {  // k = 2: [1/2, 1], node 3/4, weight 4/3
    const T r[4] = {T(0.5) * dq[2], g1_4 - g1_2, g2_4 - g2_2 + T(0.5) * dap,
                    T(0.5) * v_[3] * dq[3]};
    T o[4];
    sign_A2(u_[3], v_[3], r, P, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) V[c] += T(2.0 / 3.0) * o[c];
  }
  {  // k = 3: [0, 1], node 1/2, weight -1/3
    const T r[4] = {dq[2], g1_4 - g1_0, g2_4 - g2_0 + dap, v_[2] * dq[3]};
    T o[4];
    sign_A2(u_[2], v_[2], r, P, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) V[c] -= T(1.0 / 6.0) * o[c];
  }
  const T vbar = T(1.0 / 3.0) * (v_[1] + v_[3]) - T(1.0 / 6.0) * v_[2];
  // G / 2
  const T G0 = T(0.5) * dq[2];
  const T G1 = T(0.5) * (g1_4 - g1_0);
  const T G2 = T(0.5) * (g2_4 - g2_0 + dap);
  const T G3 = vbar * dq[3];
  Dm[0] = G0 - V[0];
  Dp[0] = G0 + V[0];
  Dm[1] = G1 - V[1];
  Dp[1] = G1 + V[1];
  Dm[2] = G2 - V[2];
  Dp[2] = G2 + V[2];
  Dm[3] = G3 - V[3];
  Dp[3] = G3 + V[3];
}

template <typename T>
__host__ __device__ __forceinline__ void yface_scalar(const T qm[4], const T qp[4], const T dq[4],
                                                      T dap, const Phys<T>& P, T Dm[4], T Dp[4]) {
  T gm[2], gp[2];
  yflux(qm[0], qm[1], qm[2], gm);
  yflux(qp[0], qp[1], qp[2], gp);
  yface_fx(qm, dq, gm, gp, dap, P, Dm, Dp);
}

// ---------------------------------------------------------------------------
// Per-cell reconstruction of Section 3.4 for one fluid cell, given the
// fluctuations of its four edge neighbours (or their wall/transmissive ghosts)
// w.r.t. the cell's water-at-rest state Q^E_ij, and the stencil min/max:
// central slopes, one Barth-Jespersen factor per cell (Eq.
// (reconstruction_fluctuation2); the factor of each component is the printed
// one for face increments |d| >= 2 eta, 1 below eta, linear between), the
// order switch alpha <= 10 eps, the half-step predictor dQ/dt = -(A1 dQ/dx +
// A2 dQ/dy) with grad Q = grad Q^E + Psi grad Q^f (Eq. (gradientEq+fluct);
// the exact balance c^2 dm^E/dy + g m^E = 0 is removed), and the fluctuation
// states at the four face midpoints at t^{n+1/2}.  A cell whose reconstructed
// states are not admissible is advanced at first order.
// In:  Qf (own fluctuation, Qf[3] = 0), fW..fN (neighbour fluctuations), mx, mn.
// Out: fW..fN overwritten by the face fluctuation states, base = centre
//      fluctuation at t^{n+1/2}; returns Psi (the slopes used are Psi g).
// ---------------------------------------------------------------------------
template <typename T>
struct ReconConsts {
  T half_dx, half_dy, inv_2dx, inv_2dy, ten_eps, half_dt;
  T eta[4], inv_eta[4];
};

template <typename T>
__host__ __device__ __forceinline__ T recon_core(const T Qf[4], T fW[4], T fE[4], T fS[4],
                                                 T fN[4], const T mx[4], const T mn[4], T aE,
                                                 T mEc, T mES, T mEN, T rEc,
                                                 const Phys<T>& P, const ReconConsts<T>& R,
                                                 T base[4], T gxa[2]) {
  T gx[4], gy[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    gx[v] = (fE[v] - fW[v]) * R.inv_2dx;
    gy[v] = (fN[v] - fS[v]) * R.inv_2dy;
  }
  T psi = T(1);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    // The faces at -h/2 and +h/2 see the increments -d and +d, bounded by up =
    // mx - Qf >= 0 on the side where the increment is positive and by -dn =
    // Qf - mn >= 0 on the other: the two factors min(1, up/|d|) and
    // min(1, -dn/|d|), of which the smaller, min(1, lim/|d|) with lim =
    // min(up, -dn), decides (the factor of a face is monotone in its ratio,
    // and so are the rounded operations: the same bits as taking both).
    const T lim = min_nonneg(mx[v] - Qf[v], Qf[v] - mn[v]);
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      const T d = dir == 0 ? R.half_dx * gx[v] : R.half_dy * gy[v];
      if (abs_gt(d, R.eta[v])) {
        const T ad = tabs(d);
        const T ramp = min_nonneg(T(1), (ad - R.eta[v]) * R.inv_eta[v]);
        const T phi = min_nonneg(T(1), lim * rcp(ad));
        psi = min_nonneg(psi, T(1) - ramp * (T(1) - phi));
      }
    }
  }
  T dtQ[4] = {0, 0, 0, 0};
  if (aE <= R.ten_eps) {
    psi = T(0);
  } else {
    const Vel<T> vel = velocity(mEc + Qf[0], Qf[1], Qf[2]);
    const T u = vel.u, v = vel.v;
    T sx[4], sy[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      sx[c] = psi * gx[c];
      sy[c] = psi * gy[c];
    }
    const T dmE = aE * (-P.kappa * rEc);
    const T uv = u * v;
    const T a1 = sx[1];
    const T a2 = (P.c2 - u * u) * sx[0] + T(2) * u * sx[1] - P.k0 * sx[3];
    const T a3 = -uv * sx[0] + v * sx[1] + u * sx[2];
    const T a4 = u * sx[3];
    const T b1 = sy[2];
    const T b2 = -uv * sy[0] + v * sy[1] + u * sy[2] - uv * dmE;
    const T b3 = (P.c2 - v * v) * sy[0] + T(2) * v * sy[2] - P.k0 * sy[3] - v * v * dmE + P.g * Qf[0];
    const T b4 = v * sy[3];
    dtQ[0] = -(a1 + b1);
    dtQ[1] = -(a2 + b2);
    dtQ[2] = -(a3 + b3);
    dtQ[3] = -(a4 + b4);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    base[c] = Qf[c] + R.half_dt * dtQ[c];
    const T sxh = psi * gx[c] * R.half_dx, syh = psi * gy[c] * R.half_dy;
    fW[c] = base[c] - sxh;
    fE[c] = base[c] + sxh;
    fS[c] = base[c] - syh;
    fN[c] = base[c] + syh;
  }
  const bool ok = gtz(mEc + fW[0]) && gtz(aE + fW[3]) && gtz(mEc + fE[0]) && gtz(aE + fE[3]) &&
                  gtz(mES + fS[0]) && gtz(aE + fS[3]) && gtz(mEN + fN[0]) && gtz(aE + fN[3]) &&
                  gtz(mEc + base[0]) && gtz(aE + base[3]);
  if (!ok) {
    psi = T(0);
#pragma unroll
    for (int c = 0; c < 4; ++c) fW[c] = fE[c] = fS[c] = fN[c] = base[c] = Qf[c];
  }
  gxa[0] = psi * gx[3];
  gxa[1] = psi * gy[3];
  return psi;
}

// Interior integral of Eq. (Scheme) for one cell with the mid-point rule:
// the conservative part f(q_E) - f(q_W), g(q_N) - g(q_S) plus B grad q, whose
// third component is the fluctuation form of Eq. (b^y_3_final_integral)
// (pressure part [(alpha p)^f]_S^N and gravity g dy (m - m^E) at the centre).
// xW, xE: the x fluxes (xflux) of the W and E face states; yS, yN: the y
// fluxes (yflux) of the S and N ones.
template <typename T>
__host__ __device__ __forceinline__ void interior_terms_fx(const T fW[4], const T fE[4],
                                                           const T fS[4], const T fN[4],
                                                           const T base[4], T mEc, const T xW[2],
                                                           const T xE[2], const T yS[2],
                                                           const T yN[2], T dax, T day, T dx,
                                                           T dy, const Phys<T>& P, T Ix[4],
                                                           T Iy[4]) {
  Ix[0] = fE[1] - fW[1];
  Ix[1] = (xE[0] - xW[0]) + P.c2 * ((fE[0] - fW[0]) - P.rho0 * (fE[3] - fW[3]));
  Ix[2] = xE[1] - xW[1];
  Iy[0] = fN[2] - fS[2];
  Iy[1] = yN[0] - yS[0];
  Iy[2] = (yN[1] - yS[1]) + P.c2 * ((fN[0] - fS[0]) - P.rho0 * (fN[3] - fS[3])) +
          P.g * dy * base[0];
  // the non-conservative alpha transport u d(alpha)/dx, v d(alpha)/dy: zero
  // where alpha is uniform (both limited slopes zero: every cell away from
  // the interface), without the centre velocity
  if (dax == T(0) && day == T(0)) {
    Ix[3] = Iy[3] = T(0);
  } else {
    const Vel<T> vc = velocity(mEc + base[0], base[1], base[2]);
    Ix[3] = dx * vc.u * dax;
    Iy[3] = dy * vc.v * day;
  }
}

template <typename T>
__host__ __device__ __forceinline__ void interior_terms(const T fW[4], const T fE[4],
                                                        const T fS[4], const T fN[4],
                                                        const T base[4], T mEc, T mES, T mEN,
                                                        T dax, T day, T dx, T dy,
                                                        const Phys<T>& P, T Ix[4], T Iy[4]) {
  T xW[2], xE[2], yS[2], yN[2];
  xflux(mEc + fW[0], fW[1], fW[2], xW);
  xflux(mEc + fE[0], fE[1], fE[2], xE);
  yflux(mES + fS[0], fS[1], fS[2], yS);
  yflux(mEN + fN[0], fN[1], fN[2], yN);
  interior_terms_fx(fW, fE, fS, fN, base, mEc, xW, xE, yS, yN, dax, day, dx, dy, P, Ix, Iy);
}

// ---------------------------------------------------------------------------
// Paired FP32 arithmetic: each helper applies one IEEE operation (rounded to
// nearest) to both lanes; on the device one paired instruction, on the host
// two scalar ones with the same results.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__host__ __device__ __forceinline__ float2 add2(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return add2(a, make_float2(-b.x, -b.y));
}
__host__ __device__ __forceinline__ float2 mul2(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
  return __fmul2_rn(a, b);
#else
  return make_float2(a.x * b.x, a.y * b.y);
#endif
}
__host__ __device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
#ifdef __CUDA_ARCH__
  return __ffma2_rn(a, b, c);
#else
  return make_float2(std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y));
#endif
}
__host__ __device__ __forceinline__ float2 abs2(float2 a) {
  return make_float2(tabs(a.x), tabs(a.y));
}
__host__ __device__ __forceinline__ float2 sgn2(float2 a) { return make_float2(sgn(a.x), sgn(a.y)); }
__host__ __device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp(a.x), rcp(a.y)); }

// One Gauss-Legendre node of xface on float2 lanes: node velocity (u, v) and
// its contributions (r0, u r0 + c (a5 - a1), v Pk + |u| w2, |u| d4, u).
struct XNode2 {
  float2 V0, V1, V2, V3, u;
};
__host__ __device__ __forceinline__ XNode2 xnode2(float2 u, float2 v, const float dq[4], float dr,
                                                 float w1c, float w5c, float B,
                                                 const Phys<float>& P) {
  // w1 = ((1 + uc) d1 - d2 / c - rho0 d4) / 2 and w5 = ((1 - uc) d1 + d2 / c - rho0 d4) / 2
  // as (w1c + uc d1 / 2), (w5c - uc d1 / 2); w2 = d3 - v dr
  const float2 uh = mul2(u, bc2(0.5f * P.inv_c * dq[0]));
  const float2 w1 = add2(bc2(w1c), uh);
  const float2 w5 = sub2(bc2(w5c), uh);
  const float2 w2 = fma2(v, bc2(-dr), bc2(dq[2]));
  const float2 l1 = abs2(add2(u, bc2(-P.c))), l5 = abs2(add2(u, bc2(P.c))), la = abs2(u);
  const float2 a1 = mul2(l1, w1), a5 = mul2(l5, w5);
  const float2 Pk = add2(a1, a5);
  const float2 r0 = fma2(la, bc2(B), Pk);
  XNode2 o;
  o.V0 = r0;
  o.V1 = fma2(u, r0, mul2(bc2(P.c), sub2(a5, a1)));
  o.V2 = fma2(v, Pk, mul2(la, w2));
  o.V3 = mul2(la, bc2(dq[3]));
  o.u = u;
  return o;
}

// xface in FP32 with the Gauss-Legendre nodes s0 and s2 (equal weights 5/18)
// in the two lanes and the middle node s1 = 1/2 (weight 8/18) in the first
// lane of a second call; the endpoint velocities of qm and qp as a pair.
__host__ __device__ __forceinline__ void xface_f2(const float qm[4], const float qp[4],
                                                  const float dq[4], const Phys<float>& P,
                                                  float Dm[4], float Dp[4]) {
  const float h = 0.38729833462074168852f;
  const float dr = dq[0] - P.rho0 * dq[3];
  const float B = P.rho0 * dq[3];
  const float A = dq[1] * P.inv_c;
  const float w1c = 0.5f * ((dq[0] - A) - B), w5c = 0.5f * ((dq[0] + A) - B);
  // nodes s0, s2 | s1 and the endpoints qm, qp: one velocity evaluation each
  const float2 s02 = make_float2(0.5f - h, 0.5f + h);
  const float2 m02 = fma2(s02, bc2(dq[0]), bc2(qm[0]));
  const float2 mu02 = fma2(s02, bc2(dq[1]), bc2(qm[1]));
  const float2 mv02 = fma2(s02, bc2(dq[2]), bc2(qm[2]));
  const float m1 = qm[0] + 0.5f * dq[0], mu1 = qm[1] + 0.5f * dq[1], mv1 = qm[2] + 0.5f * dq[2];
  const float2 r02 = rcp2(m02);
  const float2 rmp = rcp2(make_float2(qm[0], qp[0]));
  const float2 r1e = make_float2(rcp(m1), 0.0f);
  const float2 u02 = mul2(mu02, r02), v02 = mul2(mv02, r02);
  const float2 mu1e = make_float2(mu1, 0.0f), mv1e = make_float2(mv1, 0.0f);
  const float2 u1 = mul2(mu1e, r1e), v1 = mul2(mv1e, r1e);
  const XNode2 a = xnode2(u02, v02, dq, dr, w1c, w5c, B, P);
  const XNode2 b = xnode2(u1, v1, dq, dr, w1c, w5c, B, P);
  const float ws = 5.0f / 18.0f, wm = 8.0f / 18.0f;
  const float V0 = ws * (a.V0.x + a.V0.y) + wm * b.V0.x;
  const float V1 = ws * (a.V1.x + a.V1.y) + wm * b.V1.x;
  const float V2 = ws * (a.V2.x + a.V2.y) + wm * b.V2.x;
  const float V3 = ws * (a.V3.x + a.V3.y) + wm * b.V3.x;
  const float ubar = ws * (a.u.x + a.u.y) + wm * b.u.x;
  // endpoint fluxes: (qm1 um, qp1 up) and (qm1 vm, qp1 vp)
  const float2 mu_mp = make_float2(qm[1], qp[1]);
  const float2 uv_u = mul2(mu_mp, rmp);                              // (um, up)
  const float2 uv_v = mul2(make_float2(qm[2], qp[2]), rmp);          // (vm, vp)
  const float2 f1 = mul2(mu_mp, uv_u), f2 = mul2(mu_mp, uv_v);
  const float F[4] = {dq[1], (f1.y - f1.x) + P.c2 * dr, f2.y - f2.x, ubar * dq[3]};
  const float V[4] = {V0, V1, V2, V3};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float2 d = mul2(bc2(0.5f), add2(bc2(F[c]), make_float2(-V[c], V[c])));
    Dm[c] = d.x;
    Dp[c] = d.y;
  }
}

// sign_A2 on float2 lanes (closed form of sign_A2): the subsonic form for
// both lanes, and the general one, selected lane by lane, when a lane is not
// subsonic (rare; the per-lane formulas are those of sign_A2).
__host__ __device__ __forceinline__ void sign_A2_f2(float2 u, float2 v, const float2 r[4],
                                                    const Phys<float>& P, float2 out[4]) {
  const float2 rr = mul2(bc2(P.rho0), r[3]);
  const float2 s3 = sgn2(v);
  const float2 D = sub2(r[0], rr);
  const float2 Pk = mul2(fma2(make_float2(-v.x, -v.y), r[0], r[2]), bc2(P.inv_c));
  const float2 o0 = fma2(s3, rr, Pk);
  out[0] = o0;
  out[1] = fma2(u, Pk, mul2(s3, fma2(make_float2(-u.x, -u.y), D, r[1])));
  out[2] = fma2(v, o0, mul2(bc2(P.c), D));
  out[3] = mul2(s3, r[3]);
  const bool sx = tabs(v.x) < P.c, sy = tabs(v.y) < P.c;
  if (!(sx && sy)) {
    const float rx[4] = {r[0].x, r[1].x, r[2].x, r[3].x}, ry[4] = {r[0].y, r[1].y, r[2].y, r[3].y};
    float ox[4], oy[4];
    sign_A2(u.x, v.x, rx, P, ox);
    sign_A2(u.y, v.y, ry, P, oy);
#pragma unroll
    for (int c = 0; c < 4; ++c) out[c] = make_float2(ox[c], oy[c]);
  }
}

// yface in FP32: the two half-segment terms of the Osher-Romberg sum (nodes
// 1/4 and 3/4, weight 4/3) in the two lanes, the whole-segment term (node
// 1/2, weight -1/3) in the first lane of a second call; the endpoint
// velocities of qm and qp as a pair.
__host__ __device__ __forceinline__ void yface_f2(const float qm[4], const float qp[4],
                                                  const float dq[4], float dap,
                                                  const Phys<float>& P, float Dm[4], float Dp[4]) {
  const float2 s13 = make_float2(0.25f, 0.75f);
  const float2 m13 = fma2(s13, bc2(dq[0]), bc2(qm[0]));
  const float2 mu13 = fma2(s13, bc2(dq[1]), bc2(qm[1]));
  const float2 mv13 = fma2(s13, bc2(dq[2]), bc2(qm[2]));
  const float m2 = qm[0] + 0.5f * dq[0], mu2 = qm[1] + 0.5f * dq[1], mv2 = qm[2] + 0.5f * dq[2];
  const float2 r13 = rcp2(m13);
  const float2 r04 = rcp2(make_float2(qm[0], qp[0]));
  const float r2_ = rcp(m2);
  const float2 u13 = mul2(mu13, r13), v13 = mul2(mv13, r13);
  const float u2 = mu2 * r2_, v2 = mv2 * r2_;
  const float2 mu04 = make_float2(qm[1], qp[1]), mv04 = make_float2(qm[2], qp[2]);
  const float2 v04 = mul2(mv04, r04);
  // g = (mv, mu v, mv v) at the nodes 0, 4 (pair) and 2
  const float2 g1_04 = mul2(mu04, v04), g2_04 = mul2(mv04, v04);
  const float g1_2 = mu2 * v2, g2_2 = mv2 * v2;
  const float hd = 0.5f * dap;
  // half segments [0, 1/2] (lane x) and [1/2, 1] (lane y)
  float2 rh[4];
  rh[0] = bc2(0.5f * dq[2]);
  rh[1] = sub2(make_float2(g1_2, g1_04.y), make_float2(g1_04.x, g1_2));
  rh[2] = add2(sub2(make_float2(g2_2, g2_04.y), make_float2(g2_04.x, g2_2)), bc2(hd));
  rh[3] = mul2(v13, bc2(0.5f * dq[3]));
  float2 oh[4];
  sign_A2_f2(u13, v13, rh, P, oh);
  // whole segment (lane x)
  const float G1 = g1_04.y - g1_04.x, G2 = (g2_04.y - g2_04.x) + dap;
  float2 rw[4];
  rw[0] = make_float2(dq[2], 0.0f);
  rw[1] = make_float2(G1, 0.0f);
  rw[2] = make_float2(G2, 0.0f);
  rw[3] = make_float2(v2 * dq[3], 0.0f);
  float2 ow[4];
  sign_A2_f2(make_float2(u2, 0.0f), make_float2(v2, 0.0f), rw, P, ow);
  const float vbar = (2.0f / 3.0f) * (v13.x + v13.y) - (1.0f / 3.0f) * v2;
  const float G[4] = {dq[2], G1, G2, vbar * dq[3]};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float Vc = (4.0f / 3.0f) * (oh[c].x + oh[c].y) - (1.0f / 3.0f) * ow[c].x;
    const float2 d = mul2(bc2(0.5f), add2(bc2(G[c]), make_float2(-Vc, Vc)));
    Dm[c] = d.x;
    Dp[c] = d.y;
  }
}

// The face solvers used by the step kernels: the paired forms in FP32 device
// code, the scalar ones otherwise (FP64, and the host).
template <typename T>
__host__ __device__ __forceinline__ void xface(const T qm[4], const T qp[4], const T dq[4],
                                               const Phys<T>& P, T Dm[4], T Dp[4]) {
#ifdef __CUDA_ARCH__
  if constexpr (std::is_same<T, float>::value) {
    xface_f2(qm, qp, dq, P, Dm, Dp);
    return;
  }
#endif
  xface_scalar(qm, qp, dq, P, Dm, Dp);
}

template <typename T>
__host__ __device__ __forceinline__ void yface(const T qm[4], const T qp[4], const T dq[4],
                                               T dap, const Phys<T>& P, T Dm[4], T Dp[4]) {
#ifdef __CUDA_ARCH__
  if constexpr (std::is_same<T, float>::value) {
    yface_f2(qm, qp, dq, dap, P, Dm, Dp);
    return;
  }
#endif
  yface_scalar(qm, qp, dq, dap, P, Dm, Dp);
}

}  // namespace fv
