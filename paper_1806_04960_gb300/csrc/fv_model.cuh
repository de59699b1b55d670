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

// A face state: full conserved state q plus the exact jump to the other side
// is formed by the caller.  Velocities from 1/m.
template <typename T>
struct Vel {
  T u, v;
};

template <typename T>
__host__ __device__ __forceinline__ Vel<T> velocity(T m, T mu, T mv) {
  const T r = T(1) / m;
  return {mu * r, mv * r};
}

// ---------------------------------------------------------------------------
// x faces: Osher viscosity, Eq. (OsherMatrixFormal_approx): 3-point
// Gauss-Legendre quadrature of |A1(Psi(s))| dq on the segment path, with
// |A1| = R1 |Lambda1| R1^-1 applied in closed form; b4x = u_bar Delta alpha with
// u_bar the same quadrature of u along the path.  D+- of Eq.
// (FIrstOrderDgeneric_x).  qm, qp: full states; dq: qp - qm formed exactly by
// the caller.
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ __forceinline__ void xface(const T qm[4], const T qp[4], const T dq[4],
                                               const Phys<T>& P, T Dm[4], T Dp[4]) {
  const T s_gl[3] = {T(0.5) - T(0.38729833462074168852), T(0.5),
                     T(0.5) + T(0.38729833462074168852)};
  const T w_gl[3] = {T(5.0 / 18.0), T(8.0 / 18.0), T(5.0 / 18.0)};
  T V0 = 0, V1 = 0, V2 = 0, V3 = 0, ubar = 0;
  const T dr = dq[0] - P.rho0 * dq[3];  // d1 - rho0 d4
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T m = qm[0] + s_gl[k] * dq[0];
    const T mu = qm[1] + s_gl[k] * dq[1];
    const T mv = qm[2] + s_gl[k] * dq[2];
    const Vel<T> w = velocity(m, mu, mv);
    const T uc = w.u * P.inv_c;
    // R1^-1 dq (rows 1, 2, 5; row 3 is d4 / c2)
    const T w1 = T(0.5) * ((T(1) + uc) * dq[0] - dq[1] * P.inv_c - P.rho0 * dq[3]);
    const T w5 = T(0.5) * ((T(1) - uc) * dq[0] + dq[1] * P.inv_c - P.rho0 * dq[3]);
    const T w2 = dq[2] - w.v * dr;
    const T l1 = tabs(w.u - P.c), l5 = tabs(w.u + P.c), la = tabs(w.u);
    const T a1 = l1 * w1, a5 = l5 * w5;
    const T Pk = a1 + a5;
    const T r0 = Pk + la * P.rho0 * dq[3];
    V0 += w_gl[k] * r0;
    V1 += w_gl[k] * (w.u * r0 + P.c * (a5 - a1));
    V2 += w_gl[k] * (w.v * Pk + la * w2);
    V3 += w_gl[k] * (la * dq[3]);
    ubar += w_gl[k] * w.u;
  }
  const Vel<T> em = velocity(qm[0], qm[1], qm[2]);
  const Vel<T> ep = velocity(qp[0], qp[1], qp[2]);
  const T F0 = dq[1];
  const T F1 = (qp[1] * ep.u - qm[1] * em.u) + P.c2 * dr;
  const T F2 = qp[1] * ep.v - qm[1] * em.v;
  const T F3 = ubar * dq[3];
  Dm[0] = T(0.5) * (F0 - V0);
  Dp[0] = T(0.5) * (F0 + V0);
  Dm[1] = T(0.5) * (F1 - V1);
  Dp[1] = T(0.5) * (F1 + V1);
  Dm[2] = T(0.5) * (F2 - V2);
  Dp[2] = T(0.5) * (F2 + V2);
  Dm[3] = T(0.5) * (F3 - V3);
  Dp[3] = T(0.5) * (F3 + V3);
}

// sign(A2(q)) r = R2 sign(Lambda2) R2^-1 r for r with zero 5th entry, closed form
// of the printed eigenstructure; the eigenvalue-0 mode has sign 0.
template <typename T>
__host__ __device__ __forceinline__ void sign_A2(T u, T v, const T r[4], const Phys<T>& P,
                                                 T out[4]) {
  const T vc = v * P.inv_c;
  const T w1 = T(0.5) * ((T(1) + vc) * r[0] - r[2] * P.inv_c - P.rho0 * r[3]);
  const T w5 = T(0.5) * ((T(1) - vc) * r[0] + r[2] * P.inv_c - P.rho0 * r[3]);
  const T w2 = r[1] - u * (r[0] - P.rho0 * r[3]);
  const T s1 = sgn(v - P.c), s5 = sgn(v + P.c), s3 = sgn(v);
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
template <typename T>
__host__ __device__ __forceinline__ void yface(const T qm[4], const T qp[4], const T dq[4],
                                               const Phys<T>& P, T Dm[4], T Dp[4]) {
  // nodes s = 0, 1/4, 1/2, 3/4, 1
  T mu_[5], mv_[5], u_[5], v_[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const T s = T(0.25) * T(k);
    const T m = qm[0] + s * dq[0];
    mu_[k] = qm[1] + s * dq[1];
    mv_[k] = qm[2] + s * dq[2];
    const Vel<T> w = velocity(m, mu_[k], mv_[k]);
    u_[k] = w.u;
    v_[k] = w.v;
  }
  // exact endpoints for the fluxes
  {
    const Vel<T> a = velocity(qm[0], qm[1], qm[2]);
    const Vel<T> b = velocity(qp[0], qp[1], qp[2]);
    mu_[0] = qm[1];
    mv_[0] = qm[2];
    u_[0] = a.u;
    v_[0] = a.v;
    mu_[4] = qp[1];
    mv_[4] = qp[2];
    u_[4] = b.u;
    v_[4] = b.v;
  }
  const T dap = P.c2 * (dq[0] - P.rho0 * dq[3]);  // Delta(alpha p) over [0, 1]
  // g components at nodes 0, 2, 4: (mv, mu v, mv v)
  const T g1_0 = mu_[0] * v_[0], g2_0 = mv_[0] * v_[0];
  const T g1_2 = mu_[2] * v_[2], g2_2 = mv_[2] * v_[2];
  const T g1_4 = mu_[4] * v_[4], g2_4 = mv_[4] * v_[4];
  T V[4] = {0, 0, 0, 0};
  {  // k = 1: [0, 1/2], node 1/4, weight 4/3
    const T r[4] = {T(0.5) * dq[2], g1_2 - g1_0, g2_2 - g2_0 + T(0.5) * dap,
                    T(0.5) * v_[1] * dq[3]};
    T o[4];
    sign_A2(u_[1], v_[1], r, P, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) V[c] += T(4.0 / 3.0) * o[c];
  }
  {  // k = 2: [1/2, 1], node 3/4, weight 4/3
    const T r[4] = {T(0.5) * dq[2], g1_4 - g1_2, g2_4 - g2_2 + T(0.5) * dap,
                    T(0.5) * v_[3] * dq[3]};
    T o[4];
    sign_A2(u_[3], v_[3], r, P, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) V[c] += T(4.0 / 3.0) * o[c];
  }
  {  // k = 3: [0, 1], node 1/2, weight -1/3
    const T r[4] = {dq[2], g1_4 - g1_0, g2_4 - g2_0 + dap, v_[2] * dq[3]};
    T o[4];
    sign_A2(u_[2], v_[2], r, P, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) V[c] -= T(1.0 / 3.0) * o[c];
  }
  const T vbar = T(2.0 / 3.0) * (v_[1] + v_[3]) - T(1.0 / 3.0) * v_[2];
  const T G0 = dq[2];
  const T G1 = g1_4 - g1_0;
  const T G2 = g2_4 - g2_0 + dap;
  const T G3 = vbar * dq[3];
  Dm[0] = T(0.5) * (G0 - V[0]);
  Dp[0] = T(0.5) * (G0 + V[0]);
  Dm[1] = T(0.5) * (G1 - V[1]);
  Dp[1] = T(0.5) * (G1 + V[1]);
  Dm[2] = T(0.5) * (G2 - V[2]);
  Dp[2] = T(0.5) * (G2 + V[2]);
  Dm[3] = T(0.5) * (G3 - V[3]);
  Dp[3] = T(0.5) * (G3 + V[3]);
}

}  // namespace fv
