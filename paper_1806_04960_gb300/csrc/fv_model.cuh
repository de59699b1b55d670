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

// Reciprocal: IEEE in double; the fast hardware reciprocal in float on the
// device (relative error ~1e-7, inside the float path's stated tolerance).
template <typename T>
__host__ __device__ __forceinline__ T rcp(T x) {
  return T(1) / x;
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
  const T s_gl[3] = {T(0.5 - 0.38729833462074168852), T(0.5), T(0.5 + 0.38729833462074168852)};
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
// dap: jump of alpha p = c2 (m - rho0 alpha) from qm to qp, formed by the
// caller so that it is exactly zero between two states of one rest profile.
template <typename T>
__host__ __device__ __forceinline__ void yface(const T qm[4], const T qp[4], const T dq[4],
                                               T dap, const Phys<T>& P, T Dm[4], T Dp[4]) {
  // nodes s = 0, 1/4, 1/2, 3/4, 1 (interior nodes on the path, exact endpoints)
  T mu_[5], mv_[5], u_[5], v_[5];
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    const T s = T(0.25 * k);
    const T m = qm[0] + s * dq[0];
    mu_[k] = qm[1] + s * dq[1];
    mv_[k] = qm[2] + s * dq[2];
    const Vel<T> w = velocity(m, mu_[k], mv_[k]);
    u_[k] = w.u;
    v_[k] = w.v;
  }
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
    const T up = mx[v] - Qf[v], dn = mn[v] - Qf[v];
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      // faces at -h/2 and +h/2 see increments -d and +d
      const T d = dir == 0 ? R.half_dx * gx[v] : R.half_dy * gy[v];
      const T ad = tabs(d);
      if (ad > R.eta[v]) {
        const T inv = rcp(d);
        const T ramp = fmin(T(1), (ad - R.eta[v]) * R.inv_eta[v]);
        // face with increment +d: bound up if d > 0, dn if d < 0; face with -d: the other
        const T phi_p = fmin(T(1), (d > T(0) ? up : dn) * inv);
        const T phi_m = fmin(T(1), -(d > T(0) ? dn : up) * inv);
        psi = fmin(psi, T(1) - ramp * (T(1) - phi_p));
        psi = fmin(psi, T(1) - ramp * (T(1) - phi_m));
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
  const bool ok = (mEc + fW[0] > T(0)) && (aE + fW[3] > T(0)) && (mEc + fE[0] > T(0)) &&
                  (aE + fE[3] > T(0)) && (mES + fS[0] > T(0)) && (aE + fS[3] > T(0)) &&
                  (mEN + fN[0] > T(0)) && (aE + fN[3] > T(0)) && (mEc + base[0] > T(0)) &&
                  (aE + base[3] > T(0));
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
template <typename T>
__host__ __device__ __forceinline__ void interior_terms(const T fW[4], const T fE[4],
                                                        const T fS[4], const T fN[4],
                                                        const T base[4], T mEc, T mES, T mEN,
                                                        T dax, T day, T dx, T dy,
                                                        const Phys<T>& P, T Ix[4], T Iy[4]) {
  const Vel<T> vE = velocity(mEc + fE[0], fE[1], fE[2]);
  const Vel<T> vW = velocity(mEc + fW[0], fW[1], fW[2]);
  const Vel<T> vN = velocity(mEN + fN[0], fN[1], fN[2]);
  const Vel<T> vS = velocity(mES + fS[0], fS[1], fS[2]);
  const Vel<T> vc = velocity(mEc + base[0], base[1], base[2]);
  Ix[0] = fE[1] - fW[1];
  Ix[1] = (fE[1] * vE.u - fW[1] * vW.u) + P.c2 * ((fE[0] - fW[0]) - P.rho0 * (fE[3] - fW[3]));
  Ix[2] = fE[1] * vE.v - fW[1] * vW.v;
  Ix[3] = dx * vc.u * dax;
  Iy[0] = fN[2] - fS[2];
  Iy[1] = fN[1] * vN.v - fS[1] * vS.v;
  Iy[2] = (fN[2] * vN.v - fS[2] * vS.v) + P.c2 * ((fN[0] - fS[0]) - P.rho0 * (fN[3] - fS[3])) +
          P.g * dy * base[0];
  Iy[3] = dy * vc.v * day;
}

}  // namespace fv
