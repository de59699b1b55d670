// First-order y face of Sections 3.2-3.3 (Eq. (SemidiscreteScheme_2)): the
// two states are the cell averages at the cell centres y_j and y_{j+1}, joined
// by the well-balanced path of Eq. (path), Phi(s) = Phi^E(s) + Phi^f(s), with
// Phi^f linear in the fluctuations, alpha^E linear in s and rho^E taken at the
// path's height y(s) = y_j + s dy.  The non-conservative term of a segment
// A -> B is (0, 0, b3, b4) with b3 the fluctuation form of Eq.
// (b^y_3_final): the jump of alpha^E p^f + alpha^f p^E + alpha^f p^f, the
// gravity part g (y_B - y_A) (abar^E rhobar^f + abar^f rhobar^E + abar^f
// rhobar^f) with arithmetic averages, and the alpha^E contact part
// (alpha^E_B - alpha^E_A) p^E(face); b4 = vbar (alpha_B - alpha_A) with the
// node velocity (sub-segments) or the Romberg combination (whole face).  The
// viscosity is the Osher-Romberg sum of Eq. (ViscosityOR).
#pragma once

#include "fv_model.cuh"

namespace fv {

// fa, fb: fluctuations (alpha rho - alpha^E rho^E, alpha rho u, alpha rho v,
// alpha - alpha^E) of the lower and upper cell; aEa, aEb: their alpha^E;
// rq[k], pq[k]: rho^E and p^E at s = k/4 (k = 0..4; k = 2 is the face);
// dy: distance of the two centres.
template <typename T>
__host__ __device__ __forceinline__ void yface_o1(const T fa[4], T aEa, const T fb[4], T aEb,
                                                  const T rq[5], const T pq[5], T dy,
                                                  const Phys<T>& P, T Dm[4], T Dp[4]) {
  T q[5][4], u[5], v[5], ap[5], rf[5], aE[5], af[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const T s = T(0.25 * k);
    aE[k] = aEa + s * (aEb - aEa);
    T f[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) f[c] = fa[c] + s * (fb[c] - fa[c]);
    q[k][0] = aE[k] * rq[k] + f[0];
    q[k][1] = f[1];
    q[k][2] = f[2];
    q[k][3] = aE[k] + f[3];
    const Vel<T> w = velocity(q[k][0], q[k][1], q[k][2]);
    u[k] = w.u;
    v[k] = w.v;
    af[k] = f[3];
    rf[k] = (f[0] - rq[k] * f[3]) / q[k][3];
    const T pf = P.c2 * rf[k];
    ap[k] = aE[k] * pf + af[k] * pq[k] + af[k] * pf;
  }
  const T pE_face = pq[2];
  // b3 of the segment a -> b (node indices), spanning (b - a) / 4 of dy
  auto b3 = [&](int a, int b) -> T {
    const T aEbar = T(0.5) * (aE[a] + aE[b]), afbar = T(0.5) * (af[a] + af[b]);
    const T rEbar = T(0.5) * (rq[a] + rq[b]), rfbar = T(0.5) * (rf[a] + rf[b]);
    return (ap[b] - ap[a]) +
           (aEbar * rfbar + afbar * rEbar + afbar * rfbar) * P.g * (T(0.25 * (b - a)) * dy) +
           (aE[b] - aE[a]) * pE_face;
  };
  T g1[5], g2[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    g1[k] = q[k][1] * v[k];
    g2[k] = q[k][2] * v[k];
  }
  T V[4] = {0, 0, 0, 0};
  {  // [0, 1/2], node 1/4, weight 4/3
    const T r[4] = {q[2][2] - q[0][2], g1[2] - g1[0], g2[2] - g2[0] + b3(0, 2),
                    v[1] * (q[2][3] - q[0][3])};
    T o[4];
    sign_A2(u[1], v[1], r, P, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) V[c] += T(4.0 / 3.0) * o[c];
  }
  {  // [1/2, 1], node 3/4, weight 4/3
    const T r[4] = {q[4][2] - q[2][2], g1[4] - g1[2], g2[4] - g2[2] + b3(2, 4),
                    v[3] * (q[4][3] - q[2][3])};
    T o[4];
    sign_A2(u[3], v[3], r, P, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) V[c] += T(4.0 / 3.0) * o[c];
  }
  {  // [0, 1], node 1/2, weight -1/3
    const T r[4] = {q[4][2] - q[0][2], g1[4] - g1[0], g2[4] - g2[0] + b3(0, 4),
                    v[2] * (q[4][3] - q[0][3])};
    T o[4];
    sign_A2(u[2], v[2], r, P, o);
#pragma unroll
    for (int c = 0; c < 4; ++c) V[c] -= T(1.0 / 3.0) * o[c];
  }
  const T vbar = T(2.0 / 3.0) * (v[1] + v[3]) - T(1.0 / 3.0) * v[2];
  const T G[4] = {q[4][2] - q[0][2], g1[4] - g1[0], g2[4] - g2[0] + b3(0, 4),
                  vbar * (q[4][3] - q[0][3])};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    Dm[c] = T(0.5) * (G[c] - V[c]);
    Dp[c] = T(0.5) * (G[c] + V[c]);
  }
}

}  // namespace fv
