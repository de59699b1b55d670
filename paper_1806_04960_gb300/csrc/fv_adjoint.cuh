// Reverse-mode (adjoint) versions of the per-cell and per-face functions of
// fv_model.cuh, for the discrete adjoint of one time step with frozen dt,
// levels K_i and branch decisions (the limiter's active factor, sign(),
// |.|, the order switch and the admissibility fallback are taken as in the
// forward evaluation at the same inputs).  Each *_adj function recomputes the
// forward values it needs from the same inputs and ADDS the input adjoints
// (lambda) for the given output adjoints.
#pragma once

#include "fv_model.cuh"

namespace fv {

// u = mu / m, v = mv / m with r = 1/m.
template <typename T>
__host__ __device__ __forceinline__ void velocity_adj(T m, T mu, T mv, T lu, T lv, T& lm, T& lmu,
                                                      T& lmv) {
  const T r = rcp(m);
  lmu += lu * r;
  lmv += lv * r;
  const T lr = lu * mu + lv * mv;
  lm -= lr * r * r;
}

template <typename T>
__host__ __device__ __forceinline__ T sgn_frozen(T x) {
  return x > T(0) ? T(1) : (x < T(0) ? T(-1) : T(0));
}

// Adjoint of xface(qm, qp, dq) for output adjoints lDm, lDp: adds to lqm, lqp
// (the caller formed dq from qm, qp and their equilibrium parts; the dq
// adjoint is returned separately in ldq).
template <typename T>
__host__ __device__ __forceinline__ void xface_adj(const T qm[4], const T qp[4], const T dq[4], const Phys<T>& P,
                                   const T lDm[4], const T lDp[4], T lqm[4], T lqp[4], T ldq[4]) {
  const T s_gl[3] = {T(0.5 - 0.38729833462074168852), T(0.5), T(0.5 + 0.38729833462074168852)};
  const T w_gl[3] = {T(5.0 / 18.0), T(8.0 / 18.0), T(5.0 / 18.0)};
  // D- = (F - V)/2, D+ = (F + V)/2
  T lF[4], lV[4];
  for (int c = 0; c < 4; ++c) {
    lF[c] = T(0.5) * (lDm[c] + lDp[c]);
    lV[c] = T(0.5) * (lDp[c] - lDm[c]);
  }
  const T dr = dq[0] - P.rho0 * dq[3];
  T ldr = T(0);
  // F0 = dq1; F1 = qp1 up - qm1 um + c2 dr; F2 = qp1 vp - qm1 vm; F3 = ubar dq3
  ldq[1] += lF[0];
  {
    const Vel<T> ep = velocity(qp[0], qp[1], qp[2]);
    const Vel<T> em = velocity(qm[0], qm[1], qm[2]);
    lqp[1] += lF[1] * ep.u + lF[2] * ep.v;
    lqm[1] -= lF[1] * em.u + lF[2] * em.v;
    T lup = lF[1] * qp[1], lvp = lF[2] * qp[1];
    T lum = -lF[1] * qm[1], lvm = -lF[2] * qm[1];
    velocity_adj(qp[0], qp[1], qp[2], lup, lvp, lqp[0], lqp[1], lqp[2]);
    velocity_adj(qm[0], qm[1], qm[2], lum, lvm, lqm[0], lqm[1], lqm[2]);
    ldr += lF[1] * P.c2;
  }
  // ubar = sum w u_k; F3 = ubar dq3
  T ubar = 0;
  for (int k = 0; k < 3; ++k) {
    const Vel<T> w = velocity(qm[0] + s_gl[k] * dq[0], qm[1] + s_gl[k] * dq[1], qm[2] + s_gl[k] * dq[2]);
    ubar += w_gl[k] * w.u;
  }
  ldq[3] += lF[3] * ubar;
  const T lubar = lF[3] * dq[3];
  for (int k = 0; k < 3; ++k) {
    const T m = qm[0] + s_gl[k] * dq[0];
    const T mu = qm[1] + s_gl[k] * dq[1];
    const T mv = qm[2] + s_gl[k] * dq[2];
    const Vel<T> w = velocity(m, mu, mv);
    const T g0 = w_gl[k] * lV[0], g1 = w_gl[k] * lV[1], g2 = w_gl[k] * lV[2], g3 = w_gl[k] * lV[3];
    if (sizeof(T) == 8 && abs_lt(w.u, P.c)) {
      // FP64 (its pipe bounds the reverse face kernel; the float kernel, bound
      // by its registers, keeps the general form): the subsonic closed form of
      // xface_scalar: e = d2 - u d1, Pk = c dr + (u / c) e,
      // a5 - a1 = e + u dr, r0 = Pk + |u| rho0 d4
      const T sua = sgn_frozen(w.u), la = sua * w.u;
      const T e = dq[1] - w.u * dq[0];
      const T Pk = P.c * dr + (w.u * P.inv_c) * e;
      const T r0 = Pk + la * P.rho0 * dq[3];
      const T w2 = dq[2] - w.v * dr;
      // V0 += w r0; V1 += w (u r0 + c (e + u dr)); V2 += w (v Pk + la w2); V3 += w la dq3
      const T lr0 = g0 + g1 * w.u;
      T lu = g1 * r0 + w_gl[k] * lubar;
      const T lamd = g1 * P.c;
      T lv = g2 * Pk;
      const T lPk = lr0 + g2 * w.v;
      const T lla = lr0 * P.rho0 * dq[3] + g2 * w2 + g3 * dq[3];
      ldq[3] += lr0 * la * P.rho0 + g3 * la;
      const T lw2 = g2 * la;
      // a5 - a1 = e + u dr and Pk = c dr + (u / c) e
      const T le = lamd + lPk * w.u * P.inv_c;
      lu += lamd * dr + lPk * P.inv_c * e;
      ldr += lamd * w.u + lPk * P.c;
      // e = d2 - u d1; w2 = d3 - v dr; la = |u|
      ldq[1] += le;
      lu -= le * dq[0];
      ldq[0] -= le * w.u;
      ldq[2] += lw2;
      lv -= lw2 * dr;
      ldr -= lw2 * w.v;
      lu += lla * sua;
      T lm = 0, lmu = 0, lmv = 0;
      velocity_adj(m, mu, mv, lu, lv, lm, lmu, lmv);
      lqm[0] += lm;
      lqm[1] += lmu;
      lqm[2] += lmv;
      ldq[0] += s_gl[k] * lm;
      ldq[1] += s_gl[k] * lmu;
      ldq[2] += s_gl[k] * lmv;
      continue;
    }
    const T uc = w.u * P.inv_c;
    const T w1 = T(0.5) * ((T(1) + uc) * dq[0] - dq[1] * P.inv_c - P.rho0 * dq[3]);
    const T w5 = T(0.5) * ((T(1) - uc) * dq[0] + dq[1] * P.inv_c - P.rho0 * dq[3]);
    const T w2 = dq[2] - w.v * dr;
    const T su1 = sgn_frozen(w.u - P.c), su5 = sgn_frozen(w.u + P.c), sua = sgn_frozen(w.u);
    const T l1 = su1 * (w.u - P.c), l5 = su5 * (w.u + P.c), la = sua * w.u;
    const T a1 = l1 * w1, a5 = l5 * w5;
    const T Pk = a1 + a5;
    const T r0 = Pk + la * P.rho0 * dq[3];
    // V0 += w r0; V1 += w (u r0 + c (a5 - a1)); V2 += w (v Pk + la w2); V3 += w la dq3
    T lu = g1 * r0 + w_gl[k] * lubar;
    T lv = g2 * Pk;
    const T lr0 = g0 + g1 * w.u;
    T la1 = -g1 * P.c, la5 = g1 * P.c;
    T lPk = lr0 + g2 * w.v;
    T lla = lr0 * P.rho0 * dq[3] + g2 * w2 + g3 * dq[3];
    ldq[3] += lr0 * la * P.rho0 + g3 * la;
    T lw2 = g2 * la;
    la1 += lPk;
    la5 += lPk;
    const T ll1 = la1 * w1, lw1 = la1 * l1;
    const T ll5 = la5 * w5, lw5 = la5 * l5;
    lu += ll1 * su1 + ll5 * su5 + lla * sua;
    // w2 = dq2 - v dr
    ldq[2] += lw2;
    lv -= lw2 * dr;
    ldr -= lw2 * w.v;
    // w1, w5
    const T luc = T(0.5) * (lw1 - lw5) * dq[0];
    ldq[0] += T(0.5) * (lw1 * (T(1) + uc) + lw5 * (T(1) - uc));
    ldq[1] += T(0.5) * (-lw1 + lw5) * P.inv_c;
    ldq[3] -= T(0.5) * (lw1 + lw5) * P.rho0;
    lu += luc * P.inv_c;
    T lm = 0, lmu = 0, lmv = 0;
    velocity_adj(m, mu, mv, lu, lv, lm, lmu, lmv);
    lqm[0] += lm;
    lqm[1] += lmu;
    lqm[2] += lmv;
    ldq[0] += s_gl[k] * lm;
    ldq[1] += s_gl[k] * lmu;
    ldq[2] += s_gl[k] * lmv;
  }
  // dr = dq0 - rho0 dq3
  ldq[0] += ldr;
  ldq[3] -= ldr * P.rho0;
}

// Adjoint of sign_A2(u, v, r) with frozen signs: adds to lu, lv, lr.
template <typename T>
__host__ __device__ __forceinline__ void sign_A2_adj(T u, T v, const T r[4], const Phys<T>& P,
                                                     const T lo[4], T& lu, T& lv, T lr[4]) {
  if (sizeof(T) == 8 && abs_lt(v, P.c)) {
    // FP64, as in xface_adj: the subsonic closed form of sign_A2: rr = rho0 r3, D = r0 - rr,
    // Pk = (r2 - v r0) / c, o0 = Pk + s3 rr; out = (o0, u Pk + s3 (r1 - u D),
    // v o0 + c D, s3 r3)
    const T s3 = sgn_frozen(v);
    const T rr = P.rho0 * r[3], D = r[0] - rr;
    const T Pk = (r[2] - v * r[0]) * P.inv_c;
    const T o0 = Pk + s3 * rr;
    const T lo0 = lo[0] + lo[2] * v;
    T lD = lo[2] * P.c;
    lv += lo[2] * o0;
    lu += lo[1] * Pk;
    const T lt = lo[1] * s3;
    lr[1] += lt;
    lu -= lt * D;
    lD -= lt * u;
    const T lPk = lo[1] * u + lo0;
    const T lrr = lo0 * s3 - lD;
    lr[3] += lo[3] * s3 + lrr * P.rho0;
    lr[2] += lPk * P.inv_c;
    lv -= lPk * P.inv_c * r[0];
    lr[0] += lD - lPk * P.inv_c * v;
    return;
  }
  const T vc = v * P.inv_c;
  const T w1 = T(0.5) * ((T(1) + vc) * r[0] - r[2] * P.inv_c - P.rho0 * r[3]);
  const T w5 = T(0.5) * ((T(1) - vc) * r[0] + r[2] * P.inv_c - P.rho0 * r[3]);
  const T w2 = r[1] - u * (r[0] - P.rho0 * r[3]);
  const T s1 = sgn_frozen(v - P.c), s5 = sgn_frozen(v + P.c), s3 = sgn_frozen(v);
  const T a1 = s1 * w1, a5 = s5 * w5;
  const T Pk = a1 + a5;
  const T srho = s3 * P.rho0 * r[3];
  // out0 = Pk + srho; out1 = u Pk + s3 w2; out2 = v (Pk + srho) + c (a5 - a1); out3 = s3 r3
  T lPk = lo[0] + lo[1] * u + lo[2] * v;
  T lsrho = lo[0] + lo[2] * v;
  lu += lo[1] * Pk;
  lv += lo[2] * (Pk + srho);
  T la1 = lPk - lo[2] * P.c, la5 = lPk + lo[2] * P.c;
  const T lw2 = lo[1] * s3;
  lr[3] += lo[3] * s3 + lsrho * s3 * P.rho0;
  const T lw1 = la1 * s1, lw5 = la5 * s5;
  // w2 = r1 - u (r0 - rho0 r3)
  lr[1] += lw2;
  lu -= lw2 * (r[0] - P.rho0 * r[3]);
  lr[0] -= lw2 * u;
  lr[3] += lw2 * u * P.rho0;
  // w1, w5
  const T lvc = T(0.5) * (lw1 - lw5) * r[0];
  lr[0] += T(0.5) * (lw1 * (T(1) + vc) + lw5 * (T(1) - vc));
  lr[2] += T(0.5) * (-lw1 + lw5) * P.inv_c;
  lr[3] -= T(0.5) * (lw1 + lw5) * P.rho0;
  lv += lvc * P.inv_c;
}

// Adjoint of yface(qm, qp, dq, dap): adds to lqm, lqp, ldq, ldap.
template <typename T>
__host__ __device__ __forceinline__ void yface_adj(const T qm[4], const T qp[4], const T dq[4], T dap,
                                   const Phys<T>& P, const T lDm[4], const T lDp[4], T lqm[4],
                                   T lqp[4], T ldq[4], T& ldap) {
  // forward values
  T m_[5], mu_[5], mv_[5], u_[5], v_[5];
  for (int k = 1; k < 4; ++k) {
    const T s = T(0.25 * k);
    m_[k] = qm[0] + s * dq[0];
    mu_[k] = qm[1] + s * dq[1];
    mv_[k] = qm[2] + s * dq[2];
    const Vel<T> w = velocity(m_[k], mu_[k], mv_[k]);
    u_[k] = w.u;
    v_[k] = w.v;
  }
  {
    const Vel<T> a = velocity(qm[0], qm[1], qm[2]);
    const Vel<T> b = velocity(qp[0], qp[1], qp[2]);
    m_[0] = qm[0]; mu_[0] = qm[1]; mv_[0] = qm[2]; u_[0] = a.u; v_[0] = a.v;
    m_[4] = qp[0]; mu_[4] = qp[1]; mv_[4] = qp[2]; u_[4] = b.u; v_[4] = b.v;
  }
  T lF[4], lV[4];
  for (int c = 0; c < 4; ++c) {
    lF[c] = T(0.5) * (lDm[c] + lDp[c]);
    lV[c] = T(0.5) * (lDp[c] - lDm[c]);
  }
  T lu[5] = {0, 0, 0, 0, 0}, lv[5] = {0, 0, 0, 0, 0}, lmu[5] = {0, 0, 0, 0, 0}, lmv[5] = {0, 0, 0, 0, 0};
  T lg1[5] = {0, 0, 0, 0, 0}, lg2[5] = {0, 0, 0, 0, 0};
  // G0 = dq2; G1 = g1_4 - g1_0; G2 = g2_4 - g2_0 + dap; G3 = vbar dq3
  ldq[2] += lF[0];
  lg1[4] += lF[1];
  lg1[0] -= lF[1];
  lg2[4] += lF[2];
  lg2[0] -= lF[2];
  ldap += lF[2];
  const T vbar = T(2.0 / 3.0) * (v_[1] + v_[3]) - T(1.0 / 3.0) * v_[2];
  ldq[3] += lF[3] * vbar;
  const T lvbar = lF[3] * dq[3];
  lv[1] += T(2.0 / 3.0) * lvbar;
  lv[3] += T(2.0 / 3.0) * lvbar;
  lv[2] -= T(1.0 / 3.0) * lvbar;
  // three Romberg terms: (node, a, b, weight, half)
  const int node[3] = {1, 3, 2}, na[3] = {0, 2, 0}, nb[3] = {2, 4, 4};
  const T wt[3] = {T(4.0 / 3.0), T(4.0 / 3.0), T(-1.0 / 3.0)};
  const T fr[3] = {T(0.5), T(0.5), T(1)};
  for (int k = 0; k < 3; ++k) {
    const int n = node[k], a = na[k], b = nb[k];
    const T g1a = mu_[a] * v_[a], g2a = mv_[a] * v_[a], g1b = mu_[b] * v_[b], g2b = mv_[b] * v_[b];
    const T r[4] = {fr[k] * dq[2], g1b - g1a, g2b - g2a + fr[k] * dap, fr[k] * v_[n] * dq[3]};
    const T lo[4] = {wt[k] * lV[0], wt[k] * lV[1], wt[k] * lV[2], wt[k] * lV[3]};
    T lr[4] = {0, 0, 0, 0};
    sign_A2_adj(u_[n], v_[n], r, P, lo, lu[n], lv[n], lr);
    ldq[2] += fr[k] * lr[0];
    lg1[b] += lr[1];
    lg1[a] -= lr[1];
    lg2[b] += lr[2];
    lg2[a] -= lr[2];
    ldap += fr[k] * lr[2];
    lv[n] += fr[k] * lr[3] * dq[3];
    ldq[3] += fr[k] * lr[3] * v_[n];
  }
  // g1 = mu v, g2 = mv v at nodes 0, 2, 4
  for (int k = 0; k < 5; k += 2) {
    lmu[k] += lg1[k] * v_[k];
    lmv[k] += lg2[k] * v_[k];
    lv[k] += lg1[k] * mu_[k] + lg2[k] * mv_[k];
  }
  // node velocities back to states
  for (int k = 0; k < 5; ++k) {
    T lm = 0, lmuk = lmu[k], lmvk = lmv[k];
    velocity_adj(m_[k], mu_[k], mv_[k], lu[k], lv[k], lm, lmuk, lmvk);
    if (k == 0) {
      lqm[0] += lm; lqm[1] += lmuk; lqm[2] += lmvk;
    } else if (k == 4) {
      lqp[0] += lm; lqp[1] += lmuk; lqp[2] += lmvk;
    } else {
      const T s = T(0.25 * k);
      lqm[0] += lm; lqm[1] += lmuk; lqm[2] += lmvk;
      ldq[0] += s * lm; ldq[1] += s * lmuk; ldq[2] += s * lmvk;
    }
  }
}


// Adjoint of interior_terms for output adjoints lIx, lIy: adds to the face
// fluctuation states, the centre state, the equilibrium masses and the limited
// alpha slopes.
template <typename T>
__host__ __device__ __forceinline__ void interior_terms_adj(const T fW[4], const T fE[4], const T fS[4],
                                            const T fN[4], const T base[4], T mEc, T mES, T mEN,
                                            T dax, T day, T dx, T dy, const Phys<T>& P,
                                            const T lIx[4], const T lIy[4], T lfW[4], T lfE[4],
                                            T lfS[4], T lfN[4], T lbase[4], T& lmEc, T& lmES,
                                            T& lmEN, T& ldax, T& lday) {
  const Vel<T> vE = velocity(mEc + fE[0], fE[1], fE[2]);
  const Vel<T> vW = velocity(mEc + fW[0], fW[1], fW[2]);
  const Vel<T> vN = velocity(mEN + fN[0], fN[1], fN[2]);
  const Vel<T> vS = velocity(mES + fS[0], fS[1], fS[2]);
  const Vel<T> vc = velocity(mEc + base[0], base[1], base[2]);
  T luE = 0, lvE = 0, luW = 0, lvW = 0, lvN = 0, lvS = 0, luN = 0, luS = 0, luc = 0, lvc = 0;
  // Ix0 = fE1 - fW1
  lfE[1] += lIx[0];
  lfW[1] -= lIx[0];
  // Ix1 = fE1 uE - fW1 uW + c2 ((fE0 - fW0) - rho0 (fE3 - fW3))
  lfE[1] += lIx[1] * vE.u;
  luE += lIx[1] * fE[1];
  lfW[1] -= lIx[1] * vW.u;
  luW -= lIx[1] * fW[1];
  lfE[0] += P.c2 * lIx[1];
  lfW[0] -= P.c2 * lIx[1];
  lfE[3] -= P.c2 * P.rho0 * lIx[1];
  lfW[3] += P.c2 * P.rho0 * lIx[1];
  // Ix2 = fE1 vE - fW1 vW
  lfE[1] += lIx[2] * vE.v;
  lvE += lIx[2] * fE[1];
  lfW[1] -= lIx[2] * vW.v;
  lvW -= lIx[2] * fW[1];
  // Ix3 = dx uc dax
  luc += lIx[3] * dx * dax;
  ldax += lIx[3] * dx * vc.u;
  // Iy0 = fN2 - fS2
  lfN[2] += lIy[0];
  lfS[2] -= lIy[0];
  // Iy1 = fN1 vN - fS1 vS
  lfN[1] += lIy[1] * vN.v;
  lvN += lIy[1] * fN[1];
  lfS[1] -= lIy[1] * vS.v;
  lvS -= lIy[1] * fS[1];
  // Iy2 = fN2 vN - fS2 vS + c2 ((fN0 - fS0) - rho0 (fN3 - fS3)) + g dy base0
  lfN[2] += lIy[2] * vN.v;
  lvN += lIy[2] * fN[2];
  lfS[2] -= lIy[2] * vS.v;
  lvS -= lIy[2] * fS[2];
  lfN[0] += P.c2 * lIy[2];
  lfS[0] -= P.c2 * lIy[2];
  lfN[3] -= P.c2 * P.rho0 * lIy[2];
  lfS[3] += P.c2 * P.rho0 * lIy[2];
  lbase[0] += P.g * dy * lIy[2];
  // Iy3 = dy vc day
  lvc += lIy[3] * dy * day;
  lday += lIy[3] * dy * vc.v;
  T lm;
  lm = 0;
  velocity_adj(mEc + fE[0], fE[1], fE[2], luE, lvE, lm, lfE[1], lfE[2]);
  lfE[0] += lm;
  lmEc += lm;
  lm = 0;
  velocity_adj(mEc + fW[0], fW[1], fW[2], luW, lvW, lm, lfW[1], lfW[2]);
  lfW[0] += lm;
  lmEc += lm;
  lm = 0;
  velocity_adj(mEN + fN[0], fN[1], fN[2], luN, lvN, lm, lfN[1], lfN[2]);
  lfN[0] += lm;
  lmEN += lm;
  lm = 0;
  velocity_adj(mES + fS[0], fS[1], fS[2], luS, lvS, lm, lfS[1], lfS[2]);
  lfS[0] += lm;
  lmES += lm;
  lm = 0;
  velocity_adj(mEc + base[0], base[1], base[2], luc, lvc, lm, lbase[1], lbase[2]);
  lbase[0] += lm;
  lmEc += lm;
}

// Adjoint of recon_core.  Inputs are those of the forward call (fWi..fNi are
// the neighbour fluctuations before recon_core overwrote them); output
// adjoints: lfW..lfN (face states), lbase (centre), lgxa (limited alpha
// slopes).  Adds to lQf, lfWi..lfNi, lmx, lmn, laE, lmEc.  The limiter's
// active factor (the first candidate attaining the minimum), the order switch
// and the admissibility fallback are taken as in the forward evaluation.
template <typename T>
__host__ __device__ __forceinline__ void recon_core_adj(const T Qf[4], const T fWi[4], const T fEi[4],
                                        const T fSi[4], const T fNi[4], const T mx[4],
                                        const T mn[4], T aE, T mEc, T mES, T mEN, T rEc,
                                        const Phys<T>& P, const ReconConsts<T>& R,
                                        const T lfW[4], const T lfE[4], const T lfS[4],
                                        const T lfN[4], const T lbase[4], const T lgxa[2],
                                        T lQf[4], T lfWi[4], T lfEi[4], T lfSi[4], T lfNi[4],
                                        T lmx[4], T lmn[4], T& laE, T& lmEc) {
  T gx[4], gy[4];
  for (int v = 0; v < 4; ++v) {
    gx[v] = (fEi[v] - fWi[v]) * R.inv_2dx;
    gy[v] = (fNi[v] - fSi[v]) * R.inv_2dy;
  }
  // limiter, recording the active candidate
  T psi = T(1);
  int act_v = -1, act_dir = 0, act_pm = 0;
  for (int v = 0; v < 4; ++v) {
    const T up = mx[v] - Qf[v], dn = mn[v] - Qf[v];
    for (int dir = 0; dir < 2; ++dir) {
      const T d = dir == 0 ? R.half_dx * gx[v] : R.half_dy * gy[v];
      const T ad = tabs(d);
      if (ad > R.eta[v]) {
        const T inv = rcp(d);
        const T ramp = fmin(T(1), (ad - R.eta[v]) * R.inv_eta[v]);
        const T phi_p = fmin(T(1), (d > T(0) ? up : dn) * inv);
        const T phi_m = fmin(T(1), -(d > T(0) ? dn : up) * inv);
        const T cp = T(1) - ramp * (T(1) - phi_p);
        const T cm = T(1) - ramp * (T(1) - phi_m);
        if (cp < psi) {
          psi = cp;
          act_v = v; act_dir = dir; act_pm = 1;
        }
        if (cm < psi) {
          psi = cm;
          act_v = v; act_dir = dir; act_pm = -1;
        }
      }
    }
  }
  const bool sw = aE <= R.ten_eps;
  if (sw) psi = T(0);
  T dtQ[4] = {0, 0, 0, 0};
  T u = 0, v = 0, dmE = 0;
  T sx[4], sy[4];
  for (int c = 0; c < 4; ++c) {
    sx[c] = psi * gx[c];
    sy[c] = psi * gy[c];
  }
  if (!sw) {
    const Vel<T> vel = velocity(mEc + Qf[0], Qf[1], Qf[2]);
    u = vel.u;
    v = vel.v;
    dmE = aE * (-P.kappa * rEc);
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
  T base[4], oW[4], oE[4], oS[4], oN[4];
  for (int c = 0; c < 4; ++c) {
    base[c] = Qf[c] + R.half_dt * dtQ[c];
    const T sxh = psi * gx[c] * R.half_dx, syh = psi * gy[c] * R.half_dy;
    oW[c] = base[c] - sxh;
    oE[c] = base[c] + sxh;
    oS[c] = base[c] - syh;
    oN[c] = base[c] + syh;
  }
  const bool ok = (mEc + oW[0] > T(0)) && (aE + oW[3] > T(0)) && (mEc + oE[0] > T(0)) &&
                  (aE + oE[3] > T(0)) && (mES + oS[0] > T(0)) && (aE + oS[3] > T(0)) &&
                  (mEN + oN[0] > T(0)) && (aE + oN[3] > T(0)) && (mEc + base[0] > T(0)) &&
                  (aE + base[3] > T(0));
  if (!ok) {
    // first order: every output state is Qf, the slopes are zero
    for (int c = 0; c < 4; ++c) lQf[c] += lfW[c] + lfE[c] + lfS[c] + lfN[c] + lbase[c];
    return;
  }
  T lb[4], lgx[4], lgy[4];
  T lpsi = lgxa[0] * gx[3] + lgxa[1] * gy[3];
  for (int c = 0; c < 4; ++c) {
    lb[c] = lbase[c] + lfW[c] + lfE[c] + lfS[c] + lfN[c];
    const T lsxh = lfE[c] - lfW[c], lsyh = lfN[c] - lfS[c];
    lpsi += lsxh * gx[c] * R.half_dx + lsyh * gy[c] * R.half_dy;
    lgx[c] = psi * R.half_dx * lsxh;
    lgy[c] = psi * R.half_dy * lsyh;
    lQf[c] += lb[c];
  }
  lgx[3] += psi * lgxa[0];
  lgy[3] += psi * lgxa[1];
  if (!sw) {
    T ldt[4];
    for (int c = 0; c < 4; ++c) ldt[c] = R.half_dt * lb[c];
    const T la1 = -ldt[0], lb1 = -ldt[0], la2 = -ldt[1], lb2 = -ldt[1];
    const T la3 = -ldt[2], lb3 = -ldt[2], la4 = -ldt[3], lb4 = -ldt[3];
    T lsx[4] = {0, 0, 0, 0}, lsy[4] = {0, 0, 0, 0};
    T lu = 0, lv = 0, ldmE = 0;
    const T uv = u * v;
    lsx[1] += la1;
    lsx[0] += la2 * (P.c2 - u * u);
    lsx[1] += la2 * T(2) * u;
    lsx[3] -= la2 * P.k0;
    lu += la2 * (T(-2) * u * sx[0] + T(2) * sx[1]);
    lsx[0] -= la3 * uv;
    lsx[1] += la3 * v;
    lsx[2] += la3 * u;
    lu += la3 * (-v * sx[0] + sx[2]);
    lv += la3 * (-u * sx[0] + sx[1]);
    lsx[3] += la4 * u;
    lu += la4 * sx[3];
    lsy[2] += lb1;
    lsy[0] -= lb2 * uv;
    lsy[1] += lb2 * v;
    lsy[2] += lb2 * u;
    lu += lb2 * (-v * sy[0] + sy[2] - v * dmE);
    lv += lb2 * (-u * sy[0] + sy[1] - u * dmE);
    ldmE -= lb2 * uv;
    lsy[0] += lb3 * (P.c2 - v * v);
    lsy[2] += lb3 * T(2) * v;
    lsy[3] -= lb3 * P.k0;
    lv += lb3 * (T(-2) * v * sy[0] + T(2) * sy[2] - T(2) * v * dmE);
    ldmE -= lb3 * v * v;
    lQf[0] += lb3 * P.g;
    lsy[3] += lb4 * v;
    lv += lb4 * sy[3];
    laE += ldmE * (-P.kappa * rEc);
    T lm = 0;
    velocity_adj(mEc + Qf[0], Qf[1], Qf[2], lu, lv, lm, lQf[1], lQf[2]);
    lQf[0] += lm;
    lmEc += lm;
    for (int c = 0; c < 4; ++c) {
      lpsi += lsx[c] * gx[c] + lsy[c] * gy[c];
      lgx[c] += psi * lsx[c];
      lgy[c] += psi * lsy[c];
    }
    // limiter: psi = 1 - ramp (1 - phi) of the active candidate (the loop
    // keeps every array index a compile-time constant)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      if (w != act_v) continue;
      const T up = mx[w] - Qf[w], dn = mn[w] - Qf[w];
      const T d = act_dir == 0 ? R.half_dx * gx[w] : R.half_dy * gy[w];
      const T ad = tabs(d);
      const T inv = rcp(d);
      const T rraw = (ad - R.eta[w]) * R.inv_eta[w];
      const T ramp = fmin(T(1), rraw);
      const bool pos = d > T(0);
      const T Bv = act_pm > 0 ? (pos ? up : dn) : -(pos ? dn : up);
      const T x = Bv * inv;
      const T phi = fmin(T(1), x);
      const T lramp = -lpsi * (T(1) - phi);
      const T lphi = lpsi * ramp;
      T ld = 0;
      if (rraw < T(1)) ld += sgn_frozen(d) * lramp * R.inv_eta[w];
      if (x < T(1)) {
        const T lB = lphi * inv;
        ld -= lphi * x * inv;
        T lup = 0, ldn = 0;
        if (act_pm > 0) {
          if (pos) lup += lB; else ldn += lB;
        } else {
          if (pos) ldn -= lB; else lup -= lB;
        }
        lmx[w] += lup;
        lmn[w] += ldn;
        lQf[w] -= lup + ldn;
      }
      if (act_dir == 0) lgx[w] += R.half_dx * ld;
      else lgy[w] += R.half_dy * ld;
    }
  }
  for (int c = 0; c < 4; ++c) {
    lfEi[c] += lgx[c] * R.inv_2dx;
    lfWi[c] -= lgx[c] * R.inv_2dx;
    lfNi[c] += lgy[c] * R.inv_2dy;
    lfSi[c] -= lgy[c] * R.inv_2dy;
  }
}

}  // namespace fv
