// Host instantiation of the device face solvers (include/fv_model_host.h).
#include <cmath>

#include "fv_adjoint.cuh"
#include "fv_model.cuh"
#include "fv_model_host.h"
#include "fv_order1.cuh"

namespace {
fv::Phys<double> phys(const double* model) {
  fv::Phys<double> P;
  P.rho0 = model[0];
  P.k0 = model[1];
  P.g = model[3];
  P.c2 = model[1] / model[0];
  P.c = std::sqrt(P.c2);
  P.inv_c = 1.0 / P.c;
  P.kappa = model[3] * model[0] / model[1];
  return P;
}
}  // namespace

extern "C" int fv_host_xface(const double* model, const double* qm, const double* qp, double* Dm,
                             double* Dp) {
  if (!model || !qm || !qp || !Dm || !Dp) return 1;
  const double dq[4] = {qp[0] - qm[0], qp[1] - qm[1], qp[2] - qm[2], qp[3] - qm[3]};
  fv::xface<double>(qm, qp, dq, phys(model), Dm, Dp);
  return 0;
}

extern "C" int fv_host_xface_or(const double* model, const double* qm, const double* qp,
                                double* Dm, double* Dp) {
  if (!model || !qm || !qp || !Dm || !Dp) return 1;
  const double dq[4] = {qp[0] - qm[0], qp[1] - qm[1], qp[2] - qm[2], qp[3] - qm[3]};
  fv::xface_or<double>(qm, qp, dq, phys(model), Dm, Dp);
  return 0;
}

extern "C" int fv_host_yface(const double* model, const double* qm, const double* qp, double* Dm,
                             double* Dp) {
  if (!model || !qm || !qp || !Dm || !Dp) return 1;
  const double dq[4] = {qp[0] - qm[0], qp[1] - qm[1], qp[2] - qm[2], qp[3] - qm[3]};
  const fv::Phys<double> P = phys(model);
  fv::yface<double>(qm, qp, dq, P.c2 * (dq[0] - P.rho0 * dq[3]), P, Dm, Dp);
  return 0;
}

extern "C" int fv_host_face_f32(int which, const double* model, const double* qm,
                                const double* qp, int paired, double* Dm, double* Dp) {
  if (!model || !qm || !qp || !Dm || !Dp || which < 0 || which > 1) return 1;
  const fv::Phys<double> Pd = phys(model);
  fv::Phys<float> P;
  P.c = (float)Pd.c;
  P.c2 = (float)Pd.c2;
  P.inv_c = (float)Pd.inv_c;
  P.rho0 = (float)Pd.rho0;
  P.k0 = (float)Pd.k0;
  P.g = (float)Pd.g;
  P.kappa = (float)Pd.kappa;
  float a[4], b[4], dq[4], m[4], p[4];
  for (int c = 0; c < 4; ++c) {
    a[c] = (float)qm[c];
    b[c] = (float)qp[c];
    dq[c] = b[c] - a[c];
  }
  if (which == 0) {
    if (paired) fv::xface_f2(a, b, dq, P, m, p);
    else fv::xface_scalar<float>(a, b, dq, P, m, p);
  } else {
    const float dap = P.c2 * (dq[0] - P.rho0 * dq[3]);
    if (paired) fv::yface_f2(a, b, dq, dap, P, m, p);
    else fv::yface_scalar<float>(a, b, dq, dap, P, m, p);
  }
  for (int c = 0; c < 4; ++c) {
    Dm[c] = m[c];
    Dp[c] = p[c];
  }
  return 0;
}

extern "C" int fv_host_yface_o1(const double* model, const double* fa, double aEa,
                                const double* fb, double aEb, double ya, double dy, double* Dm,
                                double* Dp) {
  if (!model || !fa || !fb || !Dm || !Dp) return 1;
  const fv::Phys<double> P = phys(model);
  double rq[5], pq[5];
  for (int k = 0; k < 5; ++k) {
    rq[k] = P.rho0 * std::exp(-P.kappa * (ya + 0.25 * k * dy));
    pq[k] = P.k0 * (rq[k] / P.rho0 - 1.0);
  }
  fv::yface_o1<double>(fa, aEa, fb, aEb, rq, pq, dy, P, Dm, Dp);
  return 0;
}

// ---------------------------------------------------------------------------
// Forward value and reverse-mode derivative of one per-face or per-cell
// function of the kernels, for finite-difference checks on the host.
// ---------------------------------------------------------------------------
namespace {

fv::ReconConsts<double> recon_consts(const double* model, const double* k) {
  const fv::Phys<double> P = phys(model);
  fv::ReconConsts<double> R;
  R.half_dx = 0.5 * k[0];
  R.half_dy = 0.5 * k[1];
  R.inv_2dx = 1.0 / (2.0 * k[0]);
  R.inv_2dy = 1.0 / (2.0 * k[1]);
  R.half_dt = 0.5 * k[2];
  R.ten_eps = 10.0 * model[4];
  const double eta[4] = {std::ldexp(P.rho0, -20), std::ldexp(P.rho0 * P.c, -10),
                         std::ldexp(P.rho0 * P.c, -10), std::ldexp(1.0, -20)};
  for (int v = 0; v < 4; ++v) {
    R.eta[v] = eta[v];
    R.inv_eta[v] = 1.0 / eta[v];
  }
  return R;
}

}  // namespace

extern "C" int fv_host_adj_check(int which, const double* model, const double* k, const double* in,
                                 const double* lout, double* out, double* lin) {
  if (!model || !in || !out || (lout && !lin)) return 1;
  const fv::Phys<double> P = phys(model);
  if (which == 0 || which == 1) {
    const double* qm = in;
    const double* qp = in + 4;
    const double dq[4] = {qp[0] - qm[0], qp[1] - qm[1], qp[2] - qm[2], qp[3] - qm[3]};
    const double dap = P.c2 * (dq[0] - P.rho0 * dq[3]);
    if (which == 0) fv::xface<double>(qm, qp, dq, P, out, out + 4);
    else fv::yface<double>(qm, qp, dq, dap, P, out, out + 4);
    if (!lout) return 0;
    double lqm[4] = {0, 0, 0, 0}, lqp[4] = {0, 0, 0, 0}, ldq[4] = {0, 0, 0, 0}, ldap = 0.0;
    if (which == 0) fv::xface_adj<double>(qm, qp, dq, P, lout, lout + 4, lqm, lqp, ldq);
    else fv::yface_adj<double>(qm, qp, dq, dap, P, lout, lout + 4, lqm, lqp, ldq, ldap);
    ldq[0] += P.c2 * ldap;
    ldq[3] -= P.c2 * P.rho0 * ldap;
    for (int c = 0; c < 4; ++c) {
      lin[c] = lqm[c] - ldq[c];
      lin[4 + c] = lqp[c] + ldq[c];
    }
    return 0;
  }
  if (!k) return 1;
  if (which == 2) {
    // in: Qf[4], fW[4], fE[4], fS[4], fN[4], mx[4], mn[4], aE; k: dx, dy, dt, rEc, rES, rEN
    // out: fW'[4], fE'[4], fS'[4], fN'[4], base[4], gxa[2]
    const fv::ReconConsts<double> R = recon_consts(model, k);
    const double rEc = k[3], rES = k[4], rEN = k[5];
    const double aE = in[28];
    const double mEc = aE * rEc, mES = aE * rES, mEN = aE * rEN;
    double f[4][4];
    for (int s = 0; s < 4; ++s)
      for (int c = 0; c < 4; ++c) f[s][c] = in[4 + 4 * s + c];
    fv::recon_core<double>(in, f[0], f[1], f[2], f[3], in + 20, in + 24, aE, mEc, mES, mEN, rEc, P,
                           R, out + 16, out + 20);
    for (int s = 0; s < 4; ++s)
      for (int c = 0; c < 4; ++c) out[4 * s + c] = f[s][c];
    if (!lout) return 0;
    for (int x = 0; x < 29; ++x) lin[x] = 0.0;
    double laE = 0.0, lmEc = 0.0;
    fv::recon_core_adj<double>(in, in + 4, in + 8, in + 12, in + 16, in + 20, in + 24, aE, mEc, mES,
                               mEN, rEc, P, R, lout, lout + 4, lout + 8, lout + 12, lout + 16,
                               lout + 20, lin, lin + 4, lin + 8, lin + 12, lin + 16, lin + 20,
                               lin + 24, laE, lmEc);
    lin[28] = laE + rEc * lmEc;
    return 0;
  }
  if (which == 3) {
    // in: fW[4], fE[4], fS[4], fN[4], base[4], aE, dax, day; k: dx, dy, dt, rEc, rES, rEN
    // out: Ix[4], Iy[4]
    const double rEc = k[3], rES = k[4], rEN = k[5];
    const double aE = in[20];
    fv::interior_terms<double>(in, in + 4, in + 8, in + 12, in + 16, aE * rEc, aE * rES, aE * rEN,
                               in[21], in[22], k[0], k[1], P, out, out + 4);
    if (!lout) return 0;
    for (int x = 0; x < 23; ++x) lin[x] = 0.0;
    double lmEc = 0.0, lmES = 0.0, lmEN = 0.0;
    fv::interior_terms_adj<double>(in, in + 4, in + 8, in + 12, in + 16, aE * rEc, aE * rES,
                                   aE * rEN, in[21], in[22], k[0], k[1], P, lout, lout + 4, lin,
                                   lin + 4, lin + 8, lin + 12, lin + 16, lmEc, lmES, lmEN, lin[21],
                                   lin[22]);
    lin[20] = rEc * lmEc + rES * lmES + rEN * lmEN;
    return 0;
  }
  return 1;
}

// ---------------------------------------------------------------------------
// Algorithmic operation count of one cell-update, obtained by running the
// kernels' own per-cell arithmetic on a counting scalar type on the host.
// One cell-update = one reconstruction (second-order branch, predictor on,
// every limiter test active), one x face, one y face, the interior integral,
// the update and the epilogue (signal rate, detector weight).  Recomputation
// of halo cells by neighbouring tiles is not counted, nor are the momentum
// fluxes of the face states a second time: each face state belongs to one
// cell, whose interior integral forms them, and the faces take them from
// there (the face solvers below are given them).
// ---------------------------------------------------------------------------
namespace {

struct Ops {
  long long add = 0, mul = 0, div = 0, sqrt = 0, cmp = 0;
};
Ops g_ops;

struct CD {
  double v;
  CD(double x = 0.0) : v(x) {}
};
inline CD operator+(CD a, CD b) { ++g_ops.add; return CD(a.v + b.v); }
inline CD operator-(CD a, CD b) { ++g_ops.add; return CD(a.v - b.v); }
inline CD operator*(CD a, CD b) { ++g_ops.mul; return CD(a.v * b.v); }
inline CD operator/(CD a, CD b) { ++g_ops.div; return CD(a.v / b.v); }
inline CD operator-(CD a) { return CD(-a.v); }
inline CD& operator+=(CD& a, CD b) { a = a + b; return a; }
inline CD& operator-=(CD& a, CD b) { a = a - b; return a; }
inline bool operator<(CD a, CD b) { ++g_ops.cmp; return a.v < b.v; }
inline bool operator>(CD a, CD b) { ++g_ops.cmp; return a.v > b.v; }
inline bool operator<=(CD a, CD b) { ++g_ops.cmp; return a.v <= b.v; }
inline bool operator==(CD a, CD b) { ++g_ops.cmp; return a.v == b.v; }
inline CD fmin(CD a, CD b) { ++g_ops.cmp; return CD(a.v < b.v ? a.v : b.v); }
inline CD fmax(CD a, CD b) { ++g_ops.cmp; return CD(a.v > b.v ? a.v : b.v); }

}  // namespace

// out[0..4] = additions/subtractions, multiplications, divisions, square roots,
// comparisons (min, max, abs, compare) of one cell-update; first_order: a cell
// that the order switch (alpha <= 10 eps) advances at first order, whose
// reconstruction is its own fluctuation (the equilibrium products only).
static int count_cell(bool first_order, double* out) {
  if (!out) return 1;
  using T = CD;
  fv::Phys<T> P;
  P.rho0 = 1000.0;
  P.k0 = 4.36e5;
  P.g = 9.81;
  P.c2 = 436.0;
  P.c = std::sqrt(436.0);
  P.inv_c = 1.0 / std::sqrt(436.0);
  P.kappa = 9.81 * 1000.0 / 4.36e5;
  fv::ReconConsts<T> R;
  R.half_dx = R.half_dy = 1.0 / 64.0;
  R.inv_2dx = R.inv_2dy = 16.0;
  R.ten_eps = 0.01;
  R.half_dt = 1e-4;
  for (int v = 0; v < 4; ++v) {
    R.eta[v] = 1e-9;
    R.inv_eta[v] = 1e9;
  }
  // a generic liquid cell in motion with all four neighbours fluid
  const double q0[4] = {1003.0, 520.0, -130.0, 0.93};
  g_ops = Ops();
  T fW[4], fE[4], fS[4], fN[4], base[4], ga[2];
  const T aE = T(0.93), rEc = T(1001.0), rES = T(1001.2), rEN = T(1000.8);
  const T mEc = aE * rEc, mES = aE * rES, mEN = aE * rEN;
  if (first_order) {
    const T Qf[4] = {T(1003.0) - mEc, T(520.0), T(-130.0), T(0.0)};
    for (int v = 0; v < 4; ++v) fW[v] = fE[v] = fS[v] = fN[v] = base[v] = Qf[v];
    ga[0] = ga[1] = T(0.0);
  } else {
  // neighbour fluctuations (8 neighbours: one multiply-subtract each for m, one
  // subtraction for alpha) and the stencil min/max are part of the kernel body
  // the cell's own fluctuation: m - alpha^E rho^E
  T Qf[4] = {T(1003.0) - mEc, T(520.0), T(-130.0), T(0.0)};
  T nb[8][4];
  const double shift[8] = {-3.1, 4.2, -1.7, 2.5, 0.7, -0.9, 1.3, -2.2};
  for (int k = 0; k < 8; ++k) {
    T rn = T(1001.0 + 0.1 * k), an = T(0.93 + 0.001 * shift[k]);
    T mraw = T(1003.0 + shift[k]);
    nb[k][0] = mraw - T(0.93) * rn;
    nb[k][1] = T(520.0 + 11.0 * shift[k]);
    nb[k][2] = T(-130.0 + 7.0 * shift[k]);
    nb[k][3] = an - T(0.93);
  }
  T mx[4], mn[4];
  for (int v = 0; v < 4; ++v) {
    fW[v] = nb[0][v];
    fE[v] = nb[1][v];
    fS[v] = nb[2][v];
    fN[v] = nb[3][v];
    mx[v] = fmax(fmax(fmax(Qf[v], fW[v]), fmax(fE[v], fS[v])), fN[v]);
    mn[v] = fmin(fmin(fmin(Qf[v], fW[v]), fmin(fE[v], fS[v])), fN[v]);
    for (int d = 4; d < 8; ++d) {
      mx[v] = fmax(mx[v], nb[d][v]);
      mn[v] = fmin(mn[v], nb[d][v]);
    }
  }
  fv::recon_core(Qf, fW, fE, fS, fN, mx, mn, aE, mEc, mES, mEN, rEc, P, R, base, ga);
  }
  // one x face and one y face per cell
  {
    const T qm[4] = {q0[0], q0[1], q0[2], q0[3]};
    const T qp[4] = {q0[0] + 2.0, q0[1] - 30.0, q0[2] + 5.0, q0[3] - 0.01};
    T dq[4], Dm[4], Dp[4];
    const T fm[2] = {T(269.6), T(-67.4)}, fp[2] = {T(239.4), T(-62.6)};
    for (int c = 0; c < 4; ++c) dq[c] = qp[c] - qm[c];
    fv::xface_fx(qm, dq, fm, fp, P, Dm, Dp);
    for (int c = 0; c < 4; ++c) dq[c] = qp[c] - qm[c];
    const T dap = P.c2 * ((T(1000.1) - P.rho0) * T(0.0) + (dq[0] - P.rho0 * dq[3]));
    fv::yface_fx(qm, dq, fm, fp, dap, P, Dm, Dp);
  }
  // the momentum fluxes of the four face states, once per cell (a first-order
  // cell's W and E states are the same), then the interior integral
  T xW[2], xE[2], yS[2], yN[2];
  fv::xflux(mEc + fW[0], fW[1], fW[2], xW);
  if (first_order) {
    xE[0] = xW[0];
    xE[1] = xW[1];
  } else {
    fv::xflux(mEc + fE[0], fE[1], fE[2], xE);
  }
  fv::yflux(mES + fS[0], fS[1], fS[2], yS);
  fv::yflux(mEN + fN[0], fN[1], fN[2], yN);
  T Ix[4], Iy[4];
  fv::interior_terms_fx(fW, fE, fS, fN, base, mEc, xW, xE, yS, yN, ga[0], ga[1], T(1.0 / 32),
                        T(1.0 / 32), P, Ix, Iy);
  // update: Q^{n+1} = Q^n - dt/dx (D+_W + D-_E + I_x) - dt/dy (D+_S + D-_N + I_y)
  const T rdx = T(1e-4) / T(1.0 / 32), rdy = T(1e-4) / T(1.0 / 32);
  T qn[4];
  for (int c = 0; c < 4; ++c) {
    const T xs = T(0.1) + T(0.2) + Ix[c];
    const T ys = T(0.3) + T(0.4) + Iy[c];
    qn[c] = T(q0[c]) - rdx * xs - rdy * ys;
  }
  // epilogue: velocities, signal rate, detector weight
  const T r = T(1.0) / qn[0];
  const T u = qn[1] * r, v = qn[2] * r;
  const T rate = (fv::tabs(u) + P.c) * T(32.0) + (fv::tabs(v) + P.c) * T(32.0);
  T w = (qn[3] - T(1e-3)) * T(1.0 / 0.999);
  w = fmin(fmax(w, T(0.0)), T(1.0));
  (void)rate;
  out[0] = (double)g_ops.add;
  out[1] = (double)g_ops.mul;
  out[2] = (double)g_ops.div;
  out[3] = (double)g_ops.sqrt;
  out[4] = (double)g_ops.cmp;
  return 0;
}

extern "C" int fv_host_cell_ops(double* out) { return count_cell(false, out); }

extern "C" int fv_host_cell_ops_first_order(double* out) { return count_cell(true, out); }
