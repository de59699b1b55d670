// Cell- and face-level pieces of one time step of Eq. (Scheme), shared by the
// two step kernels: step_kernel (fv_kernels.cu, one CTA per 32 x 8 tile) and
// strip_kernel (fv_strip.cu, one CTA per 32-column strip marching upwards in
// blocks of 8 rows).  The kernels differ only in how they stage the window of
// Q^n and the reconstructed states in shared memory; every arithmetic
// operation of a step is written here once, so both produce the same bits.
//
// Window coordinates: a window row is an array of cells of one grid row,
// indexed by the window column wi = gi - i0 + 2 (two halo cells on the left
// of the tile's first column i0).  Reconstructed (ring) coordinates: rx =
// gi - i0 + 1.
#pragma once

#include <cstdint>

#include "fv_consts.cuh"
#include "fv_kernels.cuh"
#include "fv_model.cuh"

namespace fv {
namespace tile {

// Four components of one state as one shared-memory element, so that a state
// moves with one vector access (LDS.128 / STS.128 in FP32, two in FP64).
template <typename T>
struct alignas(4 * sizeof(T)) V4 {
  T x, y, z, w;
};

template <typename T>
__device__ __forceinline__ void unpack(const V4<T>& v, T a[4]) {
  a[0] = v.x;
  a[1] = v.y;
  a[2] = v.z;
  a[3] = v.w;
}

template <typename T>
__device__ __forceinline__ V4<T> pack(const T a[4]) {
  return V4<T>{a[0], a[1], a[2], a[3]};
}

// Largest / smallest of three values.  In FP32 one three-input instruction
// (sm_100 and later); max and min are exact, so the result is that of two
// fmax / fmin whatever the order.
template <typename T>
__device__ __forceinline__ T max3(T a, T b, T c) {
  return fmax(fmax(a, b), c);
}
template <typename T>
__device__ __forceinline__ T min3(T a, T b, T c) {
  return fmin(fmin(a, b), c);
}
// In FP64 the bounds are formed on the integer pipe: a double's bits, with
// the magnitude bits of a negative value inverted, order as a signed 64-bit
// integer exactly as the values do (-0 before +0); the largest / smallest of
// three is then selected by two integer comparisons.
__device__ __forceinline__ long long ord64(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
template <>
__device__ __forceinline__ double max3<double>(double a, double b, double c) {
  const long long ia = ord64(a), ib = ord64(b), ic = ord64(c);
  const double ab = ia >= ib ? a : b;
  return max(ia, ib) >= ic ? ab : c;
}
template <>
__device__ __forceinline__ double min3<double>(double a, double b, double c) {
  const long long ia = ord64(a), ib = ord64(b), ic = ord64(c);
  const double ab = ia <= ib ? a : b;
  return min(ia, ib) <= ic ? ab : c;
}
template <>
__device__ __forceinline__ float max3<float>(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
template <>
__device__ __forceinline__ float min3<float>(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// One domain of a batch as the batched step kernel reads it (device table
// filled on the host by batch_fill_table): parameters, constants, the two
// state buffers (parity selects the one read), mask, levels, accumulators,
// equilibrium tables.
template <typename T>
struct BatchDomain {
  StepParams p;
  KConsts<T> kc;
  T* q[2];
  const uint8_t* solid;
  int32_t* Kref;
  int32_t* Kcur;
  unsigned long long* colsum;
  DevScalars* sc;
  const double* rhoE_d;
  const T* rt;
};

constexpr unsigned char F_FLUID = 0, F_SOLID = 1, F_OUT = 2;
constexpr unsigned long long ONE_FIXED = 1ull << 32;
enum { F_W = 0, F_E = 1, F_S = 2, F_N = 3 };

// Boundary kinds of the four domain sides (true = transmissive, else wall).
struct Sides {
  bool W, E, S, N;
};

__device__ __forceinline__ Sides sides_of(const StepParams& p) {
  return Sides{p.side[0] == 1, p.side[1] == 1, p.side[2] == 1, p.side[3] == 1};
}

// Raw global loads of one window cell (gi, gj), issued together (the state
// arrays hold zeros in solid cells), so that they can be started a phase
// before they are used.
template <typename T>
struct CellLoad {
  T m, mu, mv, a;
  int Kr, Kc;  // levels the column was stored with / of this step (deviation form)
  uint8_t solid;
  bool in;  // inside the domain
};

template <typename T, bool DEV>
__device__ __forceinline__ void fetch_cell(const T* __restrict__ qin,
                                           const uint8_t* __restrict__ solid,
                                           const int32_t* __restrict__ Kref,
                                           const int32_t* __restrict__ Kcur, int nx, int ny,
                                           size_t N, int gi, int gj, CellLoad<T>& L) {
  L.in = gi >= 0 && gj >= 0 && gi < nx && gj < ny;
  if (!L.in) {  // every field defined on every path: no live range spans two fetches
    L.m = L.mu = L.mv = L.a = T(0);
    L.Kr = L.Kc = 0;
    L.solid = 0;
    return;
  }
  const size_t c = (size_t)gj * nx + gi;
  L.solid = solid[c];
  L.m = qin[c];
  L.mu = qin[N + c];
  L.mv = qin[2 * N + c];
  L.a = qin[3 * N + c];
  if (DEV) {
    L.Kr = Kref[gi];
    L.Kc = Kcur[gi];
  }
}

// The cell's flag and, if fluid, its state (m, mu, mv, a) into w.  In
// deviation form m^f is re-based from the level it was stored with (Kref) to
// this step's level (Kcur) of its column; gj is the cell's grid row.
template <typename T, bool DEV>
__device__ __forceinline__ unsigned char commit_cell(const CellLoad<T>& L,
                                                     const T* __restrict__ rt, int ny, int gj,
                                                     V4<T>& w) {
  if (!L.in) return F_OUT;
  if (L.solid) return F_SOLID;
  T m = L.m;
  if (DEV && L.Kr != L.Kc)
    m += L.a * (tab(rt, 2 * (gj - L.Kr) + 1, ny) - tab(rt, 2 * (gj - L.Kc) + 1, ny));
  w = V4<T>{m, L.mu, L.mv, L.a};
  return F_FLUID;
}

template <typename T, bool DEV>
__device__ __forceinline__ unsigned char load_cell(const T* __restrict__ qin,
                                                   const uint8_t* __restrict__ solid,
                                                   const int32_t* __restrict__ Kref,
                                                   const int32_t* __restrict__ Kcur,
                                                   const T* __restrict__ rt, int nx, int ny,
                                                   size_t N, int gi, int gj, V4<T>& w) {
  CellLoad<T> L;
  fetch_cell<T, DEV>(qin, solid, Kref, Kcur, nx, ny, N, gi, gj, L);
  return commit_cell<T, DEV>(L, rt, ny, gj, w);
}

// Reconstruction of one cell (Section 3.4): fluctuations of the cell and its
// eight neighbours with respect to the cell's water-at-rest state Q^E (alpha^E
// = alpha of the cell, rho^E of its column level K at the neighbour's height);
// walls and solid neighbours seen as the mirror state; the limiter bounds over
// the 3 x 3 stencil; recon_core (slopes, Barth-Jespersen factor, order
// switch, half-step predictor).  wS, wC, wN: window rows below, of and above
// the cell (and their flags fS, fC, fN); Kw: the levels of the window columns;
// wi: the cell's window column; gj: its grid row.
// Outputs: rs = (alpha^E, m^E at the centre, bottom and top face), rf = the
// four face fluctuation states (W, E, S, N) at t^{n+1/2}, base = the centre
// fluctuation at t^{n+1/2}, ga = the limited alpha slopes.
template <typename T, bool DEV>
__device__ __forceinline__ void recon_cell(const V4<T>* wS, const V4<T>* wC, const V4<T>* wN,
                                           const unsigned char* fS, const unsigned char* fC,
                                           const unsigned char* fN, const int* Kw, int wi, int gj,
                                           const T* __restrict__ rt, int ny, const Sides& sd,
                                           const Phys<T>& P, const ReconConsts<T>& RC, V4<T>& rs,
                                           V4<T> rf[4], T base[4], T ga[2]) {
  auto rE = [&](int h) -> T { return tab(rt, h, ny); };
  const int K = Kw[wi];
  const V4<T> wc = wC[wi];
  const T aE = wc.w;
  const T rEc = rE(2 * (gj - K) + 1);
  const T rES = rE(2 * (gj - K));
  const T rEN = rE(2 * (gj + 1 - K));
  const T mEc = aE * rEc;
  T Qf[4];
  Qf[0] = DEV ? wc.x : wc.x - mEc;
  Qf[1] = wc.y;
  Qf[2] = wc.z;
  Qf[3] = T(0);
  // The order switch of Section 3.4: a cell with alpha <= 10 eps is advanced
  // at first order (no slopes, no predictor), so its four face states and its
  // centre state at t^{n+1/2} are its own fluctuation whatever its
  // neighbours: the stencil is not read (recon_core gives the same states,
  // up to the sign of zero components, after evaluating it).
  if (aE <= RC.ten_eps) {
    rs = V4<T>{aE, mEc, aE * rES, aE * rEN};
    const V4<T> q = pack(Qf);
    rf[F_W] = q;
    rf[F_E] = q;
    rf[F_S] = q;
    rf[F_N] = q;
#pragma unroll
    for (int c = 0; c < 4; ++c) base[c] = Qf[c];
    ga[0] = ga[1] = T(0);
    return;
  }

  auto wrow = [&](int dwj) -> const V4<T>* { return dwj < 0 ? wS : (dwj > 0 ? wN : wC); };
  auto frow = [&](int dwj) -> const unsigned char* { return dwj < 0 ? fS : (dwj > 0 ? fN : fC); };
  // fluctuation of a neighbour w.r.t. this cell's Q^E; false if not fluid
  auto nbf = [&](int dwi, int dwj, T out[4]) -> bool {
    const int ni = wi + dwi;
    if (frow(dwj)[ni] != F_FLUID) return false;
    const V4<T> wn = wrow(dwj)[ni];
    const T an = wn.w;
    const int gjn = gj + dwj;
    const T rn = rE(2 * (gjn - K) + 1);
    if (DEV) {
      const int Kn = Kw[ni];
      T mshift;
      if (Kn == K) mshift = (an - aE) * rn;
      else mshift = an * rE(2 * (gjn - Kn) + 1) - aE * rn;
      out[0] = wn.x + mshift;
    } else {
      out[0] = wn.x - aE * rn;
    }
    out[1] = wn.y;
    out[2] = wn.z;
    out[3] = an - aE;
    return true;
  };
  // mirror state behind a wall or a solid neighbour; the cell's own state
  // behind a transmissive side
  auto ghost = [&](int dwi, int dwj, int normal, bool tr, T out[4]) {
    const unsigned char f = frow(dwj)[wi + dwi];
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v] = Qf[v];
    if (!(f == F_OUT && tr)) {
      if (normal == 1) out[1] = -out[1];
      else out[2] = -out[2];
    }
  };
  T fW[4], fE[4], fSo[4], fNo[4];
  T fd[4][4];  // diagonal neighbours SW, SE, NW, NE
  // In deviation form most cells have a fluid 3 x 3 stencil whose three
  // columns share one level: every neighbour then takes the one formula of nbf
  // below, evaluated without the per-neighbour tests (an issue-bound FP32
  // kernel gains; the FP64 kernel is bound by its FP64 pipe and does not).
  const bool all_fluid = (fS[wi - 1] | fS[wi] | fS[wi + 1] | fC[wi - 1] | fC[wi + 1] |
                          fN[wi - 1] | fN[wi] | fN[wi + 1]) == F_FLUID;
  const bool one_level = Kw[wi - 1] == K && Kw[wi + 1] == K;
  if (DEV && all_fluid && one_level) {
    const T rnS = rE(2 * (gj - 1 - K) + 1), rnN = rE(2 * (gj + 1 - K) + 1);
    auto fl = [&](const V4<T>& wn, T rn, T out[4]) {
      const T an = wn.w;
      if (DEV) {
        const T mshift = (an - aE) * rn;
        out[0] = wn.x + mshift;
      } else {
        out[0] = wn.x - aE * rn;
      }
      out[1] = wn.y;
      out[2] = wn.z;
      out[3] = an - aE;
    };
    fl(wC[wi - 1], rEc, fW);
    fl(wC[wi + 1], rEc, fE);
    fl(wS[wi], rnS, fSo);
    fl(wN[wi], rnN, fNo);
    fl(wS[wi - 1], rnS, fd[0]);
    fl(wS[wi + 1], rnS, fd[1]);
    fl(wN[wi - 1], rnN, fd[2]);
    fl(wN[wi + 1], rnN, fd[3]);
  } else {
    if (!nbf(-1, 0, fW)) ghost(-1, 0, 1, sd.W, fW);
    if (!nbf(1, 0, fE)) ghost(1, 0, 1, sd.E, fE);
    if (!nbf(0, -1, fSo)) ghost(0, -1, 2, sd.S, fSo);
    if (!nbf(0, 1, fNo)) ghost(0, 1, 2, sd.N, fNo);
    // limiter bounds over the 3 x 3 stencil; a diagonal neighbour that is not
    // fluid contributes the cell's own fluctuation, already among the bounds
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      if (!nbf((d & 1) ? 1 : -1, (d & 2) ? 1 : -1, fd[d])) {
#pragma unroll
        for (int v = 0; v < 4; ++v) fd[d][v] = Qf[v];
      }
    }
  }
  T mx[4], mn[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    mx[v] = max3(max3(Qf[v], fW[v], fE[v]), max3(fSo[v], fNo[v], fd[0][v]),
                 max3(fd[1][v], fd[2][v], fd[3][v]));
    mn[v] = min3(min3(Qf[v], fW[v], fE[v]), min3(fSo[v], fNo[v], fd[0][v]),
                 min3(fd[1][v], fd[2][v], fd[3][v]));
  }
  const T mES = aE * rES, mEN = aE * rEN;
  recon_core(Qf, fW, fE, fSo, fNo, mx, mn, aE, mEc, mES, mEN, rEc, P, RC, base, ga);
  rs = V4<T>{aE, mEc, mES, mEN};
  rf[F_W] = pack(fW);
  rf[F_E] = pack(fE);
  rf[F_S] = pack(fSo);
  rf[F_N] = pack(fNo);
}

// Face-flux records of a reconstructed cell (rs, rf as recon_cell writes
// them): xf = the x fluxes of its W and E face states, yf = the y fluxes of
// its S and N ones (xflux, yflux), formed once for the cell's two x faces,
// two y faces and interior integral.  first: the cell is advanced at first
// order (recon_cell's order switch), so its W and E states are the same.
template <typename T>
__device__ __forceinline__ void face_fluxes(const V4<T>& rs, const V4<T> rf[4], bool first,
                                            V4<T>& xf, V4<T>& yf) {
  T a[2], b[2], c[2], d[2];
  xflux(rs.y + rf[F_W].x, rf[F_W].y, rf[F_W].z, a);
  if (first) {
    b[0] = a[0];
    b[1] = a[1];
  } else {
    xflux(rs.y + rf[F_E].x, rf[F_E].y, rf[F_E].z, b);
  }
  yflux(rs.z + rf[F_S].x, rf[F_S].y, rf[F_S].z, c);
  yflux(rs.w + rf[F_N].x, rf[F_N].y, rf[F_N].z, d);
  xf = V4<T>{a[0], a[1], b[0], b[1]};
  yf = V4<T>{c[0], c[1], d[0], d[1]};
}

// x face between the reconstructed cells L (left) and R (right) with flags fl,
// fr: L's (alpha^E, m^E ...) record sL and east face state eL, R's record sR
// and west face state wR (read only where the cell is fluid).  Both fluid: the
// Osher solver on the two reconstructed states; one fluid: the mirror state
// (a wall or a solid neighbour) or the transmissive copy on the other side.
// XOR selects the conservative Osher-Romberg viscosity of Eq. (OR_cons)
// instead of the Gauss-Legendre quadrature of Eq. (OsherMatrixFormal_approx).
// xfL, xfR (optional, FP64): L's and R's face-flux records (face_fluxes), whose
// E and W parts replace the solver's own evaluation of the endpoint fluxes
// with the same bits.
template <typename T, bool XOR>
__device__ __forceinline__ void x_face(unsigned char fl, unsigned char fr, const V4<T>* sL,
                                       const V4<T>* eL, const V4<T>* sR, const V4<T>* wR,
                                       const Sides& sd, const Phys<T>& P, T Dm[4], T Dp[4],
                                       const V4<T>* xfL = nullptr, const V4<T>* xfR = nullptr) {
#pragma unroll
  for (int c = 0; c < 4; ++c) Dm[c] = Dp[c] = T(0);
  const bool L = fl == F_FLUID, R = fr == F_FLUID;
  if (!(L || R)) return;
  T qm[4], qp[4], dq[4];
  if (L && R) {
    const V4<T> a = *sL, b = *sR;
    const T mEL = a.y, mER = b.y;
    const T aL = a.x, aR = b.x;
    T fl4[4], fr4[4];
    unpack(*eL, fl4);
    unpack(*wR, fr4);
    qm[0] = mEL + fl4[0]; qm[1] = fl4[1]; qm[2] = fl4[2]; qm[3] = aL + fl4[3];
    qp[0] = mER + fr4[0]; qp[1] = fr4[1]; qp[2] = fr4[2]; qp[3] = aR + fr4[3];
    dq[0] = (mER - mEL) + (fr4[0] - fl4[0]);
    dq[1] = fr4[1] - fl4[1];
    dq[2] = fr4[2] - fl4[2];
    dq[3] = (aR - aL) + (fr4[3] - fl4[3]);
    if (!XOR && xfL) {
      const V4<T> a2 = *xfL, b2 = *xfR;
      const T fm[2] = {a2.z, a2.w}, fp[2] = {b2.x, b2.y};
      xface_fx(qm, dq, fm, fp, P, Dm, Dp);
      return;
    }
  } else {
    const V4<T> s = L ? *sL : *sR;
    const V4<T> fc = L ? *eL : *wR;
    const T mE = s.y, aE = s.x;
    T q[4];
    q[0] = mE + fc.x;
    q[1] = fc.y;
    q[2] = fc.z;
    q[3] = aE + fc.w;
    const bool outside = L ? (fr == F_OUT) : (fl == F_OUT);
    const bool transmissive = outside && (L ? sd.E : sd.W);
    T g[4] = {q[0], transmissive ? q[1] : -q[1], q[2], q[3]};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      qm[c] = L ? q[c] : g[c];
      qp[c] = L ? g[c] : q[c];
    }
    dq[0] = T(0);
    dq[1] = qp[1] - qm[1];
    dq[2] = T(0);
    dq[3] = T(0);
  }
  if (XOR) xface_or(qm, qp, dq, P, Dm, Dp);
  else xface(qm, qp, dq, P, Dm, Dp);
}

// y face between the reconstructed cells B (below) and T (above) of a column
// with level K; gjT is T's grid row.  sB, nB: B's record and north face
// state; sT, sT_: T's record and south face state.  The jump of alpha p is
// split into its equilibrium part (rho^E_f - rho0) Delta alpha^E, exactly
// zero at the level face, and the fluctuation part c2 (dm^f - rho0 da^f).
// yfB, yfT (optional, FP64): B's and T's face-flux records, whose N and S
// parts replace the solver's own evaluation of the endpoint fluxes.
template <typename T>
__device__ __forceinline__ void y_face(unsigned char fb, unsigned char ft, const V4<T>* sB,
                                       const V4<T>* nB, const V4<T>* sT, const V4<T>* sT_,
                                       int K, int gjT, const T* __restrict__ rt, int ny,
                                       const Sides& sd, const Phys<T>& P, T Dm[4], T Dp[4],
                                       const V4<T>* yfB = nullptr, const V4<T>* yfT = nullptr) {
#pragma unroll
  for (int c = 0; c < 4; ++c) Dm[c] = Dp[c] = T(0);
  const bool B = fb == F_FLUID, Tt = ft == F_FLUID;
  if (!(B || Tt)) return;
  T qm[4], qp[4], dq[4];
  T dap = T(0);
  if (B && Tt) {
    const V4<T> a = *sB, b = *sT;
    const T mEB = a.w, mET = b.z;
    const T aB = a.x, aT = b.x;
    T fb4[4], ft4[4];
    unpack(*nB, fb4);
    unpack(*sT_, ft4);
    qm[0] = mEB + fb4[0]; qm[1] = fb4[1]; qm[2] = fb4[2]; qm[3] = aB + fb4[3];
    qp[0] = mET + ft4[0]; qp[1] = ft4[1]; qp[2] = ft4[2]; qp[3] = aT + ft4[3];
    dq[0] = (mET - mEB) + (ft4[0] - fb4[0]);
    dq[1] = ft4[1] - fb4[1];
    dq[2] = ft4[2] - fb4[2];
    dq[3] = (aT - aB) + (ft4[3] - fb4[3]);
    const T rEf = tab(rt, 2 * (gjT - K), ny);
    dap = P.c2 * ((rEf - P.rho0) * (aT - aB) + ((ft4[0] - fb4[0]) - P.rho0 * (ft4[3] - fb4[3])));
    if (yfB) {
      const V4<T> a2 = *yfB, b2 = *yfT;
      const T gm[2] = {a2.z, a2.w}, gp[2] = {b2.x, b2.y};
      yface_fx(qm, dq, gm, gp, dap, P, Dm, Dp);
      return;
    }
  } else {
    const V4<T> s = B ? *sB : *sT;
    const V4<T> fc = B ? *nB : *sT_;
    const T mE = B ? s.w : s.z, aE = s.x;
    T q[4];
    q[0] = mE + fc.x;
    q[1] = fc.y;
    q[2] = fc.z;
    q[3] = aE + fc.w;
    const bool outside = B ? (ft == F_OUT) : (fb == F_OUT);
    const bool transmissive = outside && (B ? sd.N : sd.S);
    T g[4] = {q[0], q[1], transmissive ? q[2] : -q[2], q[3]};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      qm[c] = B ? q[c] : g[c];
      qp[c] = B ? g[c] : q[c];
    }
    dq[0] = T(0);
    dq[1] = T(0);
    dq[2] = qp[2] - qm[2];
    dq[3] = T(0);
  }
  yface(qm, qp, dq, dap, P, Dm, Dp);
}

// Update of one fluid cell: Q^{n+1} = Q^n - dt/dx (D+_W + D-_E + I_x)
// - dt/dy (D+_S + D-_N + I_y) with the interior integral of Eq.
// (b^y_3_final_integral) plus the conservative part.  rs, rf, base, ga: the
// cell's reconstruction; DpW, DmE, DpS, DmN: the fluctuations of its four
// faces; rEc: rho^E at its centre (deviation form).  qn: the new state in
// stored form; returns the full alpha rho.
// xf, yf (optional, FP64): the cell's face-flux records (face_fluxes), in
// place of the interior integral's own evaluation of the same fluxes.
template <typename T, bool DEV>
__device__ __forceinline__ T update_cell(const T qold[4], const V4<T>& rs, const V4<T>* rf,
                                         const V4<T>& base4, T dax, T day, const V4<T>& DpW4,
                                         const V4<T>& DmE4, const V4<T>& DpS4, const V4<T>& DmN4,
                                         T rEc, T rdx, T rdy, T dx, T dy, const Phys<T>& P,
                                         T qn[4], const V4<T>* xf = nullptr,
                                         const V4<T>* yf = nullptr) {
  const T mEc = rs.y, mES = rs.z, mEN = rs.w;
  T fW[4], fE[4], fS[4], fN[4], base[4];
  unpack(rf[F_W], fW);
  unpack(rf[F_E], fE);
  unpack(rf[F_S], fS);
  unpack(rf[F_N], fN);
  unpack(base4, base);
  T Ix[4], Iy[4];
  if (xf) {
    const V4<T> a = *xf, b = *yf;
    const T xW[2] = {a.x, a.y}, xE[2] = {a.z, a.w}, yS[2] = {b.x, b.y}, yN[2] = {b.z, b.w};
    interior_terms_fx(fW, fE, fS, fN, base, mEc, xW, xE, yS, yN, dax, day, dx, dy, P, Ix, Iy);
  } else {
    interior_terms(fW, fE, fS, fN, base, mEc, mES, mEN, dax, day, dx, dy, P, Ix, Iy);
  }
  T xs[4], ys[4], DpW[4], DmE[4], DpS[4], DmN[4];
  unpack(DpW4, DpW);
  unpack(DmE4, DmE);
  unpack(DpS4, DpS);
  unpack(DmN4, DmN);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    xs[c] = DpW[c] + DmE[c] + Ix[c];
    ys[c] = DpS[c] + DmN[c] + Iy[c];
  }
  if constexpr (DEV) {
    // deviation form: m^f_new = m^f + dm - rho^E_c da (own level, own new alpha)
    T dQ[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) dQ[c] = -rdx * xs[c] - rdy * ys[c];
    qn[0] = qold[0] + (dQ[0] - rEc * dQ[3]);
    qn[1] = qold[1] + dQ[1];
    qn[2] = qold[2] + dQ[2];
    qn[3] = qold[3] + dQ[3];
    return qn[3] * rEc + qn[0];
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) qn[c] = qold[c] - rdx * xs[c] - rdy * ys[c];
    return qn[0];
  }
}

}  // namespace tile
}  // namespace fv
