// fv_adjoint: gradient of a gauge loss after n time steps with respect to the
// state the steps start from, by the discrete adjoint (reverse mode) of the
// fused step.
//
// The loss is L = sum_n dt_n sum_g (m_g^n - T_g^n)^2 over the steps n = 1..N
// (m = alpha rho at gauge cell g after step n).  dt_n and the detected levels
// K_i^n are piecewise constant in the state and are held at their values in
// the forward run; so is every branch of the step (the limiter's active
// factor and the stencil extrema it uses, sign() and |.|, the order switch,
// the admissibility fallback).  The result is the exact derivative of that
// frozen-branch map, evaluated in the arithmetic type of the handle; the
// adjoint state itself is accumulated in double.
//
// Memory/time trade-off: states at every s-th step are kept (s = ceil(sqrt N)
// by default) and each segment is replayed with the forward kernel before it
// is reversed, so the reverse sweep costs one extra forward pass and holds
// about 2 sqrt(N) states.
//
// One reverse step (state Q^{n-1} in, adjoint of Q^n in, adjoint of Q^{n-1}
// out) is four kernels:
//   rec     per cell: the Section 3.4 reconstruction of the forward step
//           (same device functions), its equilibrium masses and face states;
//   faces   per face: the adjoint of the x (Osher) and y (Osher-Romberg)
//           fluctuations for D- -> left/bottom cell and D+ -> right/top cell,
//           written to one slot per cell side (each slot has one writer);
//   cells   per cell: the adjoint of the interior integral and of the
//           reconstruction, scattered into per-cell contributions to its 3x3
//           stencil;
//   gather  per cell: adjoint of Q^{n-1} = adjoint of Q^n plus the nine
//           contributions addressed to it, summed in a fixed order in double.
// Every sum has a fixed order, so the result is bitwise reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fv.h"
#include "fv_adjoint.cuh"
#include "fv_consts.cuh"
#include "fv_handle.cuh"
#include "fv_kernels.cuh"
#include "fv_model.cuh"
#include "fv_model_host.h"

namespace fv {
namespace {

constexpr int BX = 32, BY = 8;
constexpr int NSLOT = 20;    // per side W, E, S, N: 4 fluctuation adjoints + 1 alpha^E adjoint
constexpr int NREC = 20;     // aE, mEc, mES, mEN, face states W, E, S, N
constexpr int NCONTRIB = 36; // 3x3 stencil x 4 components
enum { R_AE = 0, R_MEC = 1, R_MES = 2, R_MEN = 3, R_FW = 4, R_FE = 8, R_FS = 12, R_FN = 16 };
enum { S_W = 0, S_E = 5, S_S = 10, S_N = 15 };

template <typename T>
struct AdjArgs {
  int nx, ny;
  int side[4];              // W, E, S, N: 0 wall, 1 transmissive
  KConsts<T> kc;            // kc.R.half_dt = dt / 2
  T dt;
  const T* q;               // Q^{n-1} in storage form (4 planes)
  const uint8_t* solid;
  const int32_t* Kref;      // level q is stored with (deviation form)
  const int32_t* Kcur;      // levels of step n
  const T* rt;              // rho^E table, index h + 2 ny
  const double* lam;        // adjoint of Q^n (4 planes)
  T* rec;                   // NREC planes
  T* slot;                  // NSLOT planes
  T* contrib;               // NCONTRIB planes
  double* lam_out;          // adjoint of Q^{n-1}
  // loss source of Q^{n-1}, added by the gather (src_dt = 0: none): gauges
  // sorted by cell (gord), gmark[c] = first position of cell c in that order or -1
  const int32_t* gmark;
  const int32_t* gord;
  const int64_t* gauges;
  int ng;
  const double* src_m;      // alpha rho at the gauges after step n-1
  const double* src_t;      // their targets
  double src_dt;            // dt of step n-1
};

template <typename T>
__host__ __device__ __forceinline__ bool fluid_at(const AdjArgs<T>& A, int i, int j) {
  return i >= 0 && j >= 0 && i < A.nx && j < A.ny && A.solid[(size_t)j * A.nx + i] == 0;
}

// alpha rho of a fluid cell as the step kernel holds it after loading: the
// full value (FP64), or m^f re-based to the cell's current level (deviation form).
template <typename T, bool DEV>
__host__ __device__ __forceinline__ T load_m(const AdjArgs<T>& A, int i, int j, T a) {
  const size_t c = (size_t)j * A.nx + i;
  T m = A.q[c];
  if (DEV) {
    const int Kr = A.Kref[i], Kc = A.Kcur[i];
    if (Kr != Kc) m += a * (tab(A.rt, 2 * (j - Kr) + 1, A.ny) - tab(A.rt, 2 * (j - Kc) + 1, A.ny));
  }
  return m;
}

// Inputs and outputs of the reconstruction of one fluid cell.
template <typename T>
struct CellRec {
  T Qf[4];
  T fi[4][4];       // edge neighbours W, E, S, N (fluctuation or ghost), before recon
  T fd[4][4];       // diagonal neighbours (-1,-1), (1,-1), (-1,1), (1,1)
  T rn[4], rd[4];   // rho^E at the edge / diagonal neighbours' centres, own column level
  bool nfl[4], dfl[4], ncopy[4];  // neighbour fluid; ghost is a plain copy (transmissive)
  T mx[4], mn[4];
  T aE, rEc, rES, rEN, mEc, mES, mEN;
  T fo[4][4];       // face states W, E, S, N at t^{n+1/2}
  T base[4], ga[2];
  bool first;       // alpha <= 10 eps: advanced at first order (the stencil is not read)
};

// Same loads, fluctuations, ghosts, extrema and reconstruction as the step kernel.
template <typename T, bool DEV>
__host__ __device__ __forceinline__ void recon_cell(const AdjArgs<T>& A, int i, int j, CellRec<T>& C) {
  const size_t N = (size_t)A.nx * A.ny;
  const int ny = A.ny;
  const int K = A.Kcur[i];
  const size_t c = (size_t)j * A.nx + i;
  const T aE = A.q[3 * N + c];
  C.aE = aE;
  C.rEc = tab(A.rt, 2 * (j - K) + 1, ny);
  C.rES = tab(A.rt, 2 * (j - K), ny);
  C.rEN = tab(A.rt, 2 * (j + 1 - K), ny);
  C.mEc = aE * C.rEc;
  const T mown = load_m<T, DEV>(A, i, j, aE);
  C.Qf[0] = DEV ? mown : mown - C.mEc;
  C.Qf[1] = A.q[N + c];
  C.Qf[2] = A.q[2 * N + c];
  C.Qf[3] = T(0);
  // the order switch, as the step kernels take it: face and centre states are
  // the cell's own fluctuation and depend on no neighbour
  C.first = aE <= A.kc.R.ten_eps;
  if (C.first) {
    C.mES = aE * C.rES;
    C.mEN = aE * C.rEN;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      C.nfl[k] = C.dfl[k] = C.ncopy[k] = false;
#pragma unroll
      for (int v = 0; v < 4; ++v) C.fo[k][v] = C.Qf[v];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) C.base[v] = C.Qf[v];
    C.ga[0] = C.ga[1] = T(0);
    return;
  }
  auto nbf = [&](int di, int dj, T out[4], T& rn) -> bool {
    const int ni = i + di, nj = j + dj;
    rn = T(0);
    if (!fluid_at(A, ni, nj)) return false;  // the table is read for in-grid rows only
    rn = tab(A.rt, 2 * (nj - K) + 1, ny);
    const size_t cn = (size_t)nj * A.nx + ni;
    const T an = A.q[3 * N + cn];
    const T mn_ = load_m<T, DEV>(A, ni, nj, an);
    if (DEV) {
      const int Kn = A.Kcur[ni];
      T mshift;
      if (Kn == K) mshift = (an - aE) * rn;
      else mshift = an * tab(A.rt, 2 * (nj - Kn) + 1, ny) - aE * rn;
      out[0] = mn_ + mshift;
    } else {
      out[0] = mn_ - aE * rn;
    }
    out[1] = A.q[N + cn];
    out[2] = A.q[2 * N + cn];
    out[3] = an - aE;
    return true;
  };
  const int ei[4] = {-1, 1, 0, 0}, ej[4] = {0, 0, -1, 1};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    C.nfl[k] = nbf(ei[k], ej[k], C.fi[k], C.rn[k]);
    const int ni = i + ei[k], nj = j + ej[k];
    const bool outside = ni < 0 || nj < 0 || ni >= A.nx || nj >= A.ny;
    C.ncopy[k] = outside && A.side[k] == 1;
    if (!C.nfl[k]) {
#pragma unroll
      for (int v = 0; v < 4; ++v) C.fi[k][v] = C.Qf[v];
      if (!C.ncopy[k]) {
        if (k < 2) C.fi[k][1] = -C.fi[k][1];
        else C.fi[k][2] = -C.fi[k][2];
      }
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    C.mx[v] = fmax(fmax(fmax(C.Qf[v], C.fi[0][v]), fmax(C.fi[1][v], C.fi[2][v])), C.fi[3][v]);
    C.mn[v] = fmin(fmin(fmin(C.Qf[v], C.fi[0][v]), fmin(C.fi[1][v], C.fi[2][v])), C.fi[3][v]);
  }
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    C.dfl[d] = nbf((d & 1) ? 1 : -1, (d & 2) ? 1 : -1, C.fd[d], C.rd[d]);
    if (C.dfl[d]) {
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        C.mx[v] = fmax(C.mx[v], C.fd[d][v]);
        C.mn[v] = fmin(C.mn[v], C.fd[d][v]);
      }
    }
  }
  C.mES = aE * C.rES;
  C.mEN = aE * C.rEN;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int v = 0; v < 4; ++v) C.fo[k][v] = C.fi[k][v];
  recon_core(C.Qf, C.fo[0], C.fo[1], C.fo[2], C.fo[3], C.mx, C.mn, aE, C.mEc, C.mES, C.mEN, C.rEc,
             A.kc.P, A.kc.R, C.base, C.ga);
}

// ------------------------------------------------------------------ rec
template <typename T, bool DEV>
__host__ __device__ void rec_body(const AdjArgs<T>& A, int i, int j) {
  if (!fluid_at(A, i, j)) return;
  CellRec<T> C;
  recon_cell<T, DEV>(A, i, j, C);
  const size_t N = (size_t)A.nx * A.ny, c = (size_t)j * A.nx + i;
  A.rec[R_AE * N + c] = C.aE;
  A.rec[R_MEC * N + c] = C.mEc;
  A.rec[R_MES * N + c] = C.mES;
  A.rec[R_MEN * N + c] = C.mEN;
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int v = 0; v < 4; ++v) A.rec[(R_FW + 4 * k + v) * N + c] = C.fo[k][v];
}

template <typename T, bool DEV>
__global__ void __launch_bounds__(BX * BY) adj_rec_kernel(AdjArgs<T> A) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i < A.nx && j < A.ny) rec_body<T, DEV>(A, i, j);
}

// ------------------------------------------------------------------ faces
template <typename T>
__host__ __device__ __forceinline__ void put_slot(const AdjArgs<T>& A, size_t c, int s, const T lf[4], T la) {
  const size_t N = (size_t)A.nx * A.ny;
#pragma unroll
  for (int v = 0; v < 4; ++v) A.slot[(size_t)(s + v) * N + c] = lf[v];
  A.slot[(size_t)(s + 4) * N + c] = la;
}

// x faces first ((nx + 1) ny of them, x fastest), then y faces (nx (ny + 1)).
template <typename T>
__host__ __device__ void face_body(const AdjArgs<T>& A, long long idx) {
  const int nx = A.nx, ny = A.ny;
  const size_t N = (size_t)nx * ny;
  const long long nfx = (long long)(nx + 1) * ny;
  const Phys<T>& P = A.kc.P;
  const T rdx = A.dt / A.kc.dx, rdy = A.dt / A.kc.dy;
  T lDm[4] = {0, 0, 0, 0}, lDp[4] = {0, 0, 0, 0};
  T lqm[4] = {0, 0, 0, 0}, lqp[4] = {0, 0, 0, 0}, ldq[4] = {0, 0, 0, 0};
  if (idx < nfx) {
    const int f = (int)(idx % (nx + 1)), j = (int)(idx / (nx + 1));
    const bool L = fluid_at(A, f - 1, j), R = fluid_at(A, f, j);
    if (!L && !R) return;
    const size_t cL = (size_t)j * nx + (f - 1), cR = (size_t)j * nx + f;
    if (L)
#pragma unroll
      for (int v = 0; v < 4; ++v) lDm[v] = -rdx * (T)A.lam[v * N + cL];
    if (R)
#pragma unroll
      for (int v = 0; v < 4; ++v) lDp[v] = -rdx * (T)A.lam[v * N + cR];
    if (L && R) {
      const T mEL = A.rec[R_MEC * N + cL], mER = A.rec[R_MEC * N + cR];
      const T aL = A.rec[R_AE * N + cL], aR = A.rec[R_AE * N + cR];
      T fl[4], fr[4], qm[4], qp[4], dq[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        fl[v] = A.rec[(R_FE + v) * N + cL];
        fr[v] = A.rec[(R_FW + v) * N + cR];
      }
      qm[0] = mEL + fl[0]; qm[1] = fl[1]; qm[2] = fl[2]; qm[3] = aL + fl[3];
      qp[0] = mER + fr[0]; qp[1] = fr[1]; qp[2] = fr[2]; qp[3] = aR + fr[3];
      dq[0] = (mER - mEL) + (fr[0] - fl[0]);
      dq[1] = fr[1] - fl[1];
      dq[2] = fr[2] - fl[2];
      dq[3] = (aR - aL) + (fr[3] - fl[3]);
      xface_adj(qm, qp, dq, P, lDm, lDp, lqm, lqp, ldq);
      T sl[4], sr[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        sl[v] = lqm[v] - ldq[v];
        sr[v] = lqp[v] + ldq[v];
      }
      const int KL = A.Kcur[f - 1], KR = A.Kcur[f];
      const T rL = tab(A.rt, 2 * (j - KL) + 1, ny), rR = tab(A.rt, 2 * (j - KR) + 1, ny);
      put_slot(A, cL, S_E, sl, rL * sl[0] + sl[3]);
      put_slot(A, cR, S_W, sr, rR * sr[0] + sr[3]);
    } else {
      const size_t c = L ? cL : cR;
      const int ci = L ? f - 1 : f;
      const int bs = L ? R_FE : R_FW;
      const T mE = A.rec[R_MEC * N + c], aE = A.rec[R_AE * N + c];
      T q[4];
      q[0] = mE + A.rec[bs * N + c];
      q[1] = A.rec[(bs + 1) * N + c];
      q[2] = A.rec[(bs + 2) * N + c];
      q[3] = aE + A.rec[(bs + 3) * N + c];
      const bool outside = L ? f == nx : f == 0;
      const bool tr = outside && A.side[L ? 1 : 0] == 1;
      const T gsign = tr ? T(1) : T(-1);
      T g[4] = {q[0], gsign * q[1], q[2], q[3]}, qm[4], qp[4], dq[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        qm[v] = L ? q[v] : g[v];
        qp[v] = L ? g[v] : q[v];
      }
      dq[0] = T(0);
      dq[1] = qp[1] - qm[1];
      dq[2] = T(0);
      dq[3] = T(0);
      xface_adj(qm, qp, dq, P, lDm, lDp, lqm, lqp, ldq);
      // q enters as itself on its side, as the ghost g on the other, and in dq1
      T lq[4];
      const T* lown = L ? lqm : lqp;
      const T* lgh = L ? lqp : lqm;
#pragma unroll
      for (int v = 0; v < 4; ++v) lq[v] = lown[v] + (v == 1 ? gsign : T(1)) * lgh[v];
      // dq1 = qp1 - qm1 = +-(gsign - 1) q1
      lq[1] += (L ? (gsign - T(1)) : (T(1) - gsign)) * ldq[1];
      const int K = A.Kcur[ci];
      const T r = tab(A.rt, 2 * (j - K) + 1, ny);
      put_slot(A, c, L ? S_E : S_W, lq, r * lq[0] + lq[3]);
    }
  } else {
    const long long k = idx - nfx;
    const int i = (int)(k % nx), f = (int)(k / nx);
    const bool B = fluid_at(A, i, f - 1), Tt = fluid_at(A, i, f);
    if (!B && !Tt) return;
    const size_t cB = (size_t)(f - 1) * nx + i, cT = (size_t)f * nx + i;
    if (B)
#pragma unroll
      for (int v = 0; v < 4; ++v) lDm[v] = -rdy * (T)A.lam[v * N + cB];
    if (Tt)
#pragma unroll
      for (int v = 0; v < 4; ++v) lDp[v] = -rdy * (T)A.lam[v * N + cT];
    const int K = A.Kcur[i];
    const T rEf = tab(A.rt, 2 * (f - K), ny);
    if (B && Tt) {
      const T mEB = A.rec[R_MEN * N + cB], mET = A.rec[R_MES * N + cT];
      const T aB = A.rec[R_AE * N + cB], aT = A.rec[R_AE * N + cT];
      T fb[4], ft[4], qm[4], qp[4], dq[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        fb[v] = A.rec[(R_FN + v) * N + cB];
        ft[v] = A.rec[(R_FS + v) * N + cT];
      }
      qm[0] = mEB + fb[0]; qm[1] = fb[1]; qm[2] = fb[2]; qm[3] = aB + fb[3];
      qp[0] = mET + ft[0]; qp[1] = ft[1]; qp[2] = ft[2]; qp[3] = aT + ft[3];
      dq[0] = (mET - mEB) + (ft[0] - fb[0]);
      dq[1] = ft[1] - fb[1];
      dq[2] = ft[2] - fb[2];
      dq[3] = (aT - aB) + (ft[3] - fb[3]);
      const T dap = P.c2 * ((rEf - P.rho0) * (aT - aB) + ((ft[0] - fb[0]) - P.rho0 * (ft[3] - fb[3])));
      T ldap = T(0);
      yface_adj(qm, qp, dq, dap, P, lDm, lDp, lqm, lqp, ldq, ldap);
      const T cd = P.c2 * ldap;
      T sb[4], st[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        sb[v] = lqm[v] - ldq[v];
        st[v] = lqp[v] + ldq[v];
      }
      const T laB = rEf * sb[0] + sb[3] - cd * (rEf - P.rho0);
      const T laT = rEf * st[0] + st[3] + cd * (rEf - P.rho0);
      sb[0] -= cd;
      sb[3] += cd * P.rho0;
      st[0] += cd;
      st[3] -= cd * P.rho0;
      put_slot(A, cB, S_N, sb, laB);
      put_slot(A, cT, S_S, st, laT);
    } else {
      const size_t c = B ? cB : cT;
      const int bs = B ? R_FN : R_FS;
      const T mE = A.rec[(B ? R_MEN : R_MES) * N + c], aE = A.rec[R_AE * N + c];
      T q[4];
      q[0] = mE + A.rec[bs * N + c];
      q[1] = A.rec[(bs + 1) * N + c];
      q[2] = A.rec[(bs + 2) * N + c];
      q[3] = aE + A.rec[(bs + 3) * N + c];
      const bool outside = B ? f == ny : f == 0;
      const bool tr = outside && A.side[B ? 3 : 2] == 1;
      const T gsign = tr ? T(1) : T(-1);
      T g[4] = {q[0], q[1], gsign * q[2], q[3]}, qm[4], qp[4], dq[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        qm[v] = B ? q[v] : g[v];
        qp[v] = B ? g[v] : q[v];
      }
      dq[0] = T(0);
      dq[1] = T(0);
      dq[2] = qp[2] - qm[2];
      dq[3] = T(0);
      T ldap = T(0);
      yface_adj(qm, qp, dq, T(0), P, lDm, lDp, lqm, lqp, ldq, ldap);
      T lq[4];
      const T* lown = B ? lqm : lqp;
      const T* lgh = B ? lqp : lqm;
#pragma unroll
      for (int v = 0; v < 4; ++v) lq[v] = lown[v] + (v == 2 ? gsign : T(1)) * lgh[v];
      lq[2] += (B ? (gsign - T(1)) : (T(1) - gsign)) * ldq[2];
      put_slot(A, c, B ? S_N : S_S, lq, rEf * lq[0] + lq[3]);
    }
  }
}

// Double: at most 128 registers, so that two CTAs fit per SM (its subsonic and
// general branches of the reverse face solvers together take up to 140 when
// the compiler is left free).  Float takes 64 unbounded (four CTAs).
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 0 : 2) adj_face_kernel(AdjArgs<T> A) {
  const long long nf = (long long)(A.nx + 1) * A.ny + (long long)A.nx * (A.ny + 1);
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx < nf) face_body<T>(A, idx);
}

// ------------------------------------------------------------------ cells
template <typename T, bool DEV>
__host__ __device__ void cell_body(const AdjArgs<T>& A, int i, int j) {
  if (!fluid_at(A, i, j)) return;
  const size_t N = (size_t)A.nx * A.ny, c = (size_t)j * A.nx + i;
  CellRec<T> C;
  recon_cell<T, DEV>(A, i, j, C);
  const Phys<T>& P = A.kc.P;
  const T rdx = A.dt / A.kc.dx, rdy = A.dt / A.kc.dy;
  // adjoints of the face states (from the faces) and of the interior integral
  T lfo[4][4], lbase[4] = {0, 0, 0, 0}, lga[2] = {0, 0};
  T laE = 0, lmEc = 0, lmES = 0, lmEN = 0;
  const int sl[4] = {S_W, S_E, S_S, S_N};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int v = 0; v < 4; ++v) lfo[k][v] = A.slot[(size_t)(sl[k] + v) * N + c];
    laE += A.slot[(size_t)(sl[k] + 4) * N + c];
  }
  T lIx[4], lIy[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const T l = (T)A.lam[v * N + c];
    lIx[v] = -rdx * l;
    lIy[v] = -rdy * l;
  }
  interior_terms_adj(C.fo[0], C.fo[1], C.fo[2], C.fo[3], C.base, C.mEc, C.mES, C.mEN, C.ga[0],
                     C.ga[1], A.kc.dx, A.kc.dy, P, lIx, lIy, lfo[0], lfo[1], lfo[2], lfo[3], lbase,
                     lmEc, lmES, lmEN, lga[0], lga[1]);
  // adjoint of the reconstruction
  T lQf[4] = {0, 0, 0, 0}, lfi[4][4], lmx[4] = {0, 0, 0, 0}, lmn[4] = {0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int v = 0; v < 4; ++v) lfi[k][v] = T(0);
  T lfd[4][4];
#pragma unroll
  for (int d = 0; d < 4; ++d)
#pragma unroll
    for (int v = 0; v < 4; ++v) lfd[d][v] = T(0);
  if (C.first) {
    // face and centre states = Qf (Qf[3] = 0 is a constant)
#pragma unroll
    for (int v = 0; v < 3; ++v) lQf[v] = lbase[v] + lfo[0][v] + lfo[1][v] + lfo[2][v] + lfo[3][v];
  } else {
    recon_core_adj(C.Qf, C.fi[0], C.fi[1], C.fi[2], C.fi[3], C.mx, C.mn, C.aE, C.mEc, C.mES, C.mEN,
                   C.rEc, P, A.kc.R, lfo[0], lfo[1], lfo[2], lfo[3], lbase, lga, lQf, lfi[0], lfi[1],
                   lfi[2], lfi[3], lmx, lmn, laE, lmEc);
    // stencil extrema: to the first candidate attaining them, in the forward's order
  #pragma unroll
    for (int v = 0; v < 4; ++v) {
  #pragma unroll
      for (int pass = 0; pass < 2; ++pass) {
        const T target = pass == 0 ? C.mx[v] : C.mn[v];
        const T l = pass == 0 ? lmx[v] : lmn[v];
        if (C.Qf[v] == target) { lQf[v] += l; continue; }
        bool done = false;
  #pragma unroll
        for (int k = 0; k < 4; ++k)
          if (!done && C.fi[k][v] == target) { lfi[k][v] += l; done = true; }
  #pragma unroll
        for (int d = 0; d < 4; ++d)
          if (!done && C.dfl[d] && C.fd[d][v] == target) { lfd[d][v] += l; done = true; }
      }
    }
    // ghosts are (mirrored) copies of Qf; Qf[3] = 0 is a constant
  #pragma unroll
    for (int k = 0; k < 4; ++k)
      if (!C.nfl[k]) {
        lQf[0] += lfi[k][0];
        lQf[1] += (k < 2 && !C.ncopy[k]) ? -lfi[k][1] : lfi[k][1];
        lQf[2] += (k >= 2 && !C.ncopy[k]) ? -lfi[k][2] : lfi[k][2];
      }
  }
  // to the state: Qf = (m - aE rEc, mu, mv, 0); neighbour fluctuations
  // (m_n - aE rn, mu_n, mv_n, a_n - aE); equilibrium masses aE rE
  laE += C.rEc * lmEc + C.rES * lmES + C.rEN * lmEN - C.rEc * lQf[0];
  T out[9][4];
#pragma unroll
  for (int p = 0; p < 9; ++p)
#pragma unroll
    for (int v = 0; v < 4; ++v) out[p][v] = T(0);
  const int epos[4] = {3, 5, 1, 7};  // W, E, S, N in the 3x3 numbering (dj+1)*3 + (di+1)
  const int dpos[4] = {0, 2, 6, 8};
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (C.nfl[k]) {
#pragma unroll
      for (int v = 0; v < 4; ++v) out[epos[k]][v] = lfi[k][v];
      laE -= C.rn[k] * lfi[k][0] + lfi[k][3];
    }
#pragma unroll
  for (int d = 0; d < 4; ++d)
    if (C.dfl[d]) {
#pragma unroll
      for (int v = 0; v < 4; ++v) out[dpos[d]][v] = lfd[d][v];
      laE -= C.rd[d] * lfd[d][0] + lfd[d][3];
    }
  out[4][0] = lQf[0];
  out[4][1] = lQf[1];
  out[4][2] = lQf[2];
  out[4][3] = laE;
#pragma unroll
  for (int p = 0; p < 9; ++p)
#pragma unroll
    for (int v = 0; v < 4; ++v) A.contrib[(size_t)(4 * p + v) * N + c] = out[p][v];
}

// Float: at most 128 registers, so that four CTAs fit per SM (unbounded it
// takes 167 and three fit, and the 1024 CTAs of a 512 x 256 grid run in 2.25
// waves at 31 % issue activity).  Double needs about 250 and is left alone.
template <typename T, bool DEV>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1) adj_cell_kernel(AdjArgs<T> A) {
  const int i = blockIdx.x * 32 + (threadIdx.x & 31), j = blockIdx.y * 4 + (threadIdx.x >> 5);
  if (i < A.nx && j < A.ny) cell_body<T, DEV>(A, i, j);
}

// ------------------------------------------------------------------ gather
template <typename T>
__host__ __device__ void gather_body(const AdjArgs<T>& A, int i, int j) {
  const size_t N = (size_t)A.nx * A.ny, c = (size_t)j * A.nx + i;
  if (!fluid_at(A, i, j)) {
#pragma unroll
    for (int v = 0; v < 4; ++v) A.lam_out[v * N + c] = 0.0;
    return;
  }
  // every load is issued before any is used (no branch between them); a source
  // outside the fluid contributes nothing but is read at the cell's own index
  bool ok[9];
  size_t src[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const int di = p % 3 - 1, dj = p / 3 - 1;
    const int si = i - di, sj = j - dj;
    ok[p] = fluid_at(A, si, sj);
    src[p] = ok[p] ? (size_t)sj * A.nx + si : c;
  }
  T val[9][4];
#pragma unroll
  for (int p = 0; p < 9; ++p)
#pragma unroll
    for (int v = 0; v < 4; ++v) val[p][v] = A.contrib[(size_t)(4 * p + v) * N + src[p]];
  double acc[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) acc[v] = A.lam[v * N + c];
  // fixed order: dj = -1..1, di = -1..1 (p = (dj+1)*3 + (di+1))
  if constexpr (sizeof(T) == 4) {
    // float contributions: summed by compensated float summation (TwoSum,
    // Knuth), whose hi + lo carries their sum to about 2^-48 relative, then
    // added to the double accumulator once (hi + lo is exact in double); the
    // double pipe, 1/64 of the float rate here, does 4 operations per
    // component instead of 18
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float hi = 0.0f, lo = 0.0f;
#pragma unroll
      for (int p = 0; p < 9; ++p) {
        const float x = ok[p] ? (float)val[p][v] : 0.0f;
        const float sum = hi + x;
        const float bb = sum - hi;
        lo += (hi - (sum - bb)) + (x - bb);
        hi = sum;
      }
      acc[v] += (double)hi + (double)lo;
    }
  } else {
#pragma unroll
    for (int p = 0; p < 9; ++p)
      if (ok[p])
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v] += (double)val[p][v];
  }
  if (A.src_dt != 0.0) {
    const int k0 = A.gmark[c];
    if (k0 >= 0)
      for (int k = k0; k < A.ng && A.gauges[A.gord[k]] == (int64_t)c; ++k)
        acc[0] += 2.0 * A.src_dt * (A.src_m[A.gord[k]] - A.src_t[A.gord[k]]);
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) A.lam_out[v * N + c] = acc[v];
}

template <typename T>
__global__ void __launch_bounds__(BX * BY) adj_gather_kernel(AdjArgs<T> A) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  if (i < A.nx && j < A.ny) gather_body<T>(A, i, j);
}

// ------------------------------------------------------------------ heights
// Derivative of one step with respect to obstacle heights, at theta = 0+ of
// the extension in which raising obstacle k by theta dy leaves each of its
// top fluid cells P the capacity c = 1 - theta.  With every face value of the
// step fixed, only the update's weights move:
//   P:  x terms (open length c dy over volume c dx dy) unchanged; y terms
//       D+_S + D-_N + (y jumps of the interior integral) divided by c; the
//       gravity integral (proportional to the height) unchanged, so
//       dQ_P/dtheta = -dt/dy (D+_S + D-_N + jumps);
//   F:  a fluid x neighbour of P that is not a top cell of the same obstacle
//       sees its face open over c dy and closed (a wall) over theta dy:
//       dQ_F/dtheta = dt/dx (D_F(face) - D_F(wall)).
// The contribution of P to dL/dtheta_k at step n is lambda^n . dQ^n/dtheta
// in storage form.

// The y terms of the interior integral (interior_terms) without the gravity
// integral g dy (alpha rho)^f.
template <typename T>
__host__ __device__ __forceinline__ void y_jumps(const T fS[4], const T fN[4], const T base[4],
                                                 T mEc, T mES, T mEN, T day, T dy,
                                                 const Phys<T>& P, T Iy[4]) {
  const Vel<T> vN = velocity(mEN + fN[0], fN[1], fN[2]);
  const Vel<T> vS = velocity(mES + fS[0], fS[1], fS[2]);
  const Vel<T> vc = velocity(mEc + base[0], base[1], base[2]);
  Iy[0] = fN[2] - fS[2];
  Iy[1] = fN[1] * vN.v - fS[1] * vS.v;
  Iy[2] = (fN[2] * vN.v - fS[2] * vS.v) + P.c2 * ((fN[0] - fS[0]) - P.rho0 * (fN[3] - fS[3]));
  Iy[3] = dy * vc.v * day;
}

// lambda . dq for a storage-form derivative (the deviation form stores
// alpha rho - alpha rho^E_c, so da also moves the first component).
template <typename T, bool DEV>
__host__ __device__ __forceinline__ double lam_dot(const AdjArgs<T>& A, size_t c, const T d[4], T rEc) {
  const size_t N = (size_t)A.nx * A.ny;
  const T d0 = DEV ? d[0] - rEc * d[3] : d[0];
  return A.lam[c] * (double)d0 + A.lam[N + c] * (double)d[1] + A.lam[2 * N + c] * (double)d[2] +
         A.lam[3 * N + c] * (double)d[3];
}

// Contribution of top cell c (hid[c] = k >= 0) to dL/dtheta_k at this step;
// A.rec holds the step's records, A.lam the adjoint of Q^n.
template <typename T, bool DEV>
__host__ __device__ double height_body(const AdjArgs<T>& A, const int32_t* hid, int64_t c) {
  const int nx = A.nx, ny = A.ny;
  const size_t N = (size_t)nx * ny;
  const int i = (int)(c % nx), j = (int)(c / nx);
  const int k = hid[c];
  const Phys<T>& P = A.kc.P;
  const T rdx = A.dt / A.kc.dx, rdy = A.dt / A.kc.dy;
  CellRec<T> C;
  recon_cell<T, DEV>(A, i, j, C);
  T Dm[4], Dp[4], qm[4], qp[4], dq[4];
  // south face: the obstacle's top, a wall below P
  const T* fs = C.fo[2];
#pragma unroll
  for (int v = 0; v < 4; ++v) qp[v] = fs[v];
  qp[0] += C.mES;
  qp[3] += C.aE;
#pragma unroll
  for (int v = 0; v < 4; ++v) qm[v] = qp[v];
  qm[2] = -qp[2];
  dq[0] = T(0);
  dq[1] = T(0);
  dq[2] = qp[2] - qm[2];
  dq[3] = T(0);
  yface(qm, qp, dq, T(0), P, Dm, Dp);
  T ys[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) ys[v] = Dp[v];
  // north face
  const T* fb = C.fo[3];
  if (fluid_at(A, i, j + 1)) {
    const size_t cT = (size_t)c + nx;
    const T mET = A.rec[R_MES * N + cT], aT = A.rec[R_AE * N + cT];
    T ft[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) ft[v] = A.rec[(R_FS + v) * N + cT];
    qm[0] = C.mEN + fb[0]; qm[1] = fb[1]; qm[2] = fb[2]; qm[3] = C.aE + fb[3];
    qp[0] = mET + ft[0]; qp[1] = ft[1]; qp[2] = ft[2]; qp[3] = aT + ft[3];
    dq[0] = (mET - C.mEN) + (ft[0] - fb[0]);
    dq[1] = ft[1] - fb[1];
    dq[2] = ft[2] - fb[2];
    dq[3] = (aT - C.aE) + (ft[3] - fb[3]);
    const T rEf = tab(A.rt, 2 * (j + 1 - A.Kcur[i]), ny);
    const T dap = P.c2 * ((rEf - P.rho0) * (aT - C.aE) + ((ft[0] - fb[0]) - P.rho0 * (ft[3] - fb[3])));
    yface(qm, qp, dq, dap, P, Dm, Dp);
  } else {
    qm[0] = C.mEN + fb[0]; qm[1] = fb[1]; qm[2] = fb[2]; qm[3] = C.aE + fb[3];
    const bool tr = j + 1 == ny && A.side[3] == 1;
#pragma unroll
    for (int v = 0; v < 4; ++v) qp[v] = qm[v];
    if (!tr) qp[2] = -qm[2];
    dq[0] = T(0);
    dq[1] = T(0);
    dq[2] = qp[2] - qm[2];
    dq[3] = T(0);
    yface(qm, qp, dq, T(0), P, Dm, Dp);
  }
  T Iy[4], d[4];
  y_jumps(C.fo[2], C.fo[3], C.base, C.mEc, C.mES, C.mEN, C.ga[1], A.kc.dy, P, Iy);
#pragma unroll
  for (int v = 0; v < 4; ++v) d[v] = -rdy * (ys[v] + Dm[v] + Iy[v]);
  double acc = lam_dot<T, DEV>(A, (size_t)c, d, C.rEc);
  // x neighbours: west (side 0) and east (side 1)
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    const int fi = sd == 0 ? i - 1 : i + 1;
    if (!fluid_at(A, fi, j)) continue;
    const size_t cF = (size_t)j * nx + fi;
    if (hid[cF] == k) continue;
    const T mEF = A.rec[R_MEC * N + cF], aF = A.rec[R_AE * N + cF];
    T fF[4];
    const int bs = sd == 0 ? R_FE : R_FW;  // F's face state toward P
#pragma unroll
    for (int v = 0; v < 4; ++v) fF[v] = A.rec[(bs + v) * N + cF];
    const T* fP = C.fo[sd == 0 ? 0 : 1];   // P's face state toward F
    T qF[4] = {mEF + fF[0], fF[1], fF[2], aF + fF[3]};
    T qP[4] = {C.mEc + fP[0], fP[1], fP[2], C.aE + fP[3]};
    const T* ql = sd == 0 ? qF : qP;
    const T* qr = sd == 0 ? qP : qF;
    const T* fl = sd == 0 ? fF : fP;
    const T* fr = sd == 0 ? fP : fF;
    const T mEl = sd == 0 ? mEF : C.mEc, mEr = sd == 0 ? C.mEc : mEF;
    const T al = sd == 0 ? aF : C.aE, ar = sd == 0 ? C.aE : aF;
    dq[0] = (mEr - mEl) + (fr[0] - fl[0]);
    dq[1] = fr[1] - fl[1];
    dq[2] = fr[2] - fl[2];
    dq[3] = (ar - al) + (fr[3] - fl[3]);
    xface(ql, qr, dq, P, Dm, Dp);
    T DF[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) DF[v] = sd == 0 ? Dm[v] : Dp[v];
    // the same face closed, seen from F
    T g[4] = {qF[0], -qF[1], qF[2], qF[3]};
    const T* wl = sd == 0 ? qF : g;
    const T* wr = sd == 0 ? g : qF;
    dq[0] = T(0);
    dq[1] = wr[1] - wl[1];
    dq[2] = T(0);
    dq[3] = T(0);
    xface(wl, wr, dq, P, Dm, Dp);
#pragma unroll
    for (int v = 0; v < 4; ++v) d[v] = rdx * (DF[v] - (sd == 0 ? Dm[v] : Dp[v]));
    const T rEcF = tab(A.rt, 2 * (j - A.Kcur[fi]) + 1, ny);
    acc += lam_dot<T, DEV>(A, cF, d, rEcF);
  }
  return acc;
}

// hacc[p] += the contribution of top cell hcell[p] at this step (one writer
// per entry; the per-obstacle sums are taken on the host in list order).
template <typename T, bool DEV>
__global__ void __launch_bounds__(128) adj_height_kernel(AdjArgs<T> A, const int64_t* hcell,
                                                         int nh, const int32_t* hid,
                                                         double* hacc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nh) hacc[p] += height_body<T, DEV>(A, hid, hcell[p]);
}

// ------------------------------------------------------------------ small kernels
// Loss source of step n: d/dm_g of dt_n (m_g - T_g)^2, gauges in order.
__global__ void adj_source_kernel(double* lam, const int64_t* gauges, int ng, const double* m,
                                  const double* target, double dt) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int g = 0; g < ng; ++g) lam[gauges[g]] += 2.0 * dt * (m[g] - target[g]);
}

// Levels and dt the next step uses.
__global__ void adj_record_kernel(int nx, const int32_t* Kcur, int32_t* Krow, const DevScalars* sc,
                                  double* dt_slot) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x)
    Krow[i] = Kcur[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) *dt_slot = sc->dt_cur;
}

// After step n of the forward sweep, one launch: alpha rho at the gauges of
// Q^n, stored relative to the levels Kq it was computed with (double), and
// the levels and dt step n + 1 will use (Krow null after the last step).
template <typename T, bool DEV>
__global__ void adj_after_step_kernel(int nx, int ny, const T* q, const int32_t* Kq,
                                      const double* rhoE, const int64_t* gauges, int ng,
                                      double* out, const int32_t* Kcur, int32_t* Krow,
                                      const DevScalars* sc, double* dt_slot) {
  const size_t N = (size_t)nx * ny;
  if (blockIdx.x == 0)
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
      const int64_t c = gauges[g];
      if (DEV) {
        const int i = (int)(c % nx), j = (int)(c / nx);
        out[g] = (double)q[3 * N + c] * rhoE[2 * (j - Kq[i]) + 1 + 2 * ny] + (double)q[c];
      } else {
        out[g] = (double)q[c];
      }
    }
  if (Krow) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x)
      Krow[i] = Kcur[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) *dt_slot = sc->dt_cur;
  }
}

__global__ void adj_set_dt_kernel(DevScalars* sc, double dt) {
  sc->dt_cur = dt;
  sc->dt_cur_f = (float)dt;
}

// ------------------------------------------------------------------ host
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { cudaFree(p); }
  bool alloc(size_t bytes) {
    if (cudaMalloc(&p, bytes ? bytes : 1) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return false;
    }
    return true;
  }
  template <typename U>
  U* as() const { return (U*)p; }
};

struct OwnedStream {
  cudaStream_t s = nullptr;
  ~OwnedStream() {
    if (s) cudaStreamDestroy(s);
  }
};

struct OwnedEvent {
  cudaEvent_t e = nullptr;
  ~OwnedEvent() {
    if (e) cudaEventDestroy(e);
  }
};

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Obstacle-height work of a reverse step, run on its own stream between the
// step's rec kernel and the next step's (which overwrites the records).
struct HeightWork {
  int nh = 0;
  const int64_t* hcell = nullptr;
  const int32_t* hid = nullptr;
  double* hacc = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t rec_done = nullptr, done = nullptr;
};

template <typename T, bool DEV>
void launch_reverse_step(AdjArgs<T> A, cudaStream_t st, const HeightWork& H) {
  const dim3 b2(BX, BY), g2((A.nx + BX - 1) / BX, (A.ny + BY - 1) / BY);
  if (H.nh > 0) cudaStreamWaitEvent(st, H.done, 0);  // the previous step's height kernel
  adj_rec_kernel<T, DEV><<<g2, b2, 0, st>>>(A);
  if (H.nh > 0) {
    // reads the records and the adjoint of Q^n while faces, cells and gather run
    cudaEventRecord(H.rec_done, st);
    cudaStreamWaitEvent(H.st, H.rec_done, 0);
    adj_height_kernel<T, DEV><<<(H.nh + 127) / 128, 128, 0, H.st>>>(A, H.hcell, H.nh, H.hid, H.hacc);
    cudaEventRecord(H.done, H.st);
  }
  const long long nf = (long long)(A.nx + 1) * A.ny + (long long)A.nx * (A.ny + 1);
  adj_face_kernel<T><<<(unsigned)((nf + 255) / 256), 256, 0, st>>>(A);
  const dim3 g3((A.nx + 31) / 32, (A.ny + 3) / 4);
  adj_cell_kernel<T, DEV><<<g3, 128, 0, st>>>(A);
  adj_gather_kernel<T><<<g2, b2, 0, st>>>(A);
}

template <typename T, bool DEV>
void launch_replay_step(const StepParams& p, const T* in, T* out, const uint8_t* solid,
                        const int32_t* Kref, const int32_t* Kcur, unsigned long long* colsum,
                        DevScalars* sc, const Tables& tb, int tiling, int strip_h,
                        cudaStream_t st) {
  if (DEV) {
    StateF32 s{(const float*)in, (float*)out};
    launch_step_f32(p, s, solid, Kref, Kcur, colsum, sc, tb, st, false, tiling, strip_h);
  } else {
    StateF64 s{(const double*)in, (double*)out};
    launch_step_f64(p, s, solid, Kcur, colsum, sc, tb, st, false, tiling, strip_h);
  }
}

template <typename T, bool DEV>
fv_status run_adjoint(fv_handle* h, const fv_adjoint_spec* spec, double* grad, int on_device,
                      fv_adjoint_info* info, const std::vector<int64_t>& hcell_h) {
  const int nx = h->grid.nx, ny = h->grid.ny, Nst = spec->nsteps, ng = spec->ngauges;
  const size_t N = h->ncell;
  const size_t qbytes = 4 * N * sizeof(T);
  const int s = spec->checkpoint_every > 0 ? std::min(spec->checkpoint_every, Nst)
                                           : (int)std::ceil(std::sqrt((double)Nst));
  const int nck = (Nst + s - 1) / s;
  const size_t segs = (size_t)std::max(1, s - 1);  // replayed states per segment
  cudaStream_t st = h->stream;
  const StepParams p = params_of(h, spec->cfl);
  const Tables tb{h->d_rhoE, h->d_rhoE_f};
  const T* rt = DEV ? (const T*)h->d_rhoE_f : (const T*)h->d_rhoE;

  DevBuf Khist, dthist, gidx, gval, tgt, ckpt, seg, lamA, lamB, rec, slot, contrib, rsc, rcol,
      gmark, gord;
  const bool ok =
      Khist.alloc(sizeof(int32_t) * (size_t)nx * (Nst + 1)) &&
      dthist.alloc(sizeof(double) * (Nst + 1)) && gidx.alloc(sizeof(int64_t) * ng) &&
      gval.alloc(sizeof(double) * (size_t)Nst * ng) && tgt.alloc(sizeof(double) * (size_t)Nst * ng) &&
      ckpt.alloc(qbytes * nck) && seg.alloc(qbytes * 2 * segs) &&
      lamA.alloc(sizeof(double) * 4 * N) && lamB.alloc(sizeof(double) * 4 * N) &&
      rec.alloc(sizeof(T) * NREC * N) && slot.alloc(sizeof(T) * NSLOT * N) &&
      contrib.alloc(sizeof(T) * NCONTRIB * N) && rsc.alloc(sizeof(DevScalars)) &&
      rcol.alloc(sizeof(unsigned long long) * nx) && gmark.alloc(sizeof(int32_t) * N) &&
      gord.alloc(sizeof(int32_t) * ng);
  const int nh = (int)hcell_h.size();
  DevBuf hcell, hid, hacc;
  const bool okh = nh == 0 || (hcell.alloc(sizeof(int64_t) * nh) &&
                               hid.alloc(sizeof(int32_t) * N) && hacc.alloc(sizeof(double) * nh));
  if (!ok || !okh) {
    set_last_error("fv_adjoint: device allocation failed");
    return FV_ENOMEM;
  }
  auto cuda_err = [](cudaError_t e, const char* where) {
    set_last_error((std::string("fv_adjoint: ") + where + ": " + cudaGetErrorString(e)).c_str());
    return FV_ECUDA;
  };
#define ADJ_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_err(e_, #call);   \
  } while (0)
  ADJ_CUDA(cudaMemcpyAsync(gidx.p, spec->gauges, sizeof(int64_t) * ng, cudaMemcpyHostToDevice, st));
  ADJ_CUDA(cudaMemcpyAsync(tgt.p, spec->target, sizeof(double) * (size_t)Nst * ng,
                           cudaMemcpyHostToDevice, st));
  // gauges in cell order (stable), and each gauge cell's first position in it
  std::vector<int32_t> ord_h(ng), mark_h(N, -1);
  for (int g = 0; g < ng; ++g) ord_h[g] = g;
  std::stable_sort(ord_h.begin(), ord_h.end(),
                   [&](int32_t a, int32_t b) { return spec->gauges[a] < spec->gauges[b]; });
  for (int k = ng - 1; k >= 0; --k) mark_h[spec->gauges[ord_h[k]]] = k;
  ADJ_CUDA(cudaMemcpyAsync(gord.p, ord_h.data(), sizeof(int32_t) * ng, cudaMemcpyHostToDevice, st));
  ADJ_CUDA(cudaMemcpyAsync(gmark.p, mark_h.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
  if (nh > 0) {
    ADJ_CUDA(cudaMemcpyAsync(hcell.p, hcell_h.data(), sizeof(int64_t) * nh, cudaMemcpyHostToDevice, st));
    ADJ_CUDA(cudaMemcpyAsync(hid.p, spec->height_id, sizeof(int32_t) * N, cudaMemcpyHostToDevice, st));
    ADJ_CUDA(cudaMemsetAsync(hacc.p, 0, sizeof(double) * nh, st));
  }
  ADJ_CUDA(cudaMemsetAsync(rsc.p, 0, sizeof(DevScalars), st));
  ADJ_CUDA(cudaMemsetAsync(rcol.p, 0, sizeof(unsigned long long) * nx, st));
  int32_t* Kh = Khist.as<int32_t>();
  double* dth = dthist.as<double>();
  EventPair evf, evr;
  OwnedStream st2;
  OwnedEvent ev_start, ev_rep[2], ev_rev[2];
  ADJ_CUDA(cudaStreamCreateWithFlags(&st2.s, cudaStreamNonBlocking));
  ADJ_CUDA(cudaEventCreateWithFlags(&ev_start.e, cudaEventDisableTiming));
  for (int k = 0; k < 2; ++k) {
    ADJ_CUDA(cudaEventCreateWithFlags(&ev_rep[k].e, cudaEventDisableTiming));
    ADJ_CUDA(cudaEventCreateWithFlags(&ev_rev[k].e, cudaEventDisableTiming));
  }
  OwnedStream st3;
  OwnedEvent ev_hrec, ev_hdone;
  HeightWork hw;
  if (nh > 0) {
    ADJ_CUDA(cudaStreamCreateWithFlags(&st3.s, cudaStreamNonBlocking));
    ADJ_CUDA(cudaEventCreateWithFlags(&ev_hrec.e, cudaEventDisableTiming));
    ADJ_CUDA(cudaEventCreateWithFlags(&ev_hdone.e, cudaEventDisableTiming));
    hw.nh = nh;
    hw.hcell = hcell.as<int64_t>();
    hw.hid = hid.as<int32_t>();
    hw.hacc = hacc.as<double>();
    hw.st = st3.s;
    hw.rec_done = ev_hrec.e;
    hw.done = ev_hdone.e;
  }
  ADJ_CUDA(cudaEventCreate(&evf.a));
  ADJ_CUDA(cudaEventCreate(&evf.b));
  ADJ_CUDA(cudaEventCreate(&evr.a));
  ADJ_CUDA(cudaEventCreate(&evr.b));

  // ---- forward sweep: states every s steps, levels, dt and gauge values of every step
  ADJ_CUDA(cudaEventRecord(evf.a, st));
  ADJ_CUDA(cudaMemcpyAsync(Kh, h->d_Kref, sizeof(int32_t) * nx, cudaMemcpyDeviceToDevice, st));
  launch_prepare(spec->cfl, h->d_sc, st);
  h->cfl = spec->cfl;
  const int rb = std::max(1, std::min(1024, (nx + 255) / 256));
  adj_record_kernel<<<rb, 256, 0, st>>>(nx, h->d_Kcur, Kh + (size_t)nx, h->d_sc, dth + 1);
  for (int n = 1; n <= Nst; ++n) {
    if ((n - 1) % s == 0)
      ADJ_CUDA(cudaMemcpyAsync(ckpt.as<char>() + qbytes * ((n - 1) / s), h->d_q[h->cur], qbytes,
                               cudaMemcpyDeviceToDevice, st));
    const int a = h->cur, b = 1 - h->cur;
    launch_replay_step<T, DEV>(p, (const T*)h->d_q[a], (T*)h->d_q[b], h->d_solid, h->d_Kref,
                               h->d_Kcur, h->d_colsum, h->d_sc, tb, h->tiling, h->strip_h, st);
    launch_finalize(p, h->d_Kref, h->d_Kcur, h->d_colsum, h->d_sc, 1, st);
    h->cur = b;
    adj_after_step_kernel<T, DEV><<<rb, 256, 0, st>>>(
        nx, ny, (const T*)h->d_q[b], Kh + (size_t)n * nx, h->d_rhoE, gidx.as<int64_t>(), ng,
        gval.as<double>() + (size_t)(n - 1) * ng, h->d_Kcur,
        n < Nst ? Kh + (size_t)(n + 1) * nx : nullptr, h->d_sc, dth + n + 1);
  }
  ADJ_CUDA(cudaGetLastError());
  ADJ_CUDA(cudaEventRecord(evf.b, st));
  std::vector<double> dt_h(Nst + 1), gv_h((size_t)Nst * ng);
  DevScalars sc_h;
  ADJ_CUDA(cudaMemcpyAsync(dt_h.data(), dth, sizeof(double) * (Nst + 1), cudaMemcpyDeviceToHost, st));
  ADJ_CUDA(cudaMemcpyAsync(gv_h.data(), gval.p, sizeof(double) * gv_h.size(), cudaMemcpyDeviceToHost, st));
  ADJ_CUDA(cudaMemcpyAsync(&sc_h, h->d_sc, sizeof(sc_h), cudaMemcpyDeviceToHost, st));
  ADJ_CUDA(cudaStreamSynchronize(st));
  if (sc_h.status) {
    set_last_error("fv_adjoint: a forward step produced a non-admissible state");
    return FV_ENONFINITE;
  }
  double loss = 0.0;
  for (int n = 1; n <= Nst; ++n) {
    double sn = 0.0;
    for (int g = 0; g < ng; ++g) {
      const double d = gv_h[(size_t)(n - 1) * ng + g] - spec->target[(size_t)(n - 1) * ng + g];
      sn += d * d;
    }
    loss += dt_h[n] * sn;
  }
  if (spec->m_series) std::memcpy(spec->m_series, gv_h.data(), sizeof(double) * gv_h.size());

  // ---- reverse sweep
  ADJ_CUDA(cudaEventRecord(evr.a, st));
  ADJ_CUDA(cudaMemsetAsync(lamA.p, 0, sizeof(double) * 4 * N, st));
  double* lam = lamA.as<double>();
  double* lam2 = lamB.as<double>();
  AdjArgs<T> A;
  A.nx = nx;
  A.ny = ny;
  for (int k = 0; k < 4; ++k) A.side[k] = h->side[k];
  A.kc = make_consts<T>(p);
  A.solid = h->d_solid;
  A.rt = rt;
  A.rec = rec.as<T>();
  A.slot = slot.as<T>();
  A.contrib = contrib.as<T>();
  A.gmark = gmark.as<int32_t>();
  A.gord = gord.as<int32_t>();
  A.gauges = gidx.as<int64_t>();
  A.ng = ng;
  // Segment k is replayed into seg set k % 2 on the second stream while the
  // reverse of segment k + 1 runs on the handle's stream.
  long long replayed = 0;
  auto state = [&](int k, int n) -> T* {  // Q^n of segment k (k s <= n < min(N, k s + s))
    const int n0 = k * s;
    if (n == n0) return (T*)(ckpt.as<char>() + qbytes * k);
    return (T*)(seg.as<char>() + qbytes * ((size_t)(k % 2) * segs + (n - n0 - 1)));
  };
  auto replay = [&](int k) {
    const int n0 = k * s, n1 = std::min(Nst, n0 + s);
    for (int n = n0 + 1; n < n1; ++n) {
      adj_set_dt_kernel<<<1, 1, 0, st2.s>>>(rsc.as<DevScalars>(), dt_h[n]);
      launch_replay_step<T, DEV>(p, state(k, n - 1), state(k, n), h->d_solid,
                                 Kh + (size_t)(n - 1) * nx, Kh + (size_t)n * nx,
                                 rcol.as<unsigned long long>(), rsc.as<DevScalars>(), tb,
                                 h->tiling, h->strip_h, st2.s);
      ++replayed;
    }
  };
  ADJ_CUDA(cudaEventRecord(ev_start.e, st));
  ADJ_CUDA(cudaStreamWaitEvent(st2.s, ev_start.e, 0));
  replay(nck - 1);
  ADJ_CUDA(cudaEventRecord(ev_rep[(nck - 1) % 2].e, st2.s));
  for (int k = nck - 1; k >= 0; --k) {
    const int n0 = k * s, n1 = std::min(Nst, n0 + s);
    ADJ_CUDA(cudaStreamWaitEvent(st, ev_rep[k % 2].e, 0));
    if (k >= 1) {
      // seg set (k - 1) % 2 was last read by the reverse of segment k + 1
      if (k + 1 < nck) ADJ_CUDA(cudaStreamWaitEvent(st2.s, ev_rev[(k + 1) % 2].e, 0));
      replay(k - 1);
      ADJ_CUDA(cudaEventRecord(ev_rep[(k - 1) % 2].e, st2.s));
    }
    for (int n = n1; n > n0; --n) {
      if (n == Nst)  // the source of Q^N; later sources are added by the gather
        adj_source_kernel<<<1, 1, 0, st>>>(lam, gidx.as<int64_t>(), ng,
                                           gval.as<double>() + (size_t)(n - 1) * ng,
                                           tgt.as<double>() + (size_t)(n - 1) * ng, dt_h[n]);
      // the gather of this step adds the source of Q^{n-1} (none for Q^0)
      A.src_dt = n >= 2 ? dt_h[n - 1] : 0.0;
      A.src_m = gval.as<double>() + (size_t)(n >= 2 ? n - 2 : 0) * ng;
      A.src_t = tgt.as<double>() + (size_t)(n >= 2 ? n - 2 : 0) * ng;
      A.dt = (T)dt_h[n];
      A.kc.R.half_dt = T(0.5) * A.dt;
      A.q = state(k, n - 1);
      A.Kref = Kh + (size_t)(n - 1) * nx;
      A.Kcur = Kh + (size_t)n * nx;
      A.lam = lam;
      A.lam_out = lam2;
      launch_reverse_step<T, DEV>(A, st, hw);
      std::swap(lam, lam2);
    }
    ADJ_CUDA(cudaEventRecord(ev_rev[k % 2].e, st));
  }
  if (nh > 0) ADJ_CUDA(cudaStreamWaitEvent(st, hw.done, 0));
  ADJ_CUDA(cudaGetLastError());
  ADJ_CUDA(cudaEventRecord(evr.b, st));
  ADJ_CUDA(cudaMemcpyAsync(grad, lam, sizeof(double) * 4 * N,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  std::vector<double> hacc_h(nh);
  if (nh > 0)
    ADJ_CUDA(cudaMemcpyAsync(hacc_h.data(), hacc.p, sizeof(double) * nh, cudaMemcpyDeviceToHost, st));
  ADJ_CUDA(cudaStreamSynchronize(st));
  if (spec->nheights > 0) {
    // dL/dh_k = (1/dy) sum of the top cells' dL/dtheta_k, in list order
    for (int k = 0; k < spec->nheights; ++k) spec->dL_dh[k] = 0.0;
    for (int q = 0; q < nh; ++q) spec->dL_dh[spec->height_id[hcell_h[q]]] += hacc_h[q];
    for (int k = 0; k < spec->nheights; ++k) spec->dL_dh[k] /= h->grid.dy;
  }
  if (info) {
    float fms = 0.f, rms = 0.f;
    ADJ_CUDA(cudaEventElapsedTime(&fms, evf.a, evf.b));
    ADJ_CUDA(cudaEventElapsedTime(&rms, evr.a, evr.b));
    info->loss = loss;
    info->t = sc_h.t;
    info->checkpoints = nck;
    info->recomputed_steps = (int32_t)replayed;
    info->forward_ms = fms;
    info->reverse_ms = rms;
  }
#undef ADJ_CUDA
  return FV_OK;
}

}  // namespace
}  // namespace fv

namespace fv {
namespace {

// Top cells named by height_id, in cell order; false on an invalid map.
bool height_cells(int nx, int ny, const uint8_t* solid, int nheights, const int32_t* height_id,
                  const double* dL_dh, std::vector<int64_t>& out) {
  out.clear();
  if (nheights < 0 || (nheights > 0) != (height_id != nullptr) ||
      (nheights > 0) != (dL_dh != nullptr))
    return false;
  if (nheights == 0) return true;
  const size_t N = (size_t)nx * ny;
  for (size_t c = 0; c < N; ++c) {
    const int32_t k = height_id[c];
    if (k == -1) continue;
    if (k < -1 || k >= nheights) return false;
    if (solid[c] || c < (size_t)nx || !solid[c - nx]) return false;
    out.push_back((int64_t)c);
  }
  return true;
}

// Buffers and arguments of one reverse step on the host.
template <typename T, bool DEV>
struct HostStep {
  std::vector<double> rtd;
  std::vector<T> rt, qs, rec, slot, contrib;
  AdjArgs<T> A;
  HostStep(const StepParams& p, const int32_t* side, const uint8_t* solid, const double* q,
           const int32_t* K, double dt, const double* lam) {
    const int nx = p.nx, ny = p.ny;
    const size_t N = (size_t)nx * ny;
    rtd.resize(4 * (size_t)ny + 1);
    for (long h2 = -2L * ny; h2 <= 2L * ny; ++h2)
      rtd[h2 + 2L * ny] = p.rho0 * std::exp(-p.kappa * (0.5 * (double)h2) * p.dy);
    rt.resize(rtd.size());
    qs.resize(4 * N);
    rec.assign(NREC * N, T(0));
    slot.assign(NSLOT * N, T(0));
    contrib.assign(NCONTRIB * N, T(0));
    for (size_t k = 0; k < rtd.size(); ++k) rt[k] = (T)rtd[k];
    // storage form: the full state (FP64) or m^f = m - alpha rho^E relative to K (deviation form)
    for (size_t c = 0; c < N; ++c) {
      const int i = (int)(c % nx), j = (int)(c / nx);
      const double m =
          solid[c] ? 0.0 : q[c] - (DEV ? q[3 * N + c] * rtd[2 * (j - K[i]) + 1 + 2 * ny] : 0.0);
      qs[c] = (T)m;
      for (int v = 1; v < 4; ++v) qs[v * N + c] = (T)q[v * N + c];
    }
    A.nx = nx;
    A.ny = ny;
    for (int k = 0; k < 4; ++k) A.side[k] = side[k];
    A.kc = make_consts<T>(p);
    A.dt = (T)dt;
    A.kc.R.half_dt = T(0.5) * A.dt;
    A.q = qs.data();
    A.solid = solid;
    A.Kref = K;
    A.Kcur = K;
    A.rt = rt.data();
    A.lam = lam;
    A.rec = rec.data();
    A.slot = slot.data();
    A.contrib = contrib.data();
    A.lam_out = nullptr;
    A.gmark = nullptr;
    A.gord = nullptr;
    A.gauges = nullptr;
    A.ng = 0;
    A.src_m = A.src_t = nullptr;
    A.src_dt = 0.0;
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) rec_body<T, DEV>(A, i, j);
  }
};

template <typename T, bool DEV>
void host_reverse_step(const StepParams& p, const int32_t* side, const uint8_t* solid,
                       const double* q, const int32_t* K, double dt, const double* lam,
                       double* lam_out) {
  HostStep<T, DEV> H(p, side, solid, q, K, dt, lam);
  AdjArgs<T>& A = H.A;
  A.lam_out = lam_out;
  const int nx = p.nx, ny = p.ny;
  const long long nf = (long long)(nx + 1) * ny + (long long)nx * (ny + 1);
  for (long long f = 0; f < nf; ++f) face_body<T>(A, f);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) cell_body<T, DEV>(A, i, j);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) gather_body<T>(A, i, j);
}

StepParams host_params(const fv_grid* grid, const fv_eos* eos, const int32_t side[4]) {
  StepParams p;
  p.nx = grid->nx;
  p.ny = grid->ny;
  p.dx = grid->dx;
  p.dy = grid->dy;
  p.rho0 = eos->rho0;
  p.k0 = eos->k0;
  p.g = eos->g;
  p.eps = eos->eps_gas;
  p.c2 = eos->k0 / eos->rho0;
  p.c = std::sqrt(p.c2);
  p.kappa = eos->g * eos->rho0 / eos->k0;
  for (int s = 0; s < 4; ++s) p.side[s] = side[s];
  p.cfl = 0.0;
  return p;
}

template <typename T, bool DEV>
void host_height_step(const StepParams& p, const int32_t* side, const uint8_t* solid,
                      const double* q, const int32_t* K, double dt, const double* lam,
                      const int32_t* hid, const std::vector<int64_t>& hcell, int nheights,
                      double* out) {
  HostStep<T, DEV> H(p, side, solid, q, K, dt, lam);
  for (int k = 0; k < nheights; ++k) out[k] = 0.0;
  for (int64_t c : hcell) out[hid[c]] += height_body<T, DEV>(H.A, hid, c);
}

}  // namespace
}  // namespace fv

// One reverse step on the host through the same per-cell and per-face bodies
// as the kernels; see fv_model_host.h.
extern "C" int fv_host_adjoint_step(const fv_grid* grid, const fv_eos* eos, const int32_t side[4],
                                    const uint8_t* solid, const double* q, const int32_t* K,
                                    double dt, const double* lam, double* lam_out, int prec) {
  using namespace fv;
  if (!grid || !eos || !side || !solid || !q || !K || !lam || !lam_out) return 1;
  if (grid->nx < 1 || grid->ny < 1 || eos->gamma != 1.0) return 1;
  if (prec != FV_FP64 && prec != FV_FP32_DEV) return 1;
  const StepParams p = host_params(grid, eos, side);
  if (prec == FV_FP64) host_reverse_step<double, false>(p, side, solid, q, K, dt, lam, lam_out);
  else host_reverse_step<float, true>(p, side, solid, q, K, dt, lam, lam_out);
  return 0;
}

extern "C" int fv_host_height_step(const fv_grid* grid, const fv_eos* eos, const int32_t side[4],
                                   const uint8_t* solid, const double* q, const int32_t* K,
                                   double dt, const double* lam, const int32_t* height_id,
                                   int nheights, double* out, int prec) {
  using namespace fv;
  if (!grid || !eos || !side || !solid || !q || !K || !lam || !height_id || !out) return 1;
  if (grid->nx < 1 || grid->ny < 1 || eos->gamma != 1.0 || nheights < 1) return 1;
  if (prec != FV_FP64 && prec != FV_FP32_DEV) return 1;
  std::vector<int64_t> hcell;
  if (!height_cells(grid->nx, grid->ny, solid, nheights, height_id, out, hcell)) return 1;
  const StepParams p = host_params(grid, eos, side);
  if (prec == FV_FP64)
    host_height_step<double, false>(p, side, solid, q, K, dt, lam, height_id, hcell, nheights, out);
  else
    host_height_step<float, true>(p, side, solid, q, K, dt, lam, height_id, hcell, nheights, out);
  return 0;
}

extern "C" fv_status fv_adjoint(fv_handle* h, const fv_adjoint_spec* spec, double* dL_dq0,
                                int on_device, fv_adjoint_info* info) {
  using namespace fv;
  if (!h || !spec || !dL_dq0) {
    set_last_error("fv_adjoint: null argument");
    return FV_EINVAL;
  }
  if (h->own_hi > 0) {
    set_last_error("fv_adjoint: the handle is one strip of a partitioned domain");
    return FV_EINVAL;
  }
  if (!h->has_state) {
    set_last_error("fv_adjoint: no state (call fv_set_state first)");
    return FV_EINVAL;
  }
  if (h->order != 2 || h->xface != FV_XFACE_GL) {
    set_last_error("fv_adjoint: the adjoint is of the second-order scheme with Gauss-Legendre x "
                   "faces (fv_set_order(h, 2), fv_set_xface(h, FV_XFACE_GL))");
    return FV_EINVAL;
  }
  if (spec->nsteps < 1 || !(spec->cfl > 0.0) || !(spec->cfl <= 1.0) || spec->ngauges < 1 ||
      !spec->gauges || !spec->target || spec->checkpoint_every < 0) {
    set_last_error("fv_adjoint: need nsteps >= 1, 0 < cfl <= 1, ngauges >= 1, gauges, target, "
                   "checkpoint_every >= 0");
    return FV_EINVAL;
  }
  std::vector<uint8_t> solid(h->ncell);
  cudaError_t e = cudaMemcpyAsync(solid.data(), h->d_solid, h->ncell, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    set_last_error((std::string("fv_adjoint: ") + cudaGetErrorString(e)).c_str());
    return FV_ECUDA;
  }
  for (int g = 0; g < spec->ngauges; ++g) {
    const int64_t c = spec->gauges[g];
    if (c < 0 || c >= (int64_t)h->ncell || solid[c]) {
      set_last_error("fv_adjoint: every gauge must be a fluid cell index j*nx + i");
      return FV_EINVAL;
    }
  }
  for (size_t k = 0; k < (size_t)spec->nsteps * spec->ngauges; ++k)
    if (!std::isfinite(spec->target[k])) {
      set_last_error("fv_adjoint: target values must be finite");
      return FV_EINVAL;
    }
  std::vector<int64_t> hcell;
  if (!height_cells(h->grid.nx, h->grid.ny, solid.data(), spec->nheights, spec->height_id,
                    spec->dL_dh, hcell)) {
    set_last_error("fv_adjoint: nheights >= 0; height_id and dL_dh given iff nheights > 0; "
                   "height_id entries in [-1, nheights), >= 0 only on a fluid cell whose lower "
                   "neighbour is solid");
    return FV_EINVAL;
  }
  if (h->prec == FV_FP64) return run_adjoint<double, false>(h, spec, dL_dq0, on_device, info, hcell);
  return run_adjoint<float, true>(h, spec, dL_dq0, on_device, info, hcell);
}

// ------------------------------------------------------------------ frozen map
// The map whose derivative fv_adjoint returns (reading R-adj): steps of Eq.
// (Scheme) with each step's dt and levels given instead of its own.
namespace {

template <typename T, bool DEV>
fv_status run_frozen(fv_handle* h, int32_t n, const double* dt, const int32_t* K, int32_t ng,
                     const int64_t* gauges, double* m_series) {
  using namespace fv;
  const int nx = h->grid.nx, ny = h->grid.ny;
  cudaStream_t st = h->stream;
  DevBuf dK, dg, dm;
  if (!dK.alloc(sizeof(int32_t) * (size_t)n * nx) ||
      (ng > 0 && (!dg.alloc(sizeof(int64_t) * ng) || !dm.alloc(sizeof(double) * (size_t)n * ng)))) {
    set_last_error("fv_step_frozen: device allocation failed");
    return FV_ENOMEM;
  }
  auto fail = [](cudaError_t e) {
    set_last_error((std::string("fv_step_frozen: ") + cudaGetErrorString(e)).c_str());
    return FV_ECUDA;
  };
  cudaError_t e = cudaMemcpyAsync(dK.p, K, sizeof(int32_t) * (size_t)n * nx,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && ng > 0)
    e = cudaMemcpyAsync(dg.p, gauges, sizeof(int64_t) * ng, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(e);
  const StepParams p = params_of(h, h->cfl);
  const Tables tb{h->d_rhoE, h->d_rhoE_f};
  for (int32_t k = 0; k < n && e == cudaSuccess; ++k) {
    // this step's levels and dt; the state stays stored relative to Kref
    e = cudaMemcpyAsync(h->d_Kcur, dK.as<int32_t>() + (size_t)k * nx, sizeof(int32_t) * nx,
                        cudaMemcpyDeviceToDevice, st);
    adj_set_dt_kernel<<<1, 1, 0, st>>>(h->d_sc, dt[k]);
    const int a = h->cur, b = 1 - h->cur;
    launch_replay_step<T, DEV>(p, (const T*)h->d_q[a], (T*)h->d_q[b], h->d_solid, h->d_Kref,
                               h->d_Kcur, h->d_colsum, h->d_sc, tb, h->tiling, h->strip_h, st);
    // Kref <- the levels just used (the new state's reference), Kcur, rate and
    // status from the step's epilogue; time and step count are not advanced
    launch_finalize(p, h->d_Kref, h->d_Kcur, h->d_colsum, h->d_sc, 0, st);
    h->cur = b;
    if (ng > 0)
      adj_after_step_kernel<T, DEV><<<1, 256, 0, st>>>(
          nx, ny, (const T*)h->d_q[b], h->d_Kref, h->d_rhoE, dg.as<int64_t>(), ng,
          dm.as<double>() + (size_t)k * ng, h->d_Kcur, nullptr, h->d_sc, nullptr);
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess && ng > 0)
    e = cudaMemcpyAsync(m_series, dm.p, sizeof(double) * (size_t)n * ng, cudaMemcpyDeviceToHost, st);
  DevScalars sc;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&sc, h->d_sc, sizeof(sc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(e);
  if (sc.status) {
    set_last_error("fv_step_frozen: a step produced a non-admissible state");
    return FV_ENONFINITE;
  }
  return FV_OK;
}

}  // namespace

extern "C" fv_status fv_step_frozen(fv_handle* h, int32_t n, const double* dt, const int32_t* K,
                                    int32_t ngauges, const int64_t* gauges, double* m_series) {
  using namespace fv;
  if (!h || n < 0 || (n > 0 && (!dt || !K)) || ngauges < 0 ||
      (ngauges > 0 && (!gauges || !m_series))) {
    set_last_error("fv_step_frozen: null argument or negative count");
    return FV_EINVAL;
  }
  if (!h->has_state) {
    set_last_error("fv_step_frozen: no state (call fv_set_state first)");
    return FV_EINVAL;
  }
  if (h->own_hi > 0 || h->order != 2 || h->xface != FV_XFACE_GL) {
    set_last_error("fv_step_frozen: second order with Gauss-Legendre x faces, undivided grids only");
    return FV_EINVAL;
  }
  for (size_t k = 0; k < (size_t)n * h->grid.nx; ++k)
    if (K[k] < 0 || K[k] > h->grid.ny) {
      set_last_error("fv_step_frozen: levels must lie in [0, ny]");
      return FV_EINVAL;
    }
  for (int32_t k = 0; k < n; ++k)
    if (!(dt[k] >= 0.0) || !std::isfinite(dt[k])) {
      set_last_error("fv_step_frozen: dt values must be finite and >= 0");
      return FV_EINVAL;
    }
  for (int g = 0; g < ngauges; ++g)
    if (gauges[g] < 0 || gauges[g] >= (int64_t)h->ncell) {
      set_last_error("fv_step_frozen: gauges must be cell indices j*nx + i");
      return FV_EINVAL;
    }
  if (n == 0) return FV_OK;
  if (h->prec == FV_FP64) return run_frozen<double, false>(h, n, dt, K, ngauges, gauges, m_series);
  return run_frozen<float, true>(h, n, dt, K, ngauges, gauges, m_series);
}
