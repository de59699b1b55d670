// One time step of Eq. (Scheme) (Gaburro, Castro, Dumbser) as a single fused
// kernel per step plus a one-block finalize kernel:
//
//   step_kernel   one CTA per TX x TY tile of cells.
//     load      Q^n of the tile plus a 2-cell halo into shared memory (SoA,
//               coalesced rows), with the solid/outside flags and the column
//               levels K_i;
//     recon     for the tile plus a 1-cell ring: fluctuations w.r.t. the
//               cell's water-at-rest state Q^E_ij (alpha^E = alpha_ij,
//               rho^E from the column level), central slopes, one
//               Barth-Jespersen factor per cell, order switch, half-step
//               predictor dQ/dt = -(A1 dQ/dx + A2 dQ/dy) in deviation form,
//               the four face-midpoint states at t^{n+1/2} (Section 3.4);
//     faces     every x face (Osher, Gauss-Legendre) and y face (well-balanced
//               Osher-Romberg) of the tile solved once into shared memory;
//               walls and solid neighbours see the mirror state;
//     update    Q^{n+1} = Q^n - dt/dx (D+_W + D-_E + I_x) - dt/dy (D+_S + D-_N + I_y)
//               with the interior integral of Eq. (b^y_3_final_integral) plus
//               the conservative part f(q_E) - f(q_W), g(q_N) - g(q_S);
//     epilogue  max signal rate for the next dt (one atomicMax per CTA) and
//               the free-surface detector's column sums of Eq.
//               (Free_surf_detector) in exact 2^-32 fixed point (one atomicAdd
//               per column per CTA), non-admissible-state flag.
//   finalize      K_i = round(column sum), dt bookkeeping, accumulator reset.
//
// The FP64 instantiation stores the full state; the FP32 instantiation stores
// the deviation m^f = m - alpha rho^E(y; K_i) so that a state at rest is
// represented by exact zeros.
#include <cuda_runtime.h>

#include <cmath>

#include "fv_consts.cuh"
#include "fv_kernels.cuh"
#include "fv_model.cuh"

namespace fv {

namespace {

constexpr int TX = 32, TY = 8;
constexpr int NT = TX * TY;
constexpr int WX = TX + 4, WY = TY + 4;  // window: tile + 2-cell halo
constexpr int RX = TX + 2, RY = TY + 2;  // reconstructed cells: tile + 1 ring
constexpr unsigned char F_FLUID = 0, F_SOLID = 1, F_OUT = 2;
constexpr unsigned long long ONE_FIXED = 1ull << 32;


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

template <typename T>
struct Smem {
  union {
    V4<T> w[WY][WX];  // load phase: (m, mu, mv, a); m: FP64 full, FP32 m^f of own level
    struct {
      V4<T> Dx[2][TY][TX + 1];  // face phase: D-, D+ of x faces
      V4<T> Dy[2][TY + 1][TX];  // y faces
    } d;
  } u;
  V4<T> rs[RY][RX];     // reconstructed cells: (aE, mEc, mES, mEN)
  V4<T> rf[4][RY][RX];  // their face fluctuation states W, E, S, N at t^{n+1/2}
  V4<T> base[TY][TX];   // centre fluctuation at t^{n+1/2}
  T ga[2][TY][TX];      // limited alpha slopes dax, day
  unsigned long long col[TY][TX];
  double wmax[NT / 32];
  int K[WX];
  unsigned char flag[WY][WX];
};

enum { F_W = 0, F_E = 1, F_S = 2, F_N = 3 };

// One tile (bx, by) of one domain; called by the whole CTA.
// XOR: x faces by the conservative Osher-Romberg viscosity of Eq. (OR_cons)
// instead of the Gauss-Legendre quadrature of Eq. (OsherMatrixFormal_approx).
template <typename T, bool DEV, bool XOR>
__device__ __forceinline__ void step_tile(const StepParams& p, const KConsts<T>& kc,
                                          const T* __restrict__ qin, T* __restrict__ qout,
                                          const uint8_t* __restrict__ solid,
                                          const int32_t* __restrict__ Kref,
                                          const int32_t* __restrict__ Kcur,
                                          unsigned long long* __restrict__ colsum,
                                          DevScalars* __restrict__ sc,
                                          const double* __restrict__ rhoE_d,
                                          const T* __restrict__ rt, int bx, int by, Smem<T>& S) {
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i0 = bx * TX, j0 = by * TY;
  const int nx = p.nx, ny = p.ny;
  const size_t N = (size_t)nx * ny;

  const Phys<T>& P = kc.P;
  // boundary kinds as scalars (a runtime index into the parameter struct would
  // place it in local memory)
  const bool trW = p.side[0] == 1, trE = p.side[1] == 1, trS = p.side[2] == 1, trN = p.side[3] == 1;
  const T dx = kc.dx, dy = kc.dy, eps = kc.eps;
  const T inv_dx = kc.inv_dx, inv_dy = kc.inv_dy, inv_1meps = kc.inv_1meps;
  // dt of this step, computed once per step by the finalize/prepare kernels
  const T dt = sizeof(T) == 8 ? (T)sc->dt_cur : (T)sc->dt_cur_f;

  // ---------------------------------------------------------------- load
  // Each warp loads whole window rows: its 32 lanes the 128-byte-aligned
  // centre (coalesced), lanes 0-3 the two halo columns on either side.
  const int lane = tid & 31, warp = tid >> 5;
  for (int wj = warp; wj < WY; wj += NT / 32) {
    const int gj = j0 - 2 + wj;
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 1 && lane >= 4) break;
      const int wi = pass == 0 ? lane + 2 : (lane < 2 ? lane : TX + lane);
      const int gi = i0 - 2 + wi;
      unsigned char f = F_OUT;
      if (gi >= 0 && gj >= 0 && gi < nx && gj < ny) f = solid[(size_t)gj * nx + gi] ? F_SOLID : F_FLUID;
      S.flag[wj][wi] = f;
      if (f == F_FLUID) {
        const size_t c = (size_t)gj * nx + gi;
        T m = qin[c];
        const T a = qin[3 * N + c];
        if (DEV) {
          // re-base m^f from the level it was stored with to this step's level
          const int Kr = Kref[gi], Kc = Kcur[gi];
          if (Kr != Kc) m += a * (tab(rt, 2 * (gj - Kr) + 1, ny) - tab(rt, 2 * (gj - Kc) + 1, ny));
        }
        S.u.w[wj][wi] = V4<T>{m, qin[N + c], qin[2 * N + c], a};
      }
    }
  }
  for (int idx = tid; idx < WX; idx += NT) {
    const int gi = i0 - 2 + idx;
    S.K[idx] = (gi >= 0 && gi < nx) ? Kcur[gi] : 0;
  }
  __syncthreads();
  // rho^E at h half cells above the level (Eq. (BNs_eq3)); levels are at most
  // ny (level_of), so h stays inside the table
  auto rE = [&](int h) -> T { return tab(rt, h, ny); };

  // Own-cell state for the update, kept in registers.
  const int gi_me = i0 + tx, gj_me = j0 + ty;
  const bool inside = gi_me < nx && gj_me < ny;
  const unsigned char flag_me = S.flag[ty + 2][tx + 2];
  T qold[4] = {0, 0, 0, 0};
  if (flag_me == F_FLUID) unpack(S.u.w[ty + 2][tx + 2], qold);

  // ---------------------------------------------------------------- recon
  ReconConsts<T> RC = kc.R;
  RC.half_dt = T(0.5) * dt;
  for (int idx = tid; idx < RX * RY; idx += NT) {
    const int rx = idx % RX, ry = idx / RX;
    const int wi = rx + 1, wj = ry + 1;
    if (S.flag[wj][wi] != F_FLUID) continue;
    const int gj = j0 - 1 + ry;
    const int K = S.K[wi];
    const V4<T> wc = S.u.w[wj][wi];
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

    // fluctuation of a neighbour w.r.t. this cell's Q^E; ghost if not fluid
    auto nbf = [&](int dwi, int dwj, T out[4]) -> bool {
      const int ni = wi + dwi, nj = wj + dwj;
      if (S.flag[nj][ni] != F_FLUID) return false;
      const V4<T> wn = S.u.w[nj][ni];
      const T an = wn.w;
      const int gjn = gj + dwj;
      const T rn = rE(2 * (gjn - K) + 1);
      if (DEV) {
        const int Kn = S.K[ni];
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
    auto ghost = [&](int dwi, int dwj, int normal, int side, T out[4]) {
      const unsigned char f = S.flag[wj + dwj][wi + dwi];
#pragma unroll
      for (int v = 0; v < 4; ++v) out[v] = Qf[v];
      const bool tr = side == 0 ? trW : side == 1 ? trE : side == 2 ? trS : trN;
      if (!(f == F_OUT && tr)) {
        if (normal == 1) out[1] = -out[1];
        else out[2] = -out[2];
      }
    };
    T fW[4], fE[4], fS[4], fN[4];
    if (!nbf(-1, 0, fW)) ghost(-1, 0, 1, 0, fW);
    if (!nbf(1, 0, fE)) ghost(1, 0, 1, 1, fE);
    if (!nbf(0, -1, fS)) ghost(0, -1, 2, 2, fS);
    if (!nbf(0, 1, fN)) ghost(0, 1, 2, 3, fN);
    T mx[4], mn[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      mx[v] = fmax(fmax(fmax(Qf[v], fW[v]), fmax(fE[v], fS[v])), fN[v]);
      mn[v] = fmin(fmin(fmin(Qf[v], fW[v]), fmin(fE[v], fS[v])), fN[v]);
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      T fd[4];
      if (nbf((d & 1) ? 1 : -1, (d & 2) ? 1 : -1, fd)) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          mx[v] = fmax(mx[v], fd[v]);
          mn[v] = fmin(mn[v], fd[v]);
        }
      }
    }
    const T mES = aE * rES, mEN = aE * rEN;
    T base[4], ga[2];
    recon_core(Qf, fW, fE, fS, fN, mx, mn, aE, mEc, mES, mEN, rEc, P, RC, base, ga);
    S.rs[ry][rx] = V4<T>{aE, mEc, mES, mEN};
    S.rf[F_W][ry][rx] = pack(fW);
    S.rf[F_E][ry][rx] = pack(fE);
    S.rf[F_S][ry][rx] = pack(fS);
    S.rf[F_N][ry][rx] = pack(fN);
    if (rx >= 1 && rx <= TX && ry >= 1 && ry <= TY) {
      S.base[ry - 1][rx - 1] = pack(base);
      S.ga[0][ry - 1][rx - 1] = ga[0];
      S.ga[1][ry - 1][rx - 1] = ga[1];
    }
  }
  __syncthreads();  // window no longer needed: its storage becomes Dx/Dy

  // ---------------------------------------------------------------- faces
  for (int idx = tid; idx < (TX + 1) * TY + TX * (TY + 1); idx += NT) {
    T Dm[4] = {0, 0, 0, 0}, Dp[4] = {0, 0, 0, 0};
    if (idx < (TX + 1) * TY) {
      const int fx = idx % (TX + 1), fy = idx / (TX + 1);
      const int rxL = fx, rxR = fx + 1, ry = fy + 1;
      const bool L = S.flag[ry + 1][rxL + 1] == F_FLUID;
      const bool R = S.flag[ry + 1][rxR + 1] == F_FLUID;
      if (L || R) {
        T qm[4], qp[4], dq[4];
        if (L && R) {
          const V4<T> sL = S.rs[ry][rxL], sR = S.rs[ry][rxR];
          const T mEL = sL.y, mER = sR.y;
          const T aL = sL.x, aR = sR.x;
          T fl[4], fr[4];
          unpack(S.rf[F_E][ry][rxL], fl);
          unpack(S.rf[F_W][ry][rxR], fr);
          qm[0] = mEL + fl[0]; qm[1] = fl[1]; qm[2] = fl[2]; qm[3] = aL + fl[3];
          qp[0] = mER + fr[0]; qp[1] = fr[1]; qp[2] = fr[2]; qp[3] = aR + fr[3];
          dq[0] = (mER - mEL) + (fr[0] - fl[0]);
          dq[1] = fr[1] - fl[1];
          dq[2] = fr[2] - fl[2];
          dq[3] = (aR - aL) + (fr[3] - fl[3]);
        } else {
          const int rx = L ? rxL : rxR;
          const V4<T> sc_ = S.rs[ry][rx];
          const V4<T> fc = S.rf[L ? F_E : F_W][ry][rx];
          const T mE = sc_.y, aE = sc_.x;
          T q[4];
          q[0] = mE + fc.x;
          q[1] = fc.y;
          q[2] = fc.z;
          q[3] = aE + fc.w;
          const bool outside = L ? (S.flag[ry + 1][rxR + 1] == F_OUT) : (S.flag[ry + 1][rxL + 1] == F_OUT);
          const bool transmissive = outside && (L ? trE : trW);
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
      S.u.d.Dx[0][fy][fx] = pack(Dm);
      S.u.d.Dx[1][fy][fx] = pack(Dp);
    } else {
      const int k = idx - (TX + 1) * TY;
      const int fx = k % TX, fy = k / TX;
      const int rx = fx + 1, ryB = fy, ryT = fy + 1;
      const bool B = S.flag[ryB + 1][rx + 1] == F_FLUID;
      const bool Tt = S.flag[ryT + 1][rx + 1] == F_FLUID;
      if (B || Tt) {
        T qm[4], qp[4], dq[4];
        T dap = T(0);
        if (B && Tt) {
          const V4<T> sB = S.rs[ryB][rx], sT = S.rs[ryT][rx];
          const T mEB = sB.w, mET = sT.z;
          const T aB = sB.x, aT = sT.x;
          T fb[4], ft[4];
          unpack(S.rf[F_N][ryB][rx], fb);
          unpack(S.rf[F_S][ryT][rx], ft);
          qm[0] = mEB + fb[0]; qm[1] = fb[1]; qm[2] = fb[2]; qm[3] = aB + fb[3];
          qp[0] = mET + ft[0]; qp[1] = ft[1]; qp[2] = ft[2]; qp[3] = aT + ft[3];
          dq[0] = (mET - mEB) + (ft[0] - fb[0]);
          dq[1] = ft[1] - fb[1];
          dq[2] = ft[2] - fb[2];
          dq[3] = (aT - aB) + (ft[3] - fb[3]);
          // jump of alpha p: equilibrium part (rho^E_f - rho0) Delta alpha^E is
          // exactly zero at the level face; fluctuation part c2 (dm^f - rho0 da^f)
          const int K = S.K[rx + 1];
          const T rEf = rE(2 * (j0 - 1 + ryT - K));
          dap = P.c2 * ((rEf - P.rho0) * (aT - aB) + ((ft[0] - fb[0]) - P.rho0 * (ft[3] - fb[3])));
        } else {
          const int ry = B ? ryB : ryT;
          const V4<T> sc_ = S.rs[ry][rx];
          const V4<T> fc = S.rf[B ? F_N : F_S][ry][rx];
          const T mE = B ? sc_.w : sc_.z, aE = sc_.x;
          T q[4];
          q[0] = mE + fc.x;
          q[1] = fc.y;
          q[2] = fc.z;
          q[3] = aE + fc.w;
          const bool outside = B ? (S.flag[ryT + 1][rx + 1] == F_OUT) : (S.flag[ryB + 1][rx + 1] == F_OUT);
          const bool transmissive = outside && (B ? trN : trS);
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
      S.u.d.Dy[0][fy][fx] = pack(Dm);
      S.u.d.Dy[1][fy][fx] = pack(Dp);
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- update
  T my_rate = T(0);
  unsigned long long my_w = 0;
  bool bad = false;
  if (inside && flag_me == F_FLUID) {
    const int rx = tx + 1, ry = ty + 1;
    const int K = S.K[tx + 2];
    const V4<T> sme = S.rs[ry][rx];
    const T mEc = sme.y, mES = sme.z, mEN = sme.w;
    T fW[4], fE[4], fS[4], fN[4], base[4];
    unpack(S.rf[F_W][ry][rx], fW);
    unpack(S.rf[F_E][ry][rx], fE);
    unpack(S.rf[F_S][ry][rx], fS);
    unpack(S.rf[F_N][ry][rx], fN);
    unpack(S.base[ty][tx], base);
    const T dax = S.ga[0][ty][tx], day = S.ga[1][ty][tx];
    T Ix[4], Iy[4];
    interior_terms(fW, fE, fS, fN, base, mEc, mES, mEN, dax, day, dx, dy, P, Ix, Iy);
    const T rdx = dt / dx, rdy = dt / dy;
    T xs[4], ys[4], DpW[4], DmE[4], DpS[4], DmN[4];
    unpack(S.u.d.Dx[1][ty][tx], DpW);
    unpack(S.u.d.Dx[0][ty][tx + 1], DmE);
    unpack(S.u.d.Dy[1][ty][tx], DpS);
    unpack(S.u.d.Dy[0][ty + 1][tx], DmN);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      xs[c] = DpW[c] + DmE[c] + Ix[c];
      ys[c] = DpS[c] + DmN[c] + Iy[c];
    }
    T qn[4];
    T m_full;
    if (DEV) {
      // deviation form: m^f_new = m^f + dm - rho^E_c da (own level, own new alpha)
      T dQ[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) dQ[c] = -rdx * xs[c] - rdy * ys[c];
      const T rEc = rE(2 * (gj_me - K) + 1);
      qn[0] = qold[0] + (dQ[0] - rEc * dQ[3]);
      qn[1] = qold[1] + dQ[1];
      qn[2] = qold[2] + dQ[2];
      qn[3] = qold[3] + dQ[3];
      m_full = qn[3] * rEc + qn[0];
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) qn[c] = qold[c] - rdx * xs[c] - rdy * ys[c];
      m_full = qn[0];
    }
    const size_t c = (size_t)gj_me * nx + gi_me;
#pragma unroll
    for (int v = 0; v < 4; ++v) qout[v * N + c] = qn[v];
    // epilogue: admissibility, signal rate, detector weight
    cell_epilogue<T, DEV>(p, kc, qn, m_full, my_rate, my_w, bad);
  } else if (inside) {
    const size_t c = (size_t)gj_me * nx + gi_me;
#pragma unroll
    for (int v = 0; v < 4; ++v) qout[v * N + c] = T(0);
    if (flag_me == F_SOLID) my_w = ONE_FIXED;
  }
  block_epilogue<T, TX, TY>(my_rate, my_w, bad, inside, gi_me, S.col, S.wmax, colsum, sc);
}

template <typename T, bool DEV, bool XOR>
__global__ void __launch_bounds__(NT, (sizeof(T) == 8 ? 2 : 4))
    step_kernel(StepParams p, KConsts<T> kc, const T* __restrict__ qin, T* __restrict__ qout,
                const uint8_t* __restrict__ solid, const int32_t* __restrict__ Kref,
                const int32_t* __restrict__ Kcur, unsigned long long* __restrict__ colsum,
                DevScalars* __restrict__ sc, const double* __restrict__ rhoE_d,
                const T* __restrict__ rt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T>& S = *reinterpret_cast<Smem<T>*>(smem_raw);
  step_tile<T, DEV, XOR>(p, kc, qin, qout, solid, Kref, Kcur, colsum, sc, rhoE_d, rt, blockIdx.x,
                         blockIdx.y, S);
}

// Batched step: every tile of every domain of an ensemble, distributed
// round-robin over a persistent grid (one or a few CTAs per SM); each domain
// uses its own dt, levels and accumulators.  parity selects which of the two
// state buffers is read.
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

template <typename T, bool DEV>
__global__ void __launch_bounds__(NT, (sizeof(T) == 8 ? 2 : 4))
    batch_step_kernel(const BatchDomain<T>* __restrict__ doms, const int4* __restrict__ tiles,
                      int ntiles, int parity) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T>& S = *reinterpret_cast<Smem<T>*>(smem_raw);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int4 td = tiles[t];
    const BatchDomain<T>& d = doms[td.x];
    step_tile<T, DEV, false>(d.p, d.kc, d.q[parity], d.q[1 - parity], d.solid, d.Kref, d.Kcur, d.colsum,
                      d.sc, d.rhoE_d, d.rt, td.y, td.z, S);
    __syncthreads();  // shared memory is reused by the next tile
  }
}

// Per-domain finalize for a batch: one CTA per domain.
template <typename T>
__global__ void batch_finalize_kernel(const BatchDomain<T>* __restrict__ doms, double cfl,
                                      int count_step) {
  const BatchDomain<T>& d = doms[blockIdx.x];
  for (int i = threadIdx.x; i < d.p.nx; i += blockDim.x) {
    d.Kref[i] = d.Kcur[i];
    d.Kcur[i] = level_of(d.colsum[i], d.p.ny);
    d.colsum[i] = 0ull;
  }
  if (threadIdx.x == 0) {
    DevScalars* sc = d.sc;
    if (count_step) {
      sc->t += sc->dt_cur;
      sc->dt_last = sc->dt_cur;
      sc->steps += 1;
    }
    sc->rate_cur = __longlong_as_double((long long)sc->rate_acc);
    sc->rate_acc = 0ull;
    sc->dt_cur = sc->rate_cur > 0.0 ? cfl / sc->rate_cur : 0.0;
    sc->dt_cur_f = (float)sc->dt_cur;
  }
}

template <typename T>
__global__ void batch_prepare_kernel(const BatchDomain<T>* __restrict__ doms, int ndom, double cfl) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ndom; k += gridDim.x * blockDim.x) {
    DevScalars* sc = doms[k].sc;
    sc->dt_cur = sc->rate_cur > 0.0 ? cfl / sc->rate_cur : 0.0;
    sc->dt_cur_f = (float)sc->dt_cur;
  }
}

// ----------------------------------------------------------------------------
__global__ void finalize_kernel(StepParams p, int32_t* Kref, int32_t* Kcur,
                                unsigned long long* colsum, DevScalars* sc, int count_step) {
  for (int i = threadIdx.x; i < p.nx; i += blockDim.x) {
    Kref[i] = Kcur[i];
    Kcur[i] = level_of(colsum[i], p.ny);
    colsum[i] = 0ull;
  }
  if (threadIdx.x == 0) {
    if (count_step) {
      const double dt = sc->rate_cur > 0.0 ? p.cfl / sc->rate_cur : 0.0;
      sc->t += dt;
      sc->dt_last = dt;
      sc->steps += 1;
    }
    sc->rate_cur = __longlong_as_double((long long)sc->rate_acc);
    sc->rate_acc = 0ull;
    sc->dt_cur = sc->rate_cur > 0.0 ? p.cfl / sc->rate_cur : 0.0;
    sc->dt_cur_f = (float)sc->dt_cur;
  }
}

// dt of the next step from the current rate and the cfl of this call.
__global__ void prepare_kernel(double cfl, DevScalars* sc) {
  sc->dt_cur = sc->rate_cur > 0.0 ? cfl / sc->rate_cur : 0.0;
  sc->dt_cur_f = (float)sc->dt_cur;
}

__global__ void prologue_kernel(StepParams p, const double* __restrict__ q,
                                const uint8_t* __restrict__ solid, unsigned long long* colsum,
                                DevScalars* sc) {
  const size_t N = (size_t)p.nx * p.ny;
  double my_rate = 0.0;
  bool bad = false;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N;
       c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % p.nx);
    if (solid[c]) {
      atomicAdd(&colsum[i], ONE_FIXED);
      continue;
    }
    const double m = q[c], mu = q[N + c], mv = q[2 * N + c], a = q[3 * N + c];
    const double u = mu / m, v = mv / m;
    if (!(m > 0.0) || !(a > 0.0) || !isfinite(u) || !isfinite(v) || !isfinite(a)) bad = true;
    double r = (fabs(u) + p.c) / p.dx + (fabs(v) + p.c) / p.dy;
    if (r >= 0.0) my_rate = fmax(my_rate, r);
    double w = (a - p.eps) / (1.0 - p.eps);
    w = w >= 0.0 ? (w > 1.0 ? 1.0 : w) : 0.0;  // NaN -> 0 (the status flag reports the state)
    const unsigned long long qw = (unsigned long long)__double2ll_rn(w * 4294967296.0);
    if (qw) atomicAdd(&colsum[i], qw);
  }
  if (bad) atomicOr(&sc->status, 1);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) my_rate = fmax(my_rate, __shfl_xor_sync(0xffffffffu, my_rate, o));
  if ((threadIdx.x & 31) == 0 && my_rate > 0.0)
    atomicMax(&sc->rate_acc, (unsigned long long)__double_as_longlong(my_rate));
}

__global__ void to_dev_kernel(StepParams p, const double* __restrict__ q,
                              const uint8_t* __restrict__ solid, const int32_t* __restrict__ K,
                              const double* __restrict__ rhoE, float* __restrict__ out) {
  const size_t N = (size_t)p.nx * p.ny;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N;
       c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % p.nx), j = (int)(c / p.nx);
    if (solid[c]) {
      for (int v = 0; v < 4; ++v) out[v * N + c] = 0.f;
      continue;
    }
    const double a = q[3 * N + c];
    out[c] = (float)(q[c] - a * rhoE[2 * (j - K[i]) + 1 + 2 * p.ny]);
    out[N + c] = (float)q[N + c];
    out[2 * N + c] = (float)q[2 * N + c];
    out[3 * N + c] = (float)a;
  }
}

__global__ void from_dev_kernel(StepParams p, const float* __restrict__ in,
                                const uint8_t* __restrict__ solid, const int32_t* __restrict__ K,
                                const double* __restrict__ rhoE, double* __restrict__ q) {
  const size_t N = (size_t)p.nx * p.ny;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N;
       c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % p.nx), j = (int)(c / p.nx);
    if (solid[c]) {
      for (int v = 0; v < 4; ++v) q[v * N + c] = 0.0;
      continue;
    }
    const double a = (double)in[3 * N + c];
    q[c] = a * rhoE[2 * (j - K[i]) + 1 + 2 * p.ny] + (double)in[c];
    q[N + c] = (double)in[N + c];
    q[2 * N + c] = (double)in[2 * N + c];
    q[3 * N + c] = a;
  }
}

__global__ void zero_solid_kernel(StepParams p, double* q, const uint8_t* solid) {
  const size_t N = (size_t)p.nx * p.ny;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N;
       c += (size_t)gridDim.x * blockDim.x)
    if (solid[c])
      for (int v = 0; v < 4; ++v) q[v * N + c] = 0.0;
}

// Deterministic mass: fixed chunk per block, fixed tree, then one block.
constexpr int MASS_T = 256;
__global__ void mass_partial_kernel(StepParams p, const double* __restrict__ q,
                                    const uint8_t* __restrict__ solid, double* partial) {
  __shared__ double s[MASS_T];
  const size_t N = (size_t)p.nx * p.ny;
  const size_t chunk = (N + gridDim.x - 1) / gridDim.x;
  const size_t b0 = blockIdx.x * chunk, b1 = b0 + chunk < N ? b0 + chunk : N;
  double acc = 0.0;
  for (size_t c = b0 + threadIdx.x; c < b1; c += MASS_T)
    if (!solid[c]) acc += q[c];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = MASS_T / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

__global__ void mass_final_kernel(const double* partial, int n, double scale, double* out) {
  __shared__ double s[MASS_T];
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += MASS_T) acc += partial[k];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = MASS_T / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0] * scale;
}

int grid_1d(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T, bool DEV, bool XOR>
void launch_step_xt(const StepParams& p, const T* in, T* out, const uint8_t* solid,
                    const int32_t* Kref, const int32_t* Kcur, unsigned long long* colsum,
                    DevScalars* sc, const double* rhoE_d, const T* rt, cudaStream_t st) {
  const size_t smem = sizeof(Smem<T>);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(step_kernel<T, DEV, XOR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr_set = true;
  }
  dim3 block(TX, TY);
  dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY);
  step_kernel<T, DEV, XOR><<<grid, block, smem, st>>>(p, make_consts<T>(p), in, out, solid, Kref,
                                                       Kcur, colsum, sc, rhoE_d, rt);
}

template <typename T, bool DEV>
void launch_step_t(const StepParams& p, const T* in, T* out, const uint8_t* solid,
                   const int32_t* Kref, const int32_t* Kcur, unsigned long long* colsum,
                   DevScalars* sc, const double* rhoE_d, const T* rt, bool osher_romberg_x,
                   cudaStream_t st) {
  if (osher_romberg_x)
    launch_step_xt<T, DEV, true>(p, in, out, solid, Kref, Kcur, colsum, sc, rhoE_d, rt, st);
  else
    launch_step_xt<T, DEV, false>(p, in, out, solid, Kref, Kcur, colsum, sc, rhoE_d, rt, st);
}

}  // namespace

// ---------------------------------------------------------------- batch helpers
size_t batch_table_bytes(int ndom, bool f64) {
  return (size_t)ndom * (f64 ? sizeof(BatchDomain<double>) : sizeof(BatchDomain<float>));
}

template <typename T>
static void fill_table_t(const BatchDomainDesc* d, int ndom, void* dst) {
  BatchDomain<T>* out = static_cast<BatchDomain<T>*>(dst);
  for (int k = 0; k < ndom; ++k) {
    BatchDomain<T> b;
    b.p = d[k].p;
    b.kc = make_consts<T>(d[k].p);
    b.q[0] = static_cast<T*>(d[k].q[0]);
    b.q[1] = static_cast<T*>(d[k].q[1]);
    b.solid = d[k].solid;
    b.Kref = d[k].Kref;
    b.Kcur = d[k].Kcur;
    b.colsum = d[k].colsum;
    b.sc = d[k].sc;
    b.rhoE_d = d[k].rhoE_d;
    b.rt = sizeof(T) == 8 ? (const T*)d[k].rhoE_d : (const T*)d[k].rhoE_f;
    out[k] = b;
  }
}

void batch_fill_table(const BatchDomainDesc* d, int ndom, bool f64, void* host_dst) {
  if (f64)
    fill_table_t<double>(d, ndom, host_dst);
  else
    fill_table_t<float>(d, ndom, host_dst);
}

template <typename T, bool DEV>
static int batch_grid_t() {
  static int grid = 0;
  if (!grid) {
    const size_t smem = sizeof(Smem<T>);
    cudaFuncSetAttribute(batch_step_kernel<T, DEV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int per_sm = 0, dev = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_step_kernel<T, DEV>, NT, smem);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  }
  return grid;
}

int batch_grid_size(bool f64) { return f64 ? batch_grid_t<double, false>() : batch_grid_t<float, true>(); }

void launch_batch_step(bool f64, const void* table, const int4* tiles, int ntiles, int parity,
                       cudaStream_t st) {
  dim3 block(TX, TY);
  if (f64) {
    const int grid = batch_grid_t<double, false>();
    batch_step_kernel<double, false><<<grid < ntiles ? grid : ntiles, block, sizeof(Smem<double>), st>>>(
        static_cast<const BatchDomain<double>*>(table), tiles, ntiles, parity);
  } else {
    const int grid = batch_grid_t<float, true>();
    batch_step_kernel<float, true><<<grid < ntiles ? grid : ntiles, block, sizeof(Smem<float>), st>>>(
        static_cast<const BatchDomain<float>*>(table), tiles, ntiles, parity);
  }
}

void launch_batch_finalize(bool f64, const void* table, int ndom, double cfl, int count_step,
                           cudaStream_t st) {
  if (f64)
    batch_finalize_kernel<double><<<ndom, 256, 0, st>>>(static_cast<const BatchDomain<double>*>(table),
                                                        cfl, count_step);
  else
    batch_finalize_kernel<float><<<ndom, 256, 0, st>>>(static_cast<const BatchDomain<float>*>(table),
                                                       cfl, count_step);
}

void launch_batch_prepare(bool f64, const void* table, int ndom, double cfl, cudaStream_t st) {
  const int grid = (ndom + 255) / 256;
  if (f64)
    batch_prepare_kernel<double><<<grid, 256, 0, st>>>(static_cast<const BatchDomain<double>*>(table), ndom, cfl);
  else
    batch_prepare_kernel<float><<<grid, 256, 0, st>>>(static_cast<const BatchDomain<float>*>(table), ndom, cfl);
}

void launch_step_f64(const StepParams& p, const StateF64& s, const uint8_t* solid,
                     const int32_t* Kcur, unsigned long long* colsum, DevScalars* sc,
                     const Tables& tb, cudaStream_t st, bool osher_romberg_x) {
  launch_step_t<double, false>(p, s.in, s.out, solid, Kcur, Kcur, colsum, sc, tb.rhoE_d,
                               tb.rhoE_d, osher_romberg_x, st);
}

void launch_step_f32(const StepParams& p, const StateF32& s, const uint8_t* solid,
                     const int32_t* Kref, const int32_t* Kcur, unsigned long long* colsum,
                     DevScalars* sc, const Tables& tb, cudaStream_t st, bool osher_romberg_x) {
  launch_step_t<float, true>(p, s.in, s.out, solid, Kref, Kcur, colsum, sc, tb.rhoE_d,
                             tb.rhoE_f, osher_romberg_x, st);
}

void launch_finalize(const StepParams& p, int32_t* Kref, int32_t* Kcur,
                     unsigned long long* colsum, DevScalars* sc, int count_step,
                     cudaStream_t st) {
  finalize_kernel<<<1, 1024, 0, st>>>(p, Kref, Kcur, colsum, sc, count_step);
}

void launch_prepare(double cfl, DevScalars* sc, cudaStream_t st) {
  prepare_kernel<<<1, 1, 0, st>>>(cfl, sc);
}

void launch_prologue_f64(const StepParams& p, const double* q, const uint8_t* solid,
                         unsigned long long* colsum, DevScalars* sc, cudaStream_t st) {
  prologue_kernel<<<grid_1d((size_t)p.nx * p.ny), 256, 0, st>>>(p, q, solid, colsum, sc);
}

void launch_to_dev(const StepParams& p, const double* q, const uint8_t* solid, const int32_t* K,
                   const Tables& tb, float* out, cudaStream_t st) {
  to_dev_kernel<<<grid_1d((size_t)p.nx * p.ny), 256, 0, st>>>(p, q, solid, K, tb.rhoE_d, out);
}

void launch_from_dev(const StepParams& p, const float* in, const uint8_t* solid,
                     const int32_t* K, const Tables& tb, double* q, cudaStream_t st) {
  from_dev_kernel<<<grid_1d((size_t)p.nx * p.ny), 256, 0, st>>>(p, in, solid, K, tb.rhoE_d, q);
}

void launch_zero_solid(const StepParams& p, double* q, const uint8_t* solid, cudaStream_t st) {
  zero_solid_kernel<<<grid_1d((size_t)p.nx * p.ny), 256, 0, st>>>(p, q, solid);
}

void launch_mass(const StepParams& p, const double* q, const uint8_t* solid, double* partial,
                 int nblocks, double* out, cudaStream_t st) {
  mass_partial_kernel<<<nblocks, MASS_T, 0, st>>>(p, q, solid, partial);
  mass_final_kernel<<<1, MASS_T, 0, st>>>(partial, nblocks, p.dx * p.dy, out);
}

}  // namespace fv
