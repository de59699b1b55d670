// One time step of the first-order scheme of Sections 3.2-3.3 (Eq.
// (SemidiscreteScheme_2) in y, its counterpart in x): the face states are
// the cell averages, x faces use the Osher solver of Section 3.2 between the
// two cells, interior y faces the well-balanced path between the two cell
// centres (yface_o1), wall and solid faces the mirror of the cell state at the
// cell's own height; there is no reconstruction and no interior term.
//
//   step_o1_kernel  one CTA per 32 x 8 tile: the tile plus a 1-cell halo in
//                   shared memory, every x and y face of the tile solved once,
//                   update, and the same epilogue as the second-order step
//                   (signal rate, detector column sums, status).
// The FP32 instantiation stores the deviation m^f = m - alpha rho^E(y; K_i)
// like the second-order FP32 path, so a state at rest is exact zeros.
#include <cuda_runtime.h>

#include "fv_consts.cuh"
#include "fv_kernels.cuh"
#include "fv_model.cuh"
#include "fv_order1.cuh"

namespace fv {
namespace {

constexpr int TX = 32, TY = 8;
constexpr int NT = TX * TY;
constexpr int WX = TX + 2, WY = TY + 2;  // window: tile + 1-cell halo
constexpr unsigned char F_FLUID = 0, F_SOLID = 1, F_OUT = 2;
constexpr unsigned long long ONE_FIXED = 1ull << 32;

template <typename T>
struct SmemO1 {
  T w[4][WY][WX];        // m (FP64: full; FP32: m^f of the cell's own level), mu, mv, alpha
  T Dx[8][TY][TX + 1];   // D-[4], D+[4] of x faces
  T Dy[8][TY + 1][TX];   // y faces
  unsigned long long col[TY][TX];
  double wmax[NT / 32];
  int K[WX];
  unsigned char flag[WY][WX];
};

template <typename T, bool DEV, bool XOR>
__global__ void __launch_bounds__(NT, (sizeof(T) == 8 ? 2 : 4))
    step_o1_kernel(StepParams p, KConsts<T> kc, const T* __restrict__ qin, T* __restrict__ qout,
                   const uint8_t* __restrict__ solid, const int32_t* __restrict__ Kref,
                   const int32_t* __restrict__ Kcur, unsigned long long* __restrict__ colsum,
                   DevScalars* __restrict__ sc, const T* __restrict__ rt,
                   const T* __restrict__ rq, const T* __restrict__ pq) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemO1<T>& S = *reinterpret_cast<SmemO1<T>*>(smem_raw);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int nx = p.nx, ny = p.ny;
  const size_t N = (size_t)nx * ny;
  const Phys<T>& P = kc.P;
  const bool trW = p.side[0] == 1, trE = p.side[1] == 1, trS = p.side[2] == 1, trN = p.side[3] == 1;
  const T dt = sizeof(T) == 8 ? (T)sc->dt_cur : (T)sc->dt_cur_f;

  // ---------------------------------------------------------------- load
  const int lane = tid & 31, warp = tid >> 5;
  for (int wj = warp; wj < WY; wj += NT / 32) {
    const int gj = j0 - 1 + wj;
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 1 && lane >= 2) break;
      const int wi = pass == 0 ? lane + 1 : (lane == 0 ? 0 : WX - 1);
      const int gi = i0 - 1 + wi;
      unsigned char f = F_OUT;
      if (gi >= 0 && gj >= 0 && gi < nx && gj < ny) f = solid[(size_t)gj * nx + gi] ? F_SOLID : F_FLUID;
      S.flag[wj][wi] = f;
      if (f == F_FLUID) {
        const size_t c = (size_t)gj * nx + gi;
        T m = qin[c];
        const T a = qin[3 * N + c];
        if (DEV) {
          const int Kr = Kref[gi], Kc = Kcur[gi];
          if (Kr != Kc) m += a * (tab(rt, 2 * (gj - Kr) + 1, ny) - tab(rt, 2 * (gj - Kc) + 1, ny));
        }
        S.w[0][wj][wi] = m;
        S.w[1][wj][wi] = qin[N + c];
        S.w[2][wj][wi] = qin[2 * N + c];
        S.w[3][wj][wi] = a;
      }
    }
  }
  for (int idx = tid; idx < WX; idx += NT) {
    const int gi = i0 - 1 + idx;
    S.K[idx] = (gi >= 0 && gi < nx) ? Kcur[gi] : 0;
  }
  __syncthreads();

  // full state and fluctuation of a window cell (alpha^E = alpha, column level)
  auto cell = [&](int wi, int wj, T q[4], T f[4], T& mE) {
    const int gj = j0 - 1 + wj;
    const T a = S.w[3][wj][wi];
    mE = mul_rn(a, tab(rt, 2 * (gj - S.K[wi]) + 1, ny));
    const T m = S.w[0][wj][wi];
    f[0] = DEV ? m : m - mE;
    f[1] = S.w[1][wj][wi];
    f[2] = S.w[2][wj][wi];
    f[3] = T(0);
    q[0] = DEV ? mE + m : m;
    q[1] = f[1];
    q[2] = f[2];
    q[3] = a;
  };

  // ---------------------------------------------------------------- faces
  for (int idx = tid; idx < (TX + 1) * TY + TX * (TY + 1); idx += NT) {
    T Dm[4] = {0, 0, 0, 0}, Dp[4] = {0, 0, 0, 0};
    if (idx < (TX + 1) * TY) {
      const int fx = idx % (TX + 1), fy = idx / (TX + 1);
      const int wj = fy + 1, wiL = fx, wiR = fx + 1;
      const bool L = S.flag[wj][wiL] == F_FLUID, R = S.flag[wj][wiR] == F_FLUID;
      if (L || R) {
        T qm[4], qp[4], dq[4];
        if (L && R) {
          T fl[4], fr[4], mEL, mER;
          cell(wiL, wj, qm, fl, mEL);
          cell(wiR, wj, qp, fr, mER);
          dq[0] = (mER - mEL) + (fr[0] - fl[0]);
          dq[1] = fr[1] - fl[1];
          dq[2] = fr[2] - fl[2];
          dq[3] = qp[3] - qm[3];
        } else {
          T q[4], f[4], mE;
          cell(L ? wiL : wiR, wj, q, f, mE);
          const bool outside = S.flag[wj][L ? wiR : wiL] == F_OUT;
          const bool tr = outside && (L ? trE : trW);
          const T g[4] = {q[0], tr ? q[1] : -q[1], q[2], q[3]};
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
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        S.Dx[c][fy][fx] = Dm[c];
        S.Dx[4 + c][fy][fx] = Dp[c];
      }
    } else {
      const int k = idx - (TX + 1) * TY;
      const int fx = k % TX, fy = k / TX;
      const int wi = fx + 1, wjB = fy, wjT = fy + 1;
      const bool B = S.flag[wjB][wi] == F_FLUID, Tt = S.flag[wjT][wi] == F_FLUID;
      if (B || Tt) {
        if (B && Tt) {
          T qb[4], qt[4], fb[4], ft[4], mEB, mET;
          cell(wi, wjB, qb, fb, mEB);
          cell(wi, wjT, qt, ft, mET);
          // rho^E, p^E at the quarter heights from the lower centre to the upper one
          const int q0 = 4 * (j0 - 1 + wjB - S.K[wi]) + 2 + 4 * ny;
          T r5[5], p5[5];
#pragma unroll
          for (int n = 0; n < 5; ++n) {
            r5[n] = rq[q0 + n];
            p5[n] = pq[q0 + n];
          }
          yface_o1(fb, qb[3], ft, qt[3], r5, p5, kc.dy, P, Dm, Dp);
        } else {
          T q[4], f[4], mE;
          cell(wi, B ? wjB : wjT, q, f, mE);
          const bool outside = S.flag[B ? wjT : wjB][wi] == F_OUT;
          const bool tr = outside && (B ? trN : trS);
          const T g[4] = {q[0], q[1], tr ? q[2] : -q[2], q[3]};
          T qm[4], qp[4], dq[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            qm[c] = B ? q[c] : g[c];
            qp[c] = B ? g[c] : q[c];
          }
          dq[0] = T(0);
          dq[1] = T(0);
          dq[2] = qp[2] - qm[2];
          dq[3] = T(0);
          yface(qm, qp, dq, T(0), P, Dm, Dp);
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        S.Dy[c][fy][fx] = Dm[c];
        S.Dy[4 + c][fy][fx] = Dp[c];
      }
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- update
  const int gi_me = i0 + tx, gj_me = j0 + ty;
  const bool inside = gi_me < nx && gj_me < ny;
  const unsigned char flag_me = S.flag[ty + 1][tx + 1];
  T my_rate = T(0);
  unsigned long long my_w = 0;
  bool bad = false;
  if (inside && flag_me == F_FLUID) {
    const T rdx = dt / kc.dx, rdy = dt / kc.dy;
    T qold[4], qn[4], m_full;
#pragma unroll
    for (int v = 0; v < 4; ++v) qold[v] = S.w[v][ty + 1][tx + 1];
    T dQ[4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
      dQ[c] = -rdx * (S.Dx[4 + c][ty][tx] + S.Dx[c][ty][tx + 1]) -
              rdy * (S.Dy[4 + c][ty][tx] + S.Dy[c][ty + 1][tx]);
    if (DEV) {
      const T rEc = tab(rt, 2 * (gj_me - S.K[tx + 1]) + 1, ny);
      qn[0] = qold[0] + (dQ[0] - rEc * dQ[3]);
      qn[1] = qold[1] + dQ[1];
      qn[2] = qold[2] + dQ[2];
      qn[3] = qold[3] + dQ[3];
      m_full = qn[3] * rEc + qn[0];
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) qn[c] = qold[c] + dQ[c];
      m_full = qn[0];
    }
    const size_t c = (size_t)gj_me * nx + gi_me;
#pragma unroll
    for (int v = 0; v < 4; ++v) qout[v * N + c] = qn[v];
    cell_epilogue<T, DEV>(p, kc, qn, m_full, my_rate, my_w, bad,
                          gi_me >= p.own_lo && gi_me < p.own_hi);
  } else if (inside) {
    const size_t c = (size_t)gj_me * nx + gi_me;
#pragma unroll
    for (int v = 0; v < 4; ++v) qout[v * N + c] = T(0);
    if (flag_me == F_SOLID) my_w = ONE_FIXED;
  }
  block_epilogue<T, TX, TY>(my_rate, my_w, bad, inside, gi_me, S.col, S.wmax, colsum, sc);
}

template <typename T, bool DEV, bool XOR>
void launch_o1_xt(const StepParams& p, const T* in, T* out, const uint8_t* solid,
                  const int32_t* Kref, const int32_t* Kcur, unsigned long long* colsum,
                  DevScalars* sc, const T* rt, const T* rq, const T* pq, cudaStream_t st) {
  const size_t smem = sizeof(SmemO1<T>);
  kernel_setup((const void*)step_o1_kernel<T, DEV, XOR>, TX * TY, smem);
  dim3 block(TX, TY);
  dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY);
  step_o1_kernel<T, DEV, XOR><<<grid, block, smem, st>>>(p, make_consts<T>(p), in, out, solid,
                                                          Kref, Kcur, colsum, sc, rt, rq, pq);
}

template <typename T, bool DEV>
void launch_o1_t(const StepParams& p, const T* in, T* out, const uint8_t* solid,
                 const int32_t* Kref, const int32_t* Kcur, unsigned long long* colsum,
                 DevScalars* sc, const T* rt, const T* rq, const T* pq, bool osher_romberg_x,
                 cudaStream_t st) {
  if (osher_romberg_x)
    launch_o1_xt<T, DEV, true>(p, in, out, solid, Kref, Kcur, colsum, sc, rt, rq, pq, st);
  else
    launch_o1_xt<T, DEV, false>(p, in, out, solid, Kref, Kcur, colsum, sc, rt, rq, pq, st);
}

}  // namespace

void launch_step_o1_f64(const StepParams& p, const StateF64& s, const uint8_t* solid,
                        const int32_t* Kcur, unsigned long long* colsum, DevScalars* sc,
                        const Tables& tb, const QuarterTables& tq, cudaStream_t st,
                        bool osher_romberg_x) {
  launch_o1_t<double, false>(p, s.in, s.out, solid, Kcur, Kcur, colsum, sc, tb.rhoE_d, tq.rhoE_d,
                             tq.pE_d, osher_romberg_x, st);
}

void launch_step_o1_f32(const StepParams& p, const StateF32& s, const uint8_t* solid,
                        const int32_t* Kref, const int32_t* Kcur, unsigned long long* colsum,
                        DevScalars* sc, const Tables& tb, const QuarterTables& tq,
                        cudaStream_t st, bool osher_romberg_x) {
  launch_o1_t<float, true>(p, s.in, s.out, solid, Kref, Kcur, colsum, sc, tb.rhoE_f, tq.rhoE_f,
                           tq.pE_f, osher_romberg_x, st);
}

}  // namespace fv
