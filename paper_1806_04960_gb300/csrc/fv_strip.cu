// One time step of Eq. (Scheme) by column strips: one CTA per strip of 32
// columns and H rows (H a multiple of 8), marching upwards in blocks of 8 rows.
// The cell and face arithmetic is that of the tile kernel (fv_tile.cuh); what
// differs is the staging.  Consecutive blocks share two reconstructed rows and
// one row of y faces, which a tile kernel recomputes for every tile: the
// window of Q^n (WRING rows), the reconstruction records and the y-face
// fluctuations (RING rows) live in ring buffers, so that per block only 8 new
// window rows are loaded, 8 rows (+ the ring columns) reconstructed and 8 rows
// of y faces solved.  The window ring holds the 10 rows a block reads plus the
// 8 the next block loads, so a block's load never waits for the previous
// block's update.  With 288 threads (FP32; 320 in FP64) every phase of a block
// is one pass, apart from the faces:
//
//   load    rows j0+2 .. j0+9 of the window (288 cells): their global loads
//           were issued by the previous block before its faces phase and are
//           only stored here (the first block of a strip loads directly)
//   recon   rows j0+1 .. j0+8, 34 columns (272 cells)
//   faces   x faces of rows j0 .. j0+7 (264; warps 0-8), then y faces above
//           rows j0 .. j0+7 (256; warps 0-7; with 320 threads warp 9 takes
//           the first 32), no warp holding both kinds at once
//   update  rows j0 .. j0+7 (256 cells)
//
// A prologue per strip loads rows jstart-2 .. jstart+1, reconstructs rows
// jstart-1 and jstart and solves the y faces between them.  The epilogue
// (signal rate, detector column sums, status) is reduced once per strip.
#include <cuda_runtime.h>

#include "fv_consts.cuh"
#include "fv_kernels.cuh"
#include "fv_model.cuh"
#include "fv_tile.cuh"

namespace fv {

namespace {

using namespace tile;

constexpr int SX = 32;          // strip width (cells)
constexpr int BY = 8;           // rows per block
constexpr int SWX = SX + 4;     // window columns: 2-cell halo on both sides
constexpr int SRX = SX + 2;     // reconstructed columns: 1-cell ring
constexpr int RING = 10;        // rows of the record and y-face rings
constexpr int WRING = 18;       // rows of the window ring
constexpr int NXF = (SX + 1) * BY;  // x faces of a block
constexpr int NYF = SX * BY;        // y faces of a block

// Threads per CTA: 9 warps in FP32 (measured faster: every warp loads, and
// at most one idles in a phase), 10 in FP64.
template <typename T>
__host__ __device__ constexpr int strip_threads() {
  return sizeof(T) == 8 ? 320 : 288;
}
static_assert(BY * SWX <= 288 && BY * SRX <= 288 && NXF <= 288, "one pass per phase");

// FP64 keeps the face fluxes of each reconstructed cell (face_fluxes) beside
// its record: its two x faces, two y faces and update then read them instead
// of forming them again (four fewer reciprocals per cell on the FP64 pipe).
// FP32 forms them where they are used: its three CTAs per SM have no room
// for the two more rings.
template <typename T>
__host__ __device__ constexpr bool keeps_fluxes() {
  return sizeof(T) == 8;
}

template <typename T>
struct StripSmem {
  static constexpr int FR = keeps_fluxes<T>() ? RING : 1, FX = keeps_fluxes<T>() ? SRX : 1;
  V4<T> w[WRING][SWX];         // window rows of Q^n (stored form, re-based)
  V4<T> rs[RING][SRX];         // (alpha^E, m^E centre, bottom, top face)
  V4<T> rf[4][RING][SRX];      // face fluctuation states W, E, S, N at t^{n+1/2}
  V4<T> fl[2][FR][FX];         // x fluxes of W, E and y fluxes of S, N (FP64)
  V4<T> base[RING][SX];        // centre fluctuation at t^{n+1/2}
  V4<T> Dx[2][BY][SX + 1];     // D-, D+ of the block's x faces
  V4<T> Dy[2][RING][SX];       // D-, D+ of the y faces, by the row below the face
  T ga[2][RING][SX];           // limited alpha slopes
  unsigned long long col[BY][SX];
  double wmax[10];
  int K[SWX];                  // levels of the window columns
  unsigned char flag[WRING][SWX];
};

// Strip (sx, sy) of one domain: columns 32 sx .. 32 sx + 31, rows H sy ..
// H sy + H - 1; called by the whole CTA.
template <typename T, bool DEV, bool XOR>
__device__ __forceinline__ void strip_body(const StepParams& p, const KConsts<T>& kc,
                                           const T* __restrict__ qin, T* __restrict__ qout,
                                           const uint8_t* __restrict__ solid,
                                           const int32_t* __restrict__ Kref,
                                           const int32_t* __restrict__ Kcur,
                                           unsigned long long* __restrict__ colsum,
                                           DevScalars* __restrict__ sc, const T* __restrict__ rt,
                                           int sx, int sy, int H, StripSmem<T>& S) {
  constexpr int NTS = strip_threads<T>();
  constexpr int YF0 = NTS - 9 * 32;  // y faces taken by the warps past the x faces' nine
  constexpr bool FLX = keeps_fluxes<T>();
  const int t = threadIdx.x;
  const int nx = p.nx, ny = p.ny;
  const size_t N = (size_t)nx * ny;
  const int i0 = sx * SX;
  const int jstart = sy * H;
  const int jend = min(jstart + H, ny);
  // Row r sits in window slot wslot(r) = (r - jstart + 2) mod WRING and in
  // record / y-face slot slot(r) = (r - jstart + 2) mod RING.  Slots are
  // carried as a base plus an offset, wrapped by one compare and subtract.
  auto wwrap = [](int x) -> int { return x >= WRING ? x - WRING : x; };
  auto rwrap = [](int x) -> int { return x >= RING ? x - RING : x; };

  const Phys<T>& P = kc.P;
  const Sides sd = sides_of(p);
  const T dx = kc.dx, dy = kc.dy;
  // dt of this step, computed once per step by the finalize/prepare kernels
  const T dt = sizeof(T) == 8 ? (T)sc->dt_cur : (T)sc->dt_cur_f;
  const T rdx = dt / dx, rdy = dt / dy;
  ReconConsts<T> RC = kc.R;
  RC.half_dt = T(0.5) * dt;

  // rows ra .. ra+nrows-1; wa = wslot(ra)
  auto load_rows = [&](int ra, int wa, int nrows) {
    for (int idx = t; idx < nrows * SWX; idx += NTS) {
      const int k = idx / SWX, wi = idx % SWX;
      const int rr = ra + k;
      const int s = wwrap(wa + k);
      S.flag[s][wi] = load_cell<T, DEV>(qin, solid, Kref, Kcur, rt, nx, ny, N, i0 - 2 + wi, rr,
                                        S.w[s][wi]);
    }
  };
  // rows ra .. ra+nrows-1; wa = wslot(ra - 1), sa = slot(ra)
  auto recon_rows = [&](int ra, int wa, int sa, int nrows) {
    for (int idx = t; idx < nrows * SRX; idx += NTS) {
      const int k = idx / SRX, rx = idx % SRX, wi = rx + 1;
      const int rr = ra + k;
      const int ws = wwrap(wa + k + 1);
      if (S.flag[ws][wi] != F_FLUID) continue;
      const int s = rwrap(sa + k), sS = wwrap(wa + k), sN = wwrap(wa + k + 2);
      V4<T> rs, rf[4];
      T base[4], ga[2];
      recon_cell<T, DEV>(S.w[sS], S.w[ws], S.w[sN], S.flag[sS], S.flag[ws], S.flag[sN], S.K, wi,
                         rr, rt, ny, sd, P, RC, rs, rf, base, ga);
      S.rs[s][rx] = rs;
#pragma unroll
      for (int f = 0; f < 4; ++f) S.rf[f][s][rx] = rf[f];
      if constexpr (FLX)
        face_fluxes(rs, rf, rs.x <= RC.ten_eps, S.fl[0][s][rx], S.fl[1][s][rx]);
      if (rx >= 1 && rx <= SX) {
        S.base[s][rx - 1] = pack(base);
        S.ga[0][s][rx - 1] = ga[0];
        S.ga[1][s][rx - 1] = ga[1];
      }
    }
  };
  // y face between rows rB and rB + 1 of strip column fx; wB = wslot(rB),
  // sB = slot(rB)
  auto yface_at = [&](int rB, int wB, int sB, int fx) {
    const int rx = fx + 1, sT = rwrap(sB + 1), wT = wwrap(wB + 1);
    T Dm[4], Dp[4];
    y_face<T>(S.flag[wB][rx + 1], S.flag[wT][rx + 1], &S.rs[sB][rx], &S.rf[F_N][sB][rx],
              &S.rs[sT][rx], &S.rf[F_S][sT][rx], S.K[rx + 1], rB + 1, rt, ny, sd, P, Dm, Dp,
              FLX ? &S.fl[1][sB][rx] : nullptr, FLX ? &S.fl[1][sT][rx] : nullptr);
    S.Dy[0][sB][fx] = pack(Dm);
    S.Dy[1][sB][fx] = pack(Dp);
  };

  // ------------------------------------------------------------ prologue
  for (int idx = t; idx < SWX; idx += NTS) {
    const int gi = i0 - 2 + idx;
    S.K[idx] = (gi >= 0 && gi < nx) ? Kcur[gi] : 0;
  }
  load_rows(jstart - 2, 0, 4);
  __syncthreads();
  recon_rows(jstart - 1, 0, 1, 2);
  __syncthreads();
  if (t < SX) yface_at(jstart - 1, 1, 1, t);

  T my_rate = T(0);
  unsigned long long my_w = 0;
  bool bad = false;
  const int ux = t % SX, uy = t / SX;  // update: column and row in the block (t < 256)
  const int gi_me = i0 + ux;
  const bool own_me = gi_me >= p.own_lo && gi_me < p.own_hi;

  // the next block's window cell of this thread (t < 288), loaded one block
  // ahead: cell (pwi, pk) of its 8 new rows
  CellLoad<T> pre{};
  const int pk = t / SWX, pwi = t % SWX;

  // slots of row j0 in the window ring and in the record ring
  int wb = 2, sb = 2;
  for (int j0 = jstart; j0 < jend; j0 += BY, wb = wwrap(wb + BY), sb = rwrap(sb + BY)) {
    // ---------------------------------------------------------- load
    if (j0 == jstart) {
      load_rows(j0 + 2, wwrap(wb + 2), BY);
    } else if (t < BY * SWX) {
      const int s = wwrap(wwrap(wb + 2) + pk);
      S.flag[s][pwi] = commit_cell<T, DEV>(pre, rt, ny, j0 + 2 + pk, S.w[s][pwi]);
    }
    __syncthreads();
    // ---------------------------------------------------------- recon
    recon_rows(j0 + 1, wb, rwrap(sb + 1), BY);
    __syncthreads();
    // ---------------------------------------------------------- faces
    // (in a strip's last block a fetch of row -1, which loads nothing: every
    // block then defines the registers, so they are not live across a block)
    if (NTS == BY * SWX || t < BY * SWX)
      fetch_cell<T, DEV>(qin, solid, Kref, Kcur, nx, ny, N, i0 - 2 + pwi,
                         j0 + BY < jend ? j0 + BY + 2 + pk : -1, pre);
    if (t < NXF) {
      const int fx = t % (SX + 1), fy = t / (SX + 1);
      const int s = rwrap(sb + fy), ws = wwrap(wb + fy);
      T Dm[4], Dp[4];
      x_face<T, XOR>(S.flag[ws][fx + 1], S.flag[ws][fx + 2], &S.rs[s][fx], &S.rf[F_E][s][fx],
                     &S.rs[s][fx + 1], &S.rf[F_W][s][fx + 1], sd, P, Dm, Dp,
                     FLX ? &S.fl[0][s][fx] : nullptr, FLX ? &S.fl[0][s][fx + 1] : nullptr);
      S.Dx[0][fy][fx] = pack(Dm);
      S.Dx[1][fy][fx] = pack(Dp);
    } else if (YF0 > 0 && t >= 9 * 32) {
      const int k = t - 9 * 32, fy = k / SX;
      yface_at(j0 + fy, wwrap(wb + fy), rwrap(sb + fy), k % SX);
    }
    if (t < NYF - YF0) {
      const int k = t + YF0, fy = k / SX;
      yface_at(j0 + fy, wwrap(wb + fy), rwrap(sb + fy), k % SX);
    }
    __syncthreads();
    // ---------------------------------------------------------- update
    if (t < SX * BY) {
      const int r = j0 + uy;
      const int s = rwrap(sb + uy), ws = wwrap(wb + uy);
      const int sbelow = s == 0 ? RING - 1 : s - 1;  // slot of row r - 1
      const bool inside = gi_me < nx && r < ny;
      const unsigned char flag_me = S.flag[ws][ux + 2];
      if (inside && flag_me == F_FLUID) {
        T qold[4];
        unpack(S.w[ws][ux + 2], qold);
        const int K = S.K[ux + 2];
        const V4<T> rf[4] = {S.rf[F_W][s][ux + 1], S.rf[F_E][s][ux + 1], S.rf[F_S][s][ux + 1],
                             S.rf[F_N][s][ux + 1]};
        const T rEc = DEV ? tab(rt, 2 * (r - K) + 1, ny) : T(0);
        T qn[4];
        const T m_full = update_cell<T, DEV>(qold, S.rs[s][ux + 1], rf, S.base[s][ux],
                                             S.ga[0][s][ux], S.ga[1][s][ux], S.Dx[1][uy][ux],
                                             S.Dx[0][uy][ux + 1], S.Dy[1][sbelow][ux],
                                             S.Dy[0][s][ux], rEc, rdx, rdy, dx, dy, P, qn,
                                             FLX ? &S.fl[0][s][ux + 1] : nullptr,
                                             FLX ? &S.fl[1][s][ux + 1] : nullptr);
        const size_t c = (size_t)r * nx + gi_me;
#pragma unroll
        for (int v = 0; v < 4; ++v) qout[v * N + c] = qn[v];
        T rate = T(0);
        unsigned long long w = 0;
        cell_epilogue<T, DEV>(p, kc, qn, m_full, rate, w, bad, own_me);
        my_rate = fmax(my_rate, rate);
        my_w += w;
      } else if (inside) {
        const size_t c = (size_t)r * nx + gi_me;
#pragma unroll
        for (int v = 0; v < 4; ++v) qout[v * N + c] = T(0);
        if (flag_me == F_SOLID) my_w += ONE_FIXED;
      }
    }
    // The next block's load writes window rows j0+10 .. j0+17, slots no
    // phase of this block reads; its recon and faces write record and y-face
    // slots read above, behind its first barrier.
  }

  // ------------------------------------------------------------ epilogue
  if (bad) atomicOr(&sc->status, 1);
  if (t < SX * BY) S.col[uy][ux] = my_w;
  T r_t = my_rate;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r_t = fmax(r_t, __shfl_xor_sync(0xffffffffu, r_t, o));
  if ((t & 31) == 0) S.wmax[t >> 5] = (double)r_t;
  __syncthreads();
  if (t < SX && gi_me < nx) {
    unsigned long long s = 0;
#pragma unroll
    for (int r = 0; r < BY; ++r) s += S.col[r][t];
    if (s) atomicAdd(&colsum[gi_me], s);
  }
  if (t == 0) {
    double mrate = 0.0;
#pragma unroll
    for (int k = 0; k < NTS / 32; ++k) mrate = fmax(mrate, S.wmax[k]);
    if (mrate > 0.0) atomicMax(&sc->rate_acc, (unsigned long long)__double_as_longlong(mrate));
  }
}

template <typename T, bool DEV, bool XOR>
__global__ void __launch_bounds__(strip_threads<T>(), (sizeof(T) == 8 ? 1 : 3))
    strip_kernel(StepParams p, KConsts<T> kc, const T* __restrict__ qin, T* __restrict__ qout,
                 const uint8_t* __restrict__ solid, const int32_t* __restrict__ Kref,
                 const int32_t* __restrict__ Kcur, unsigned long long* __restrict__ colsum,
                 DevScalars* __restrict__ sc, const T* __restrict__ rt, int H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StripSmem<T>& S = *reinterpret_cast<StripSmem<T>*>(smem_raw);
  strip_body<T, DEV, XOR>(p, kc, qin, qout, solid, Kref, Kcur, colsum, sc, rt, blockIdx.x,
                          blockIdx.y, H, S);
}

// Batched step: every strip (domain, sx, sy, H) of an ensemble, either one
// CTA per strip (the block scheduler hands strips out as CTAs finish) or
// round-robin over a persistent grid of the resident CTAs; each domain uses
// its own parameters, dt, levels and accumulators.  parity selects the state
// buffer read.
template <typename T, bool DEV>
__global__ void __launch_bounds__(strip_threads<T>(), (sizeof(T) == 8 ? 1 : 3))
    batch_strip_kernel(const BatchDomain<T>* __restrict__ doms, const int4* __restrict__ work,
                       int nwork, int parity) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  StripSmem<T>& S = *reinterpret_cast<StripSmem<T>*>(smem_raw);
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int4 sw = work[w];
    const BatchDomain<T>& d = doms[sw.x];
    strip_body<T, DEV, false>(d.p, d.kc, d.q[parity], d.q[1 - parity], d.solid, d.Kref, d.Kcur,
                              d.colsum, d.sc, d.rt, sw.y, sw.z, sw.w, S);
    __syncthreads();  // shared memory is reused by the next strip
  }
}

template <typename T, bool DEV, bool XOR>
void launch_strip_xt(const StepParams& p, const T* in, T* out, const uint8_t* solid,
                     const int32_t* Kref, const int32_t* Kcur, unsigned long long* colsum,
                     DevScalars* sc, const T* rt, int strip_h, cudaStream_t st) {
  constexpr int NTS = strip_threads<T>();
  const size_t smem = sizeof(StripSmem<T>);
  const int resident = kernel_setup((const void*)strip_kernel<T, DEV, XOR>, NTS, smem);
  const int H = strip_h > 0 ? strip_h : strip_height(p.nx, p.ny, resident);
  const dim3 grid((p.nx + SX - 1) / SX, (p.ny + H - 1) / H);
  strip_kernel<T, DEV, XOR><<<grid, NTS, smem, st>>>(p, make_consts<T>(p), in, out, solid, Kref,
                                                      Kcur, colsum, sc, rt, H);
}

template <typename T, bool DEV>
int batch_grid_t() {
  return kernel_setup((const void*)batch_strip_kernel<T, DEV>, strip_threads<T>(),
                      sizeof(StripSmem<T>));
}

}  // namespace

int batch_grid_size(bool f64) {
  return f64 ? batch_grid_t<double, false>() : batch_grid_t<float, true>();
}

void launch_batch_step(bool f64, const void* table, const int4* work, int nwork, int parity,
                       bool persistent, cudaStream_t st) {
  if (f64) {
    const int res = batch_grid_t<double, false>();
    const int grid = persistent && res < nwork ? res : nwork;
    batch_strip_kernel<double, false><<<grid, strip_threads<double>(), sizeof(StripSmem<double>), st>>>(
        static_cast<const BatchDomain<double>*>(table), work, nwork, parity);
  } else {
    const int res = batch_grid_t<float, true>();
    const int grid = persistent && res < nwork ? res : nwork;
    batch_strip_kernel<float, true><<<grid, strip_threads<float>(), sizeof(StripSmem<float>), st>>>(
        static_cast<const BatchDomain<float>*>(table), work, nwork, parity);
  }
}

int strip_height(int nx, int ny, int resident) {
  // Every CTA does about (H/8 + 0.4) blocks of work (the prologue is about
  // 0.4 of a block); CTAs run in waves of `resident`.  Minimise waves x work.
  const int ncol = (nx + SX - 1) / SX;
  const int hmax = ((ny + BY - 1) / BY) * BY;
  if (resident < 1) resident = 1;
  int best = BY;
  double best_cost = 1e300;
  for (int k = 32; k >= 1; --k) {
    const int H = k * BY;
    if (H > hmax) continue;
    const long long ctas = (long long)ncol * ((ny + H - 1) / H);
    const long long waves = (ctas + resident - 1) / resident;
    const double cost = (double)waves * ((double)H / BY + 0.4);
    if (cost < best_cost) {
      best_cost = cost;
      best = H;
    }
  }
  return best;
}

void launch_strip_f64(const StepParams& p, const StateF64& s, const uint8_t* solid,
                      const int32_t* Kcur, unsigned long long* colsum, DevScalars* sc,
                      const Tables& tb, cudaStream_t st, bool osher_romberg_x, int strip_h) {
  if (osher_romberg_x)
    launch_strip_xt<double, false, true>(p, s.in, s.out, solid, Kcur, Kcur, colsum, sc, tb.rhoE_d,
                                         strip_h, st);
  else
    launch_strip_xt<double, false, false>(p, s.in, s.out, solid, Kcur, Kcur, colsum, sc,
                                          tb.rhoE_d, strip_h, st);
}

void launch_strip_f32(const StepParams& p, const StateF32& s, const uint8_t* solid,
                      const int32_t* Kref, const int32_t* Kcur, unsigned long long* colsum,
                      DevScalars* sc, const Tables& tb, cudaStream_t st, bool osher_romberg_x,
                      int strip_h) {
  if (osher_romberg_x)
    launch_strip_xt<float, true, true>(p, s.in, s.out, solid, Kref, Kcur, colsum, sc, tb.rhoE_f,
                                       strip_h, st);
  else
    launch_strip_xt<float, true, false>(p, s.in, s.out, solid, Kref, Kcur, colsum, sc,
                                        tb.rhoE_f, strip_h, st);
}

}  // namespace fv
