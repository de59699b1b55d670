// One time step of Eq. (Scheme) (Gaburro, Castro, Dumbser) is one step
// kernel plus a finalize kernel.  The default step kernel stages by column
// strips (strip_kernel, fv_strip.cu); this file holds the tile staging
// (fv_set_tiling(h, FV_TILING_TILE)) and the kernels around the step:
//
//   step_kernel   one CTA per TX x TY tile of cells (the cell and face
//                 arithmetic of fv_tile.cuh, shared with strip_kernel):
//     load      Q^n of the tile plus a 2-cell halo into shared memory, with
//               the solid/outside flags and the column levels K_i;
//     recon     for the tile plus a 1-cell ring: fluctuations w.r.t. the
//               cell's water-at-rest state, slopes, Barth-Jespersen factor,
//               order switch, half-step predictor, face-midpoint states at
//               t^{n+1/2} (Section 3.4);
//     faces     every x face (Osher, Gauss-Legendre) and y face (well-balanced
//               Osher-Romberg) of the tile solved once into shared memory;
//     update    Q^{n+1} with the interior integral of Eq.
//               (b^y_3_final_integral) plus the conservative part;
//     epilogue  max signal rate for the next dt, the free-surface detector's
//               column sums of Eq. (Free_surf_detector) in exact 2^-32 fixed
//               point, non-admissible-state flag.
//   finalize_kernel   K_i = round(column sum), dt bookkeeping, accumulator
//                     reset (one thread per column over the grid);
//   prepare_kernel, prologue_kernel, to_dev/from_dev, mass and the batch's
//   per-domain finalize and prepare.
//
// The FP64 instantiation stores the full state; the FP32 instantiation stores
// the deviation m^f = m - alpha rho^E(y; K_i) so that a state at rest is
// represented by exact zeros.
#include <cuda_runtime.h>

#include <cmath>
#include <map>
#include <mutex>
#include <utility>

#include "fv_consts.cuh"
#include "fv_kernels.cuh"
#include "fv_model.cuh"
#include "fv_tile.cuh"

namespace fv {

namespace {

using namespace tile;

constexpr int TX = 32, TY = 8;
constexpr int NT = TX * TY;
constexpr int WX = TX + 4, WY = TY + 4;  // window: tile + 2-cell halo
constexpr int RX = TX + 2, RY = TY + 2;  // reconstructed cells: tile + 1 ring


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
  const Sides sd = sides_of(p);
  const T dx = kc.dx, dy = kc.dy;
  // dt of this step, computed once per step by the finalize/prepare kernels
  const T dt = sizeof(T) == 8 ? (T)sc->dt_cur : (T)sc->dt_cur_f;

  // ---------------------------------------------------------------- load
  // The window row by row (coalesced), every cell's loads issued together.
#pragma unroll
  for (int k = 0; k < (WX * WY + NT - 1) / NT; ++k) {
    const int idx = tid + k * NT;
    if (idx < WX * WY) {
      const int wj = idx / WX, wi = idx % WX;
      S.flag[wj][wi] = load_cell<T, DEV>(qin, solid, Kref, Kcur, rt, nx, ny, N, i0 - 2 + wi,
                                         j0 - 2 + wj, S.u.w[wj][wi]);
    }
  }
  for (int idx = tid; idx < WX; idx += NT) {
    const int gi = i0 - 2 + idx;
    S.K[idx] = (gi >= 0 && gi < nx) ? Kcur[gi] : 0;
  }
  __syncthreads();

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
    V4<T> rs, rf[4];
    T base[4], ga[2];
    recon_cell<T, DEV>(S.u.w[wj - 1], S.u.w[wj], S.u.w[wj + 1], S.flag[wj - 1], S.flag[wj],
                       S.flag[wj + 1], S.K, wi, j0 - 1 + ry, rt, ny, sd, P, RC, rs, rf, base, ga);
    S.rs[ry][rx] = rs;
#pragma unroll
    for (int f = 0; f < 4; ++f) S.rf[f][ry][rx] = rf[f];
    if (rx >= 1 && rx <= TX && ry >= 1 && ry <= TY) {
      S.base[ry - 1][rx - 1] = pack(base);
      S.ga[0][ry - 1][rx - 1] = ga[0];
      S.ga[1][ry - 1][rx - 1] = ga[1];
    }
  }
  __syncthreads();  // window no longer needed: its storage becomes Dx/Dy

  // ---------------------------------------------------------------- faces
  for (int idx = tid; idx < (TX + 1) * TY + TX * (TY + 1); idx += NT) {
    T Dm[4], Dp[4];
    if (idx < (TX + 1) * TY) {
      const int fx = idx % (TX + 1), fy = idx / (TX + 1);
      const int rxL = fx, rxR = fx + 1, ry = fy + 1;
      x_face<T, XOR>(S.flag[ry + 1][rxL + 1], S.flag[ry + 1][rxR + 1], &S.rs[ry][rxL],
                     &S.rf[F_E][ry][rxL], &S.rs[ry][rxR], &S.rf[F_W][ry][rxR], sd, P, Dm, Dp);
      S.u.d.Dx[0][fy][fx] = pack(Dm);
      S.u.d.Dx[1][fy][fx] = pack(Dp);
    } else {
      const int k = idx - (TX + 1) * TY;
      const int fx = k % TX, fy = k / TX;
      const int rx = fx + 1, ryB = fy, ryT = fy + 1;
      y_face<T>(S.flag[ryB + 1][rx + 1], S.flag[ryT + 1][rx + 1], &S.rs[ryB][rx],
                &S.rf[F_N][ryB][rx], &S.rs[ryT][rx], &S.rf[F_S][ryT][rx], S.K[rx + 1],
                j0 - 1 + ryT, rt, ny, sd, P, Dm, Dp);
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
    const V4<T> rf[4] = {S.rf[F_W][ry][rx], S.rf[F_E][ry][rx], S.rf[F_S][ry][rx],
                         S.rf[F_N][ry][rx]};
    const T rEc = DEV ? tab(rt, 2 * (gj_me - K) + 1, ny) : T(0);
    T qn[4];
    const T m_full = update_cell<T, DEV>(qold, S.rs[ry][rx], rf, S.base[ty][tx], S.ga[0][ty][tx],
                                         S.ga[1][ty][tx], S.u.d.Dx[1][ty][tx],
                                         S.u.d.Dx[0][ty][tx + 1], S.u.d.Dy[1][ty][tx],
                                         S.u.d.Dy[0][ty + 1][tx], rEc, dt / dx, dt / dy, dx, dy, P,
                                         qn);
    const size_t c = (size_t)gj_me * nx + gi_me;
#pragma unroll
    for (int v = 0; v < 4; ++v) qout[v * N + c] = qn[v];
    // epilogue: admissibility, signal rate, detector weight
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
// One thread per column over the grid; the scalars in block 0.
__global__ void finalize_kernel(StepParams p, int32_t* __restrict__ Kref, int32_t* __restrict__ Kcur,
                                unsigned long long* __restrict__ colsum,
                                DevScalars* __restrict__ sc, int count_step) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.nx; i += gridDim.x * blockDim.x) {
    const unsigned long long cs = colsum[i];
    const int32_t k = Kcur[i];
    colsum[i] = 0ull;
    Kref[i] = k;
    Kcur[i] = level_of(cs, p.ny);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
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
                                DevScalars* sc, int status_bits) {
  const size_t N = (size_t)p.nx * p.ny;
  // the step kernels' constants (KConsts<double>): IEEE division here as on the host
  const double inv_dx = 1.0 / p.dx, inv_dy = 1.0 / p.dy, inv_1meps = 1.0 / (1.0 - p.eps);
  double my_rate = 0.0;
  bool bad = false;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < N;
       c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % p.nx);
    if (solid[c]) {
      atomicAdd(&colsum[i], ONE_FIXED);
      continue;
    }
    double r;
    unsigned long long qw;
    bool b;
    rate_weight_f64(p, inv_dx, inv_dy, inv_1meps, q[c], q[N + c], q[2 * N + c], q[3 * N + c], r,
                    qw, b);
    if (b) bad = true;
    if (r >= 0.0) my_rate = fmax(my_rate, r);
    if (qw) atomicAdd(&colsum[i], qw);
  }
  if (bad) atomicOr(&sc->status, status_bits);
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
  kernel_setup((const void*)step_kernel<T, DEV, XOR>, NT, smem);
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

int kernel_setup(const void* kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> resident;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(kernel, dev);
  auto it = resident.find(key);
  if (it != resident.end()) return it->second;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  resident.emplace(key, n);
  return n;
}

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
                     const Tables& tb, cudaStream_t st, bool osher_romberg_x, int tiling,
                     int strip_h) {
  if (tiling == TILING_TILE)
    launch_step_t<double, false>(p, s.in, s.out, solid, Kcur, Kcur, colsum, sc, tb.rhoE_d,
                                 tb.rhoE_d, osher_romberg_x, st);
  else
    launch_strip_f64(p, s, solid, Kcur, colsum, sc, tb, st, osher_romberg_x, strip_h);
}

void launch_step_f32(const StepParams& p, const StateF32& s, const uint8_t* solid,
                     const int32_t* Kref, const int32_t* Kcur, unsigned long long* colsum,
                     DevScalars* sc, const Tables& tb, cudaStream_t st, bool osher_romberg_x,
                     int tiling, int strip_h) {
  if (tiling == TILING_TILE)
    launch_step_t<float, true>(p, s.in, s.out, solid, Kref, Kcur, colsum, sc, tb.rhoE_d,
                               tb.rhoE_f, osher_romberg_x, st);
  else
    launch_strip_f32(p, s, solid, Kref, Kcur, colsum, sc, tb, st, osher_romberg_x, strip_h);
}

void launch_finalize(const StepParams& p, int32_t* Kref, int32_t* Kcur,
                     unsigned long long* colsum, DevScalars* sc, int count_step,
                     cudaStream_t st) {
  int blocks = (p.nx + 255) / 256;
  if (blocks > 152) blocks = 152;
  finalize_kernel<<<blocks, 256, 0, st>>>(p, Kref, Kcur, colsum, sc, count_step);
}

void launch_prepare(double cfl, DevScalars* sc, cudaStream_t st) {
  prepare_kernel<<<1, 1, 0, st>>>(cfl, sc);
}

void launch_prologue_f64(const StepParams& p, const double* q, const uint8_t* solid,
                         unsigned long long* colsum, DevScalars* sc, cudaStream_t st,
                         int status_bits) {
  prologue_kernel<<<grid_1d((size_t)p.nx * p.ny), 256, 0, st>>>(p, q, solid, colsum, sc,
                                                                 status_bits);
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
