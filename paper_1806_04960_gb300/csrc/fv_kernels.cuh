// Kernels of one time step of the well-balanced path-conservative scheme
// (Gaburro, Castro, Dumbser, Eq. (Scheme)) and the launch helpers used by the
// C ABI.  Internal header of libfv.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fv {

// Per-launch parameters shared by both precisions (doubles, converted in-kernel).
struct StepParams {
  int nx, ny;
  double dx, dy;
  double rho0, k0, g, eps, c, c2, kappa;
  int side[4];            // W, E, S, N: 0 wall, 1 transmissive
  double cfl;
  // Columns whose cells count in the signal rate and the status (a partitioned
  // domain's own columns; its halo columns are replaced by their owner's
  // values after each step); the whole grid unless set.
  int own_lo = 0, own_hi = 1 << 30;
};

// Device-resident step bookkeeping (one per domain).
struct DevScalars {
  double rate_cur;        // max signal rate of the state the next step starts from
  unsigned long long rate_acc;  // bits of the max rate being accumulated (>= 0 doubles)
  double t;               // simulated time
  double dt_last;         // dt of the last step
  long long steps;
  double dt_cur;          // dt of the next step (cfl / rate_cur)
  float dt_cur_f;         // same, rounded to float
  int status;             // bit 0: non-admissible state produced; bit 1 (fv_step_static
                          // only): non-admissible input state
};

// Equilibrium density table: rhoE[h + 2 ny] = rho0 exp(-kappa (h dy / 2)) for
// h in [-2 ny, 2 ny] (h counts half cells between a point and the level y0).
struct Tables {
  const double* rhoE_d;   // 4 ny + 1 doubles
  const float* rhoE_f;    // same, rounded to float
};

// rho^E and p^E = k0 (rho^E / rho0 - 1) at quarter-cell heights: entry
// q + 4 ny holds the value q dy / 4 above the level, q in [-4 ny, 4 ny]
// (first-order y faces evaluate the path at s = 0, 1/4, ..., 1).
struct QuarterTables {
  const double* rhoE_d;
  const double* pE_d;
  const float* rhoE_f;
  const float* pE_f;
};

struct StateF64 {
  const double* in;       // 4 planes of nx*ny, full conserved state
  double* out;
};

struct StateF32 {
  const float* in;        // 4 planes: m^f, mu, mv, a (m^f relative to Kref)
  float* out;             // written relative to Kcur
};

// osher_romberg_x: x faces by the conservative Osher-Romberg viscosity of Eq.
// (OR_cons) instead of the Gauss-Legendre Osher of Eq. (OsherMatrixFormal_approx).
// tiling: which kernel stages the step (the same arithmetic, the same results):
// TILING_TILE = step_kernel, one CTA per 32 x 8 tile (csrc/fv_kernels.cu);
// TILING_STRIP = strip_kernel, one CTA per 32-column strip (csrc/fv_strip.cu);
// TILING_AUTO = the strip kernel.
// strip_h: rows of a strip (a multiple of 8), 0 = chosen by strip_height.
enum StepTiling { TILING_AUTO = 0, TILING_TILE = 1, TILING_STRIP = 2 };
void launch_step_f64(const StepParams& p, const StateF64& s, const uint8_t* solid,
                     const int32_t* Kcur, unsigned long long* colsum, DevScalars* sc,
                     const Tables& tb, cudaStream_t st, bool osher_romberg_x = false,
                     int tiling = TILING_AUTO, int strip_h = 0);
void launch_step_f32(const StepParams& p, const StateF32& s, const uint8_t* solid,
                     const int32_t* Kref, const int32_t* Kcur, unsigned long long* colsum,
                     DevScalars* sc, const Tables& tb, cudaStream_t st,
                     bool osher_romberg_x = false, int tiling = TILING_AUTO, int strip_h = 0);
void launch_strip_f64(const StepParams& p, const StateF64& s, const uint8_t* solid,
                      const int32_t* Kcur, unsigned long long* colsum, DevScalars* sc,
                      const Tables& tb, cudaStream_t st, bool osher_romberg_x, int strip_h);
void launch_strip_f32(const StepParams& p, const StateF32& s, const uint8_t* solid,
                      const int32_t* Kref, const int32_t* Kcur, unsigned long long* colsum,
                      DevScalars* sc, const Tables& tb, cudaStream_t st, bool osher_romberg_x,
                      int strip_h);
// Strip height (rows, a multiple of 8) for an nx x ny grid when `resident`
// strip CTAs fit on the device at once.
int strip_height(int nx, int ny, int resident);
// First-order scheme of Sections 3.2-3.3 (csrc/fv_order1.cu).
void launch_step_o1_f64(const StepParams& p, const StateF64& s, const uint8_t* solid,
                        const int32_t* Kcur, unsigned long long* colsum, DevScalars* sc,
                        const Tables& tb, const QuarterTables& tq, cudaStream_t st,
                        bool osher_romberg_x = false);
void launch_step_o1_f32(const StepParams& p, const StateF32& s, const uint8_t* solid,
                        const int32_t* Kref, const int32_t* Kcur, unsigned long long* colsum,
                        DevScalars* sc, const Tables& tb, const QuarterTables& tq,
                        cudaStream_t st, bool osher_romberg_x = false);
void launch_finalize(const StepParams& p, int32_t* Kref, int32_t* Kcur,
                     unsigned long long* colsum, DevScalars* sc, int count_step,
                     cudaStream_t st);
void launch_prepare(double cfl, DevScalars* sc, cudaStream_t st);
// Levels' column sums and the signal rate of a state q (before its first
// step); a non-admissible fluid cell sets status_bits in sc->status.
void launch_prologue_f64(const StepParams& p, const double* q, const uint8_t* solid,
                         unsigned long long* colsum, DevScalars* sc, cudaStream_t st,
                         int status_bits = 1);
void launch_to_dev(const StepParams& p, const double* q, const uint8_t* solid,
                   const int32_t* K, const Tables& tb, float* out, cudaStream_t st);
void launch_from_dev(const StepParams& p, const float* in, const uint8_t* solid,
                     const int32_t* K, const Tables& tb, double* q, cudaStream_t st);
void launch_mass(const StepParams& p, const double* q, const uint8_t* solid, double* partial,
                 int nblocks, double* out, cudaStream_t st);
void launch_zero_solid(const StepParams& p, double* q, const uint8_t* solid, cudaStream_t st);

// Host description of one domain of a batch (device pointers).
struct BatchDomainDesc {
  StepParams p;
  void* q[2];
  const uint8_t* solid;
  int32_t* Kref;
  int32_t* Kcur;
  unsigned long long* colsum;
  DevScalars* sc;
  const double* rhoE_d;
  const float* rhoE_f;
};

// Device table of a batch: batch_table_bytes bytes, filled on the host by
// batch_fill_table and copied to the device by the caller.
size_t batch_table_bytes(int ndom, bool f64);
void batch_fill_table(const BatchDomainDesc* descs, int ndom, bool f64, void* host_dst);
// The batched step stages by strips (csrc/fv_strip.cu): work[k] = (domain,
// strip column, strip row, strip height, a multiple of 8).  BATCH_STRIP_H is
// the height of a new batch's work list, until fv_batch_tune picks another.
constexpr int BATCH_STRIP_H = 128;
int batch_grid_size(bool f64);
// persistent: a grid of the resident CTAs striding over the work list;
// otherwise one CTA per strip.
void launch_batch_step(bool f64, const void* table, const int4* work, int nwork, int parity,
                       bool persistent, cudaStream_t st);
void launch_batch_finalize(bool f64, const void* table, int ndom, double cfl, int count_step,
                           cudaStream_t st);
void launch_batch_prepare(bool f64, const void* table, int ndom, double cfl, cudaStream_t st);

// One-time set-up of a kernel on the current device, cached per kernel and
// device ordinal (thread-safe): opts the kernel into `smem` bytes of dynamic
// shared memory and returns the number of CTAs of `threads` threads that are
// resident at once on that device (CTAs per SM x SMs, at least 1).  Every
// launch with more than 48 KB of dynamic shared memory goes through it, so a
// handle created on a second GPU gets the opt-in on that GPU too.
int kernel_setup(const void* kernel, int threads, size_t smem);

// Message returned by fv_last_error() on this thread.
void set_last_error(const char* msg);

}  // namespace fv
