// fv_step_static: one FP64 time step without any device allocation.
//
// Some callers cannot allocate device memory: an application that owns all
// of its GPU memory through its own pool and forbids further allocations, or a
// latency-critical loop where cudaMalloc's implicit device synchronisation is
// not acceptable.  For them this entry point keeps the step's scratch (column
// sums of the free-surface detector, detected levels, the equilibrium density
// table and the step scalars) in one file-scope device array instead of
// memory allocated by fv_create.  The caller passes the state in and out.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "fv.h"
#include "fv_kernels.cuh"

using namespace fv;

namespace {

constexpr int kMaxNx = FV_STATIC_MAX_NX;
constexpr int kMaxNy = FV_STATIC_MAX_NY;

// Layout of the scratch array (all offsets 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffScalars = 0;
constexpr size_t kOffColsum = align256(kOffScalars + sizeof(DevScalars));
constexpr size_t kOffK = align256(kOffColsum + sizeof(unsigned long long) * kMaxNx);
constexpr size_t kOffRhoE = align256(kOffK + sizeof(int32_t) * 2 * kMaxNx);
constexpr size_t kScratchBytes = align256(kOffRhoE + sizeof(double) * (4 * (size_t)kMaxNy + 1));

// Held by every GPU that loads the library until the process exits.  Its name
// is only a host-side stand-in: host code must use the address obtained from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_fv_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Host copy of the equilibrium density table rho^E(h dy / 2) = rho0 exp(-kappa
// h dy / 2), h in [-2 ny, 2 ny], filled with the same host arithmetic as
// fv_create's table; a fixed static buffer, guarded by g_table_mutex while it is
// filled and copied.  The table is copied to a device's array only when its
// parameters (ny, dy, rho0, kappa) differ from the ones last copied there.
double g_host_table[4 * (size_t)kMaxNy + 1];
std::mutex g_table_mutex;
struct TableKey {
  int ny = -1;
  double dy = 0.0, rho0 = 0.0, kappa = 0.0;
  bool operator==(const TableKey& o) const {
    return ny == o.ny && dy == o.dy && rho0 == o.rho0 && kappa == o.kappa;
  }
};
TableKey g_table_key[kMaxDevices];

fv_status static_fail(fv_status s, const std::string& m) {
  fv::set_last_error(m.c_str());
  return s;
}

// Device address of this device's scratch array, looked up once per device
// with that device current.
fv_status scratch_for_current_device(unsigned char** out, int* dev_out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_fail(FV_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return static_fail(FV_EINVAL, "fv_step_static: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fv_static_scratch);
    if (e != cudaSuccess || !p)
      return static_fail(FV_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  *out = g_scratch_ptr[dev];
  *dev_out = dev;
  return FV_OK;
}

}  // namespace

extern "C" fv_status fv_step_static(const fv_grid* grid, const fv_eos* eos, const int32_t side[4],
                                    const uint8_t* solid, const double* q_in, double* q_out,
                                    double cfl, void* cuda_stream, double* dt_out) {
  if (!grid || !eos || !side || !solid || !q_in || !q_out)
    return static_fail(FV_EINVAL, "fv_step_static: null argument");
  if (grid->nx < 1 || grid->ny < 1 || grid->nx > kMaxNx || grid->ny > kMaxNy)
    return static_fail(FV_EINVAL, "fv_step_static: grid must satisfy 1 <= nx <= " +
                                      std::to_string(kMaxNx) + " and 1 <= ny <= " +
                                      std::to_string(kMaxNy) + " (static scratch size)");
  if (!(grid->dx > 0.0) || !(grid->dy > 0.0)) return static_fail(FV_EINVAL, "fv_step_static: dx, dy must be > 0");
  if (eos->gamma != 1.0 || !(eos->rho0 > 0.0) || !(eos->k0 > 0.0) || !(eos->g >= 0.0) ||
      !(eos->eps_gas > 0.0) || !(eos->eps_gas < 0.1))
    return static_fail(FV_EINVAL, "fv_step_static: invalid equation-of-state parameters");
  for (int s = 0; s < 4; ++s)
    if (side[s] != FV_BC_WALL && side[s] != FV_BC_TRANSMISSIVE)
      return static_fail(FV_EINVAL, "fv_step_static: side must be FV_BC_WALL or FV_BC_TRANSMISSIVE");
  if (!(cfl > 0.0) || !(cfl <= 1.0)) return static_fail(FV_EINVAL, "fv_step_static: cfl must be in (0, 1]");
  if (q_in == q_out) return static_fail(FV_EINVAL, "fv_step_static: q_in and q_out must not alias");

  int dev = 0;
  unsigned char* base = nullptr;
  fv_status st = scratch_for_current_device(&base, &dev);
  if (st != FV_OK) return st;
  DevScalars* sc = (DevScalars*)(base + kOffScalars);
  unsigned long long* colsum = (unsigned long long*)(base + kOffColsum);
  int32_t* Kref = (int32_t*)(base + kOffK);
  int32_t* Kcur = Kref + kMaxNx;
  double* rhoE = (double*)(base + kOffRhoE);

  cudaStream_t stream = (cudaStream_t)cuda_stream;
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
  p.cfl = cfl;

  // The array keeps the previous call's contents: reset what accumulates.
  cudaError_t e = cudaMemsetAsync(sc, 0, sizeof(DevScalars), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(colsum, 0, sizeof(unsigned long long) * p.nx, stream);
  if (e != cudaSuccess) return static_fail(FV_ECUDA, std::string("fv_step_static: ") + cudaGetErrorString(e));
  {
    std::lock_guard<std::mutex> lock(g_table_mutex);
    TableKey key;
    key.ny = p.ny;
    key.dy = p.dy;
    key.rho0 = p.rho0;
    key.kappa = p.kappa;
    if (!(key == g_table_key[dev])) {
      for (long h2 = -2L * p.ny; h2 <= 2L * p.ny; ++h2)
        g_host_table[h2 + 2L * p.ny] = p.rho0 * std::exp(-p.kappa * (0.5 * (double)h2) * p.dy);
      // pageable source: the copy has consumed the buffer when the call returns
      e = cudaMemcpyAsync(rhoE, g_host_table, sizeof(double) * (4 * (size_t)p.ny + 1),
                          cudaMemcpyHostToDevice, stream);
      g_table_key[dev] = e == cudaSuccess ? key : TableKey{};
    }
  }
  if (e != cudaSuccess) return static_fail(FV_ECUDA, std::string("fv_step_static: ") + cudaGetErrorString(e));
  // Levels and signal rate of q_in (Eq. (Free_surf_detector), CFL), then the step.
  launch_prologue_f64(p, q_in, solid, colsum, sc, stream, 2);
  launch_finalize(p, Kref, Kcur, colsum, sc, 0, stream);
  launch_prepare(cfl, sc, stream);
  Tables tb{rhoE, nullptr};
  StateF64 s{q_in, q_out};
  launch_step_f64(p, s, solid, Kcur, colsum, sc, tb, stream);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(FV_ECUDA, std::string("fv_step_static: ") + cudaGetErrorString(e));
  if (dt_out) {
    DevScalars h;
    e = cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return static_fail(FV_ECUDA, std::string("fv_step_static: ") + cudaGetErrorString(e));
    *dt_out = h.dt_cur;
    if (h.status & 2)
      return static_fail(FV_EINVAL, "fv_step_static: q_in has a fluid cell with alpha <= 0, "
                                    "alpha*rho <= 0 or a non-finite value");
    if (h.status & 1)
      return static_fail(FV_ENONFINITE, "fv_step_static: the step produced a non-admissible state");
  }
  return FV_OK;
}
