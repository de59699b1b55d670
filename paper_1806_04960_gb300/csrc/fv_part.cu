// Partitioned domains: one grid split into column strips, each advanced by its
// own handle (on one GPU or one per GPU), with a halo exchange between steps.
//
// The scheme's stencil is nearest-neighbour in faces (Eq. (Scheme)): the update
// of column i reads the x faces i -/+ 1/2, whose states come from the
// reconstructions of columns i-1 .. i+1, which read columns i-2 .. i+2.  A strip
// that owns columns [a, b) of the grid is therefore stepped as a grid of its
// own over [a-2, b+2) (fewer at the grid's own sides): its owned cells come out
// exactly as in the undivided grid, provided that
//   * every column of the strip holds the undivided grid's state and level
//     before the step (the two halo columns on each inner side are copied from
//     the neighbouring strip after every step: fv_part_pack / fv_part_unpack);
//   * dt is the undivided grid's: the largest signal rate over all strips
//     (reading R-cfl; a max is exact in any order), exchanged through
//     fv_part_rate / fv_part_set_rate;
//   * the free-surface levels of Eq. (Free_surf_detector) need no exchange: a
//     level is a sum over one column, and columns are never split.
// The halo columns' own new values are wrong (they see the strip's edge) and
// are excluded from the signal rate and the status (fv_set_partition).
#include <cuda_runtime.h>

#include <string>

#include "fv.h"
#include "fv_handle.cuh"
#include "fv_kernels.cuh"

namespace {

fv_status part_fail(fv_status s, const std::string& m) {
  fv::set_last_error(m.c_str());
  return s;
}

fv_status part_cuda(cudaError_t e, const char* where) {
  return part_fail(FV_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Buffer of one side: the 4 planes of 2 columns (plane-major, then row, then
// column), then Kref and Kcur of those 2 columns.
template <typename T>
__global__ void pack_kernel(const T* __restrict__ q, const int32_t* __restrict__ Kref,
                            const int32_t* __restrict__ Kcur, int nx, int ny, int col0,
                            unsigned char* __restrict__ buf) {
  T* vals = reinterpret_cast<T*>(buf);
  const size_t N = (size_t)nx * ny;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 2 * ny; k += gridDim.x * blockDim.x) {
    const int j = k >> 1, c = k & 1;
    const size_t src = (size_t)j * nx + col0 + c;
#pragma unroll
    for (int v = 0; v < 4; ++v) vals[(size_t)v * 2 * ny + k] = q[v * N + src];
  }
  if (blockIdx.x == 0 && threadIdx.x < 2) {
    int32_t* K = reinterpret_cast<int32_t*>(buf + sizeof(T) * 8 * (size_t)ny);
    K[threadIdx.x] = Kref[col0 + threadIdx.x];
    K[2 + threadIdx.x] = Kcur[col0 + threadIdx.x];
  }
}

template <typename T>
__global__ void unpack_kernel(T* __restrict__ q, int32_t* __restrict__ Kref,
                              int32_t* __restrict__ Kcur, int nx, int ny, int col0,
                              const unsigned char* __restrict__ buf) {
  const T* vals = reinterpret_cast<const T*>(buf);
  const size_t N = (size_t)nx * ny;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 2 * ny; k += gridDim.x * blockDim.x) {
    const int j = k >> 1, c = k & 1;
    const size_t dst = (size_t)j * nx + col0 + c;
#pragma unroll
    for (int v = 0; v < 4; ++v) q[v * N + dst] = vals[(size_t)v * 2 * ny + k];
  }
  if (blockIdx.x == 0 && threadIdx.x < 2) {
    const int32_t* K = reinterpret_cast<const int32_t*>(buf + sizeof(T) * 8 * (size_t)ny);
    Kref[col0 + threadIdx.x] = K[threadIdx.x];
    Kcur[col0 + threadIdx.x] = K[2 + threadIdx.x];
  }
}

// rate_cur = the largest of n rates (max is exact, so the order is immaterial).
__global__ void adopt_max_rate_kernel(const double* __restrict__ rates, int n,
                                      fv::DevScalars* __restrict__ sc) {
  double r = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) r = fmax(r, rates[k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
  if (threadIdx.x == 0) sc->rate_cur = r;
}

size_t halo_bytes(const fv_handle* h) {
  const size_t elem = h->prec == FV_FP64 ? sizeof(double) : sizeof(float);
  return elem * 8 * (size_t)h->grid.ny + 4 * sizeof(int32_t);
}

bool partitioned(const fv_handle* h) { return h->own_hi > 0; }

// First column of the side's packed (own) or unpacked (halo) pair; -1 if that
// side has no neighbour.
int side_column(const fv_handle* h, int side, bool halo) {
  if (side == 0) return h->own_lo == 2 ? (halo ? 0 : 2) : -1;
  return h->grid.nx - h->own_hi == 2 ? (halo ? h->own_hi : h->own_hi - 2) : -1;
}

int grid_for(int ny) {
  int b = (2 * ny + 255) / 256;
  return b > 152 ? 152 : (b < 1 ? 1 : b);
}

}  // namespace

extern "C" {

fv_status fv_set_partition(fv_handle* h, int32_t own_lo, int32_t own_hi) {
  if (!h) return part_fail(FV_EINVAL, "fv_set_partition: null handle");
  if (own_lo == 0 && own_hi == 0) {
    h->own_lo = h->own_hi = 0;
    return FV_OK;
  }
  const int nx = h->grid.nx;
  if ((own_lo != 0 && own_lo != 2) || (nx - own_hi != 0 && nx - own_hi != 2) ||
      own_hi - own_lo < 2)
    return part_fail(FV_EINVAL,
                     "fv_set_partition: own columns must be [0 or 2, nx or nx-2) and at least 2 wide");
  h->own_lo = own_lo;
  h->own_hi = own_hi;
  return FV_OK;
}

fv_status fv_part_halo_bytes(const fv_handle* h, int64_t* bytes) {
  if (!h || !bytes) return part_fail(FV_EINVAL, "fv_part_halo_bytes: null argument");
  *bytes = (int64_t)halo_bytes(h);
  return FV_OK;
}

fv_status fv_part_rate(fv_handle* h, double* rate_dev) {
  if (!h || !rate_dev) return part_fail(FV_EINVAL, "fv_part_rate: null argument");
  if (!h->has_state) return part_fail(FV_EINVAL, "fv_part_rate: no state");
  cudaError_t e = cudaMemcpyAsync(rate_dev, &h->d_sc->rate_cur, sizeof(double),
                                  cudaMemcpyDeviceToDevice, h->stream);
  return e == cudaSuccess ? FV_OK : part_cuda(e, "fv_part_rate");
}

fv_status fv_part_set_rate(fv_handle* h, const double* rates_dev, int32_t n) {
  if (!h || !rates_dev || n < 1)
    return part_fail(FV_EINVAL, "fv_part_set_rate: null argument or n < 1");
  if (!h->has_state) return part_fail(FV_EINVAL, "fv_part_set_rate: no state");
  if (n == 1) {
    cudaError_t e = cudaMemcpyAsync(&h->d_sc->rate_cur, rates_dev, sizeof(double),
                                    cudaMemcpyDeviceToDevice, h->stream);
    return e == cudaSuccess ? FV_OK : part_cuda(e, "fv_part_set_rate");
  }
  adopt_max_rate_kernel<<<1, 32, 0, h->stream>>>(rates_dev, n, h->d_sc);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FV_OK : part_cuda(e, "fv_part_set_rate");
}

fv_status fv_part_pack(fv_handle* h, int32_t side, void* buf_dev) {
  if (!h || !buf_dev || (side != 0 && side != 1))
    return part_fail(FV_EINVAL, "fv_part_pack: null argument or side not 0 (W) / 1 (E)");
  if (!h->has_state || !partitioned(h)) return part_fail(FV_EINVAL, "fv_part_pack: no state or no partition");
  const int c0 = side_column(h, side, false);
  if (c0 < 0) return part_fail(FV_EINVAL, "fv_part_pack: that side has no neighbouring strip");
  const int nx = h->grid.nx, ny = h->grid.ny;
  if (h->prec == FV_FP64)
    pack_kernel<double><<<grid_for(ny), 256, 0, h->stream>>>(
        (const double*)h->d_q[h->cur], h->d_Kref, h->d_Kcur, nx, ny, c0, (unsigned char*)buf_dev);
  else
    pack_kernel<float><<<grid_for(ny), 256, 0, h->stream>>>(
        (const float*)h->d_q[h->cur], h->d_Kref, h->d_Kcur, nx, ny, c0, (unsigned char*)buf_dev);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FV_OK : part_cuda(e, "fv_part_pack");
}

fv_status fv_part_unpack(fv_handle* h, int32_t side, const void* buf_dev) {
  if (!h || !buf_dev || (side != 0 && side != 1))
    return part_fail(FV_EINVAL, "fv_part_unpack: null argument or side not 0 (W) / 1 (E)");
  if (!h->has_state || !partitioned(h)) return part_fail(FV_EINVAL, "fv_part_unpack: no state or no partition");
  const int c0 = side_column(h, side, true);
  if (c0 < 0) return part_fail(FV_EINVAL, "fv_part_unpack: that side has no neighbouring strip");
  const int nx = h->grid.nx, ny = h->grid.ny;
  if (h->prec == FV_FP64)
    unpack_kernel<double><<<grid_for(ny), 256, 0, h->stream>>>(
        (double*)h->d_q[h->cur], h->d_Kref, h->d_Kcur, nx, ny, c0, (const unsigned char*)buf_dev);
  else
    unpack_kernel<float><<<grid_for(ny), 256, 0, h->stream>>>(
        (float*)h->d_q[h->cur], h->d_Kref, h->d_Kcur, nx, ny, c0, (const unsigned char*)buf_dev);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FV_OK : part_cuda(e, "fv_part_unpack");
}

}  // extern "C"
