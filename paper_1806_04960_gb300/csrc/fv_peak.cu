// Measured peak of the plain floating-point pipes the step kernels run on:
// fused multiply-add throughput in FP32 (scalar FFMA and the paired FFMA2 of
// sm_100 and later) and FP64 (DFMA) on the current device.  The roofline of a
// step kernel that is not a tensor contraction is this rate, not a tensor-core
// one; the benchmark measures it in the same run as the kernels it rates.
//
// Each thread advances CHAINS independent recurrences a <- a * b + c (b < 1,
// so the values settle and never overflow or reach subnormals), unrolled so
// that loop control is a few percent of the issued instructions; 8 CTAs of
// 256 threads per SM keep every scheduler supplied.  Flops = 2 per FMA lane.
#include <cuda_runtime.h>

#include <string>

#include "fv.h"
#include "fv_kernels.cuh"
#include "fv_model.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_peak_kernel(T* out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  // never true for these recurrences; keeps the chains live
  if (s == T(-1)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) ffma2_peak_kernel(float* out, int iters, float b,
                                                              float c) {
  float2 a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k)
    a[k] = make_float2(float(threadIdx.x + k) * 1e-3f, float(threadIdx.x + 2 * k) * 1e-3f);
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
  if (s == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

std::string cuda_msg(const char* where, cudaError_t e) {
  return std::string("fv_measure_fma_peak: ") + where + ": " + cudaGetErrorString(e);
}

}  // namespace

extern "C" fv_status fv_measure_fma_peak(int32_t kind, int32_t reps, double* tflops,
                                         double* best_ms) {
  if (kind < 0 || kind > 2 || reps < 1 || !tflops) {
    fv::set_last_error("fv_measure_fma_peak: kind must be 0, 1 or 2, reps >= 1, tflops non-null");
    return FV_EINVAL;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    fv::set_last_error(cuda_msg("device", e).c_str());
    return FV_ECUDA;
  }
  const int blocks = 8 * sms;
  // about 20-40 ms per launch at the expected rates
  const int iters = kind == 2 ? 500 : 30000;
  void* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&out, (size_t)blocks * kThreads * 8);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto launch = [&]() {
    if (kind == 0)
      fma_peak_kernel<float><<<blocks, kThreads, 0, st>>>((float*)out, iters, 0.999f, 1e-3f);
    else if (kind == 1)
      ffma2_peak_kernel<<<blocks, kThreads, 0, st>>>((float*)out, iters, 0.999f, 1e-3f);
    else
      fma_peak_kernel<double><<<blocks, kThreads, 0, st>>>((double*)out, iters, 0.999, 1e-3);
  };
  float best = 1e30f;
  if (e == cudaSuccess) {
    launch();  // warm-up (module load, clocks)
    e = cudaGetLastError();
  }
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, st);
    launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  if (e != cudaSuccess) {
    fv::set_last_error(cuda_msg("launch", e).c_str());
    return FV_ECUDA;
  }
  const double lanes = kind == 1 ? 2.0 : 1.0;
  const double fmas = (double)blocks * kThreads * iters * kUnroll * kChains * lanes;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  if (best_ms) *best_ms = best;
  return FV_OK;
}

namespace {
__global__ void rcp_probe_kernel(const double* __restrict__ x, double* __restrict__ out,
                                 long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    out[k] = fv::rcp(x[k]);
}
}  // namespace

extern "C" fv_status fv_device_rcp(const double* x_dev, double* out_dev, int64_t n,
                                   void* cuda_stream) {
  if (!x_dev || !out_dev || n < 0) {
    fv::set_last_error("fv_device_rcp: null argument or n < 0");
    return FV_EINVAL;
  }
  if (n == 0) return FV_OK;
  const long long blocks = (n + 255) / 256;
  rcp_probe_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0,
                     (cudaStream_t)cuda_stream>>>(x_dev, out_dev, n);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fv::set_last_error(cuda_msg("fv_device_rcp", e).c_str());
    return FV_ECUDA;
  }
  return FV_OK;
}
