// Measured fused multiply-add throughput of the device for FP32 or FP64: the denominator
// of the arithmetic rooflines (the paper has no counterpart; a measurement aid).
//
// Every thread runs kChains independent FMA chains x <- x a + b for `iters` iterations with
// no memory access inside the loop, 8 CTAs of 256 threads per SM, so the FMA pipe of the
// type is the only unit kept busy.  With 0 < a < 1 the chains converge to b / (1 - a) and
// stay finite; each thread stores its sum once, so the work cannot be removed.
#include <cuda_runtime.h>

#include "../../include/ppml.h"
#include "ppml_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_peak_kernel(int iters, T a, T b,
                                                            T* __restrict__ out) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) x[k] = T(threadIdx.x + k) * T(1e-3);
#pragma unroll 4
  for (int i = 0; i < iters; i++)
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; k++) s += x[k];
  out[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

template <typename T>
int run_peak(int iters, double* fma_per_s, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8;
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * kThreads) != cudaSuccess) {
    cudaGetLastError();
    return ppml_fail(PPML_E_NOMEM, "FMA peak scratch");
  }
  int rc = PPML_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = ppml_fail(PPML_E_CUDA, "FMA peak events");
  } else {
    const T a = T(0.999), b = T(1e-3);
    fma_peak_kernel<T><<<blocks, kThreads, 0, st>>>(iters, a, b, out);  // warm-up
    rc = ppml_check_launch("fma_peak_kernel");
    if (!rc) {
      cudaEventRecord(e0, st);
      fma_peak_kernel<T><<<blocks, kThreads, 0, st>>>(iters, a, b, out);
      cudaEventRecord(e1, st);
      rc = ppml_check_launch("fma_peak_kernel");
    }
    float ms = 0.f;
    if (!rc && (cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)))
      rc = ppml_fail(PPML_E_CUDA, "FMA peak timing: %s", cudaGetErrorString(cudaGetLastError()));
    if (!rc)
      *fma_per_s = (double)blocks * kThreads * kChains * (double)iters / (ms * 1e-3);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

}  // namespace

extern "C" int ppml_fma_peak(int dtype, int iters, double* fma_per_s, void* stream) {
  if (!fma_per_s) return ppml_fail(PPML_E_INVAL, "fma_per_s is NULL");
  if (iters < 1) return ppml_fail(PPML_E_INVAL, "iters = %d must be >= 1", iters);
  const cudaStream_t st = (cudaStream_t)stream;
  if (dtype == PPML_F32) return run_peak<float>(iters, fma_per_s, st);
  if (dtype == PPML_F64) return run_peak<double>(iters, fma_per_s, st);
  return ppml_fail(PPML_E_INVAL, "bad dtype %d", dtype);
}
