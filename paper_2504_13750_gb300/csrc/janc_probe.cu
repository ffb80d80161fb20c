// Diagnostics: a measured FP64 peak for roofline fractions, and an accuracy
// check of the library's reciprocal against IEEE division.
#include <cmath>
#include <cstring>

#include "../../include/janc.h"
#include "janc_device.cuh"

using namespace janc;

namespace {

// Eight independent DFMA chains per thread; the result is stored so the
// loop cannot be removed.
__global__ void k_dfma_chains(double* out, int n_iter, double s) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double a0 = 1.0 + tid * 1e-9, a1 = a0 + 0.1, a2 = a0 + 0.2, a3 = a0 + 0.3;
  double a4 = a0 + 0.4, a5 = a0 + 0.5, a6 = a0 + 0.6, a7 = a0 + 0.7;
  for (int i = 0; i < n_iter; ++i) {
    a0 = fma(a0, s, 0.5); a1 = fma(a1, s, 0.5); a2 = fma(a2, s, 0.5); a3 = fma(a3, s, 0.5);
    a4 = fma(a4, s, 0.5); a5 = fma(a5, s, 0.5); a6 = fma(a6, s, 0.5); a7 = fma(a7, s, 0.5);
  }
  out[tid] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

__global__ void k_rcp_check(const double* __restrict__ x, int n, unsigned long long* max_ulp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double r = rcp(x[i]);
  const double q = 1.0 / x[i];
  long long a = __double_as_longlong(r), b = __double_as_longlong(q);
  unsigned long long d = (unsigned long long)(a > b ? a - b : b - a);
  atomicMax(max_ulp, d);
}

__global__ void k_exp_check(const double* __restrict__ x, int n, unsigned long long* max_ulp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double r = exp_t(x[i]);
  const double q = exp(x[i]);
  long long a = __double_as_longlong(r), b = __double_as_longlong(q);
  unsigned long long d = (unsigned long long)(a > b ? a - b : b - a);
  atomicMax(max_ulp, d);
}

}  // namespace

extern "C" {

int janc_fp64_peak(void* cuda_stream, int n_iter, double* dfma_per_s) {
  if (!dfma_per_s || n_iter <= 0) return JANC_E_INVALID;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return JANC_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return JANC_E_CUDA;
  const int threads = 256, blocks = sms * 8;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * threads * blocks) != cudaSuccess) return JANC_E_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_dfma_chains<<<blocks, threads, 0, st>>>(out, n_iter / 10 + 1, 0.9999999);
  cudaEventRecord(e0, st);
  k_dfma_chains<<<blocks, threads, 0, st>>>(out, n_iter, 0.9999999);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return JANC_E_CUDA;
  *dfma_per_s = (double)blocks * threads * 8.0 * n_iter / (ms * 1e-3);
  return JANC_OK;
}

static int run_check(const double* x_host, int n, long long* max_ulp, bool is_exp) {
  if (!x_host || n <= 0 || !max_ulp) return JANC_E_INVALID;
  double* dx = nullptr;
  unsigned long long* dm = nullptr;
  if (cudaMalloc(&dx, sizeof(double) * n) != cudaSuccess) return JANC_E_NOMEM;
  if (cudaMalloc(&dm, sizeof(unsigned long long)) != cudaSuccess) { cudaFree(dx); return JANC_E_NOMEM; }
  cudaError_t e = cudaMemcpy(dx, x_host, sizeof(double) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(dm, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) {
    if (is_exp) k_exp_check<<<(n + 255) / 256, 256>>>(dx, n, dm);
    else k_rcp_check<<<(n + 255) / 256, 256>>>(dx, n, dm);
    e = cudaGetLastError();
  }
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, dm, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dm);
  if (e != cudaSuccess) return JANC_E_CUDA;
  *max_ulp = (long long)h;
  return JANC_OK;
}

int janc_selfcheck_exp(const double* x_host, int n, long long* max_ulp) {
  return run_check(x_host, n, max_ulp, true);
}

int janc_selfcheck_rcp(const double* x_host, int n, long long* max_ulp) {
  return run_check(x_host, n, max_ulp, false);
}

}  // extern "C"
