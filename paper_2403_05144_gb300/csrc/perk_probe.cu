// FP64 throughput microbenchmarks: the denominators of the FP64-pipe roofline.
#include <cuda_runtime.h>
#include <math.h>

#include "perk.h"

namespace {

__global__ void k_fma(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = threadIdx.x * 1e-3 + q;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_div(double* out, int iters, double a) {
  double x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) x[q] = 1.0 + threadIdx.x * 1e-3 + q;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = a / x[q] + 1.0;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3];
}

__global__ void k_log(double* out, int iters) {
  double x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) x[q] = 1.5 + threadIdx.x * 1e-3 + q;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = log(x[q]) + 2.0;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3];
}

}  // namespace

extern "C" perk_status perk_measure_fp64(double* fma_flops, double* div_per_s, double* log_per_s) {
  if (!fma_flops || !div_per_s || !log_per_s) return PERK_E_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PERK_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PERK_E_CUDA;
  const int threads = 256, blocks = sms * 8;
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * blocks * threads) != cudaSuccess) return PERK_E_OOM;
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  double best_fma = 0.0, best_div = 0.0, best_log = 0.0;
  k_fma<<<blocks, threads, 0, st>>>(d, 200, 1.0000001, 1e-9);  // warm-up
  for (int rep = 0; rep < 2; ++rep) {
    const int it_fma = 8000, it_div = 1000, it_log = 500;
    cudaEventRecord(e0, st);
    k_fma<<<blocks, threads, 0, st>>>(d, it_fma, 1.0000001, 1e-9);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    best_fma = fmax(best_fma, 2.0 * 8.0 * it_fma * (double)blocks * threads / (ms * 1e-3));
    cudaEventRecord(e0, st);
    k_div<<<blocks, threads, 0, st>>>(d, it_div, 0.7);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    best_div = fmax(best_div, 4.0 * it_div * (double)blocks * threads / (ms * 1e-3));
    cudaEventRecord(e0, st);
    k_log<<<blocks, threads, 0, st>>>(d, it_log);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    best_log = fmax(best_log, 4.0 * it_log * (double)blocks * threads / (ms * 1e-3));
  }
  const cudaError_t err = cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  cudaFree(d);
  if (err != cudaSuccess) return PERK_E_CUDA;
  *fma_flops = best_fma;
  *div_per_s = best_div;
  *log_per_s = best_log;
  return PERK_OK;
}
