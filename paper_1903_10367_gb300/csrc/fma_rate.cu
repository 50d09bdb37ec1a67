// Measures the device's FP64 and FP32 fused multiply-add rates: a stand-alone
// program (not part of the library) whose figures bound what any FP64
// implementation of the cycle can reach on this GPU.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fma_rate fma_rate.cu
//   ./fma_rate
//
// 8 resident blocks of 256 threads per SM, each thread running 8 independent
// FMA chains; the kernels touch memory only to keep the result alive.
#include <cstdio>

#include <cuda_runtime.h>

template <typename T>
__global__ void k_fma(T* out, int iters, T a, T c) {
  T x[8];
  for (int j = 0; j < 8; ++j) x[j] = (T)threadIdx.x * (T)1e-3 + (T)j;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = x[j] * a + c;
  T s = 0;
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == (T)12345.678) out[0] = s;  // never true: keeps the chains alive
}

template <typename T>
double rate(T* out, int blocks, int iters) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  k_fma<T><<<blocks, 256>>>(out, iters, (T)0.999999, (T)1e-9);
  cudaEventRecord(a);
  k_fma<T><<<blocks, 256>>>(out, iters, (T)0.999999, (T)1e-9);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return (double)blocks * 256 * iters * 8 / (ms * 1e-3);
}

int main() {
  double* d = nullptr;
  float* f = nullptr;
  int sms = 0;
  if (cudaMalloc(&d, sizeof(double)) != cudaSuccess || cudaMalloc(&f, sizeof(float)) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess)
    return 1;
  double best64 = 0.0, best32 = 0.0;
  for (int rep = 0; rep < 3; ++rep) {
    const double r64 = rate(d, sms * 8, 4096), r32 = rate(f, sms * 8, 65536);
    best64 = r64 > best64 ? r64 : best64;
    best32 = r32 > best32 ? r32 : best32;
  }
  printf("{\"sms\": %d, \"fp64_fma_per_s\": %.4g, \"fp32_fma_per_s\": %.4g, \"ratio\": %.1f}\n", sms,
         best64, best32, best32 / best64);
  cudaFree(d);
  cudaFree(f);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
