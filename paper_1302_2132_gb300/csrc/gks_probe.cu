// Throughput probe of the FP32 and FP64 FMA pipes (independent FMA chains, every SM busy); context
// for the ALU roofline of the step kernel.  Reads and writes only its own small buffers.
#include <cuda_runtime.h>

#include "gks.h"

namespace {

constexpr int kIters = 4096;

__global__ void fma32_kernel(float* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1.0f + 1e-9f * (float)(i + k);
  const float m = 0.999999f, c = 1e-7f;
#pragma unroll 16
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[i] = s;
}

__global__ void fma64_kernel(double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = 1.0 + 1e-12 * (double)(i + k);
  const double m = 0.9999999, c = 1e-9;
#pragma unroll 16
  for (int it = 0; it < kIters / 8; ++it)
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = fma(a[k], m, c);
  out[i] = a[0] + a[1] + a[2] + a[3];
}

// The same chains with the paired single-precision FMA (two lanes' worth of FMA per thread
// instruction, sm_100 and later): shows whether pairing raises the FP32 rate or only saves issue slots.
__global__ void fma32x2_kernel(float* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float2 a[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = make_float2(1.0f + 1e-9f * (float)(i + 2 * k), 1.0f + 1e-9f * (float)(i + 2 * k + 1));
  const float2 m = make_float2(0.999999f, 0.999999f), c = make_float2(1e-7f, 1e-7f);
#pragma unroll 16
  for (int it = 0; it < kIters; ++it)
#pragma unroll
    for (int k = 0; k < 4; ++k) a[k] = __ffma2_rn(a[k], m, c);
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k) s += a[k].x + a[k].y;
  out[i] = s;
}

// Conversion throughput between double and float: independent chains per thread, each iteration one
// conversion plus two or three integer or FP32 operations on the full-rate pipes that keep the
// chains dependent (the conversion rate binds when it is well below the FP32 rate).
__global__ void cvt_d2f_kernel(float* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d[8];
  float acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    d[k] = 1.0 + 1e-9 * (double)(i + k);
    acc[k] = 0.0f;
  }
#pragma unroll 8
  for (int it = 0; it < kIters / 4; ++it)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      acc[k] += __double2float_rn(d[k]);
      d[k] = __longlong_as_double(__double_as_longlong(d[k]) + 1);
    }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += acc[k];
  out[i] = s;
}

__global__ void cvt_f2d_kernel(float* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float f[8];
  unsigned long long acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    f[k] = 1.0f + 1e-6f * (float)(i + k);
    acc[k] = 0ull;
  }
#pragma unroll 8
  for (int it = 0; it < kIters / 4; ++it)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      acc[k] ^= (unsigned long long)__double_as_longlong((double)f[k]);
      f[k] = __int_as_float(__float_as_int(f[k]) + 1);
    }
  unsigned long long s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= acc[k];
  out[i] = (float)(s & 0xffff);
}

}  // namespace

// Conversions per second (in units of 1e9) of double -> float and float -> double, measured as
// gks_probe_alu measures the FMA pipes: context for the double-state form of the step kernel.
extern "C" gks_status gks_probe_cvt(double* d2f_gops, double* f2d_gops) {
  int dev;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return GKS_ECUDA;
  const int threads = 256, blocks = p.multiProcessorCount * 8, n = threads * blocks;
  void* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)n * sizeof(float)) != cudaSuccess) return GKS_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.0f;
  cvt_d2f_kernel<<<blocks, threads>>>((float*)buf, n);
  cudaEventRecord(e0);
  cvt_d2f_kernel<<<blocks, threads>>>((float*)buf, n);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  if (d2f_gops) *d2f_gops = 8.0 * (kIters / 4) * (double)n / (ms * 1e-3) / 1e9;
  cvt_f2d_kernel<<<blocks, threads>>>((float*)buf, n);
  cudaEventRecord(e0);
  cvt_f2d_kernel<<<blocks, threads>>>((float*)buf, n);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  if (f2d_gops) *f2d_gops = 8.0 * (kIters / 4) * (double)n / (ms * 1e-3) / 1e9;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaGetLastError();
  cudaFree(buf);
  return e == cudaSuccess ? GKS_OK : GKS_ECUDA;
}

extern "C" gks_status gks_probe_alu_packed(double* fp32x2_tflops) {
  int dev;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return GKS_ECUDA;
  const int threads = 256, blocks = p.multiProcessorCount * 8, n = threads * blocks;
  void* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)n * sizeof(float)) != cudaSuccess) return GKS_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.0f;
  fma32x2_kernel<<<blocks, threads>>>((float*)buf, n);
  cudaEventRecord(e0);
  fma32x2_kernel<<<blocks, threads>>>((float*)buf, n);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  if (fp32x2_tflops) *fp32x2_tflops = 2.0 * 8.0 * kIters * (double)n / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaGetLastError();
  cudaFree(buf);
  return e == cudaSuccess ? GKS_OK : GKS_ECUDA;
}

extern "C" gks_status gks_probe_alu(double* fp32_tflops, double* fp64_tflops) {
  int dev;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return GKS_ECUDA;
  const int threads = 256, blocks = p.multiProcessorCount * 8, n = threads * blocks;
  void* buf = nullptr;
  if (cudaMalloc(&buf, (size_t)n * sizeof(double)) != cudaSuccess) return GKS_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.0f;
  fma32_kernel<<<blocks, threads>>>((float*)buf, n);
  cudaEventRecord(e0);
  fma32_kernel<<<blocks, threads>>>((float*)buf, n);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  if (fp32_tflops) *fp32_tflops = 2.0 * 8.0 * kIters * (double)n / (ms * 1e-3) / 1e12;
  fma64_kernel<<<blocks, threads>>>((double*)buf, n);
  cudaEventRecord(e0);
  fma64_kernel<<<blocks, threads>>>((double*)buf, n);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  cudaEventElapsedTime(&ms, e0, e1);
  if (fp64_tflops) *fp64_tflops = 2.0 * 4.0 * (kIters / 8) * (double)n / (ms * 1e-3) / 1e12;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaGetLastError();
  cudaFree(buf);
  return e == cudaSuccess ? GKS_OK : GKS_ECUDA;
}
