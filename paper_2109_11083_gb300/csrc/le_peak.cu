// Arithmetic peak of the CUDA cores in FP32: every thread runs independent
// FMA chains, scalar (fma.rn.f32) or paired (fma.rn.f32x2, the form the pair
// kernel uses), on enough blocks to fill every SM.  It is the denominator of
// the pair kernel's secondary check (FP32 flops per pair x pairs / time): the
// pair kernel is bound by its L1 gathers, and this says how far its
// arithmetic is from being the limit.
#include <cuda_runtime.h>

#include <algorithm>

#include "le.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma(float *out, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)threadIdx.x * 1e-3f + (float)c;
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 1.2345f) out[blockIdx.x] = s;  // keeps the chains live; a and b make it unreachable
}

__global__ void __launch_bounds__(kThreads) k_fma2(float *out, float a, float b) {
  float2 x[kChains];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int c = 0; c < kChains; ++c)
    x[c] = make_float2((float)threadIdx.x * 1e-3f + (float)c, (float)c - 1.f);
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  if (s == 1.2345f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" LE_API le_status le_fp32_peak(double *tflops_fma, double *tflops_fma2) {
  if (!tflops_fma || !tflops_fma2) return LE_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LE_ERR_CUDA;
  const int blocks = sms * 8;
  float *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaMalloc(&out, sizeof(float) * blocks);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  // a = 1 - 2^-20, b = 2^-30: the chains stay finite and never reach 1.2345
  const float a = 0.99999905f, b = 9.3132257e-10f;
  double best[2] = {0.0, 0.0};
  for (int rep = 0; rep < 4 && ce == cudaSuccess; ++rep) {
    for (int kind = 0; kind < 2 && ce == cudaSuccess; ++kind) {
      ce = cudaEventRecord(e0, 0);
      if (kind == 0) k_fma<<<blocks, kThreads>>>(out, a, b);
      else k_fma2<<<blocks, kThreads>>>(out, a, b);
      if (ce == cudaSuccess) ce = cudaGetLastError();
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, 0);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce == cudaSuccess && ms > 0.f && rep > 0) {  // the first round warms up
        const double flops = 2.0 * (kind ? 2.0 : 1.0) * kChains * (double)kIters *
                             (double)blocks * kThreads;
        best[kind] = std::max(best[kind], flops / (ms * 1e-3) * 1e-12);
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (ce != cudaSuccess) return LE_ERR_CUDA;
  *tflops_fma = best[0];
  *tflops_fma2 = best[1];
  return LE_OK;
}
