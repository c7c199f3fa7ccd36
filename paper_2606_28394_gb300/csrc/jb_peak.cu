// FP32 fused multiply-add rate of the GPU: the denominator of the physics
// kernel's roofline (the step is bound by FP32 issue, not by HBM or tensor
// cores).  Every thread runs kChains independent multiply-add chains for
// `iters` rounds, scalar (FFMA) or packed (FFMA2 on float2, two lanes of
// arithmetic per instruction), and stores one value so the work is live.
#include <cuda_runtime.h>

#include "jb_internal.cuh"

namespace {
constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_rate_scalar(float* __restrict__ sink, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  sink[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma_rate_packed(float* __restrict__ sink, int iters, float a, float b) {
  float2 x[kChains];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = make_float2((float)(threadIdx.x + k), (float)(threadIdx.x - k));
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k].x + x[k].y;
  sink[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
}
}  // namespace

extern "C" {

double jb_fma_probe_flops(int32_t packed, int32_t blocks, int32_t iters) {
  if (blocks <= 0 || iters <= 0) return 0.0;
  return 2.0 * kChains * (packed ? 2.0 : 1.0) * (double)kThreads * (double)blocks * (double)iters;
}

jb_status jb_fma_probe(int32_t packed, int32_t blocks, int32_t iters, float* d_sink, void* cuda_stream) {
  if (!d_sink || blocks <= 0 || iters <= 0) return jbk::fail(JB_EINVAL, "jb_fma_probe: bad arguments");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // a, b keep the chains bounded (x -> b / (1 - a)) and unknown to the compiler
  const float a = 0.999f, b = 1e-3f;
  if (packed) fma_rate_packed<<<blocks, kThreads, 0, s>>>(d_sink, iters, a, b);
  else fma_rate_scalar<<<blocks, kThreads, 0, s>>>(d_sink, iters, a, b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return jbk::fail(JB_ECUDA, "jb_fma_probe launch: %s", cudaGetErrorString(e));
  return JB_OK;
}

}  // extern "C"
