// Arithmetic-throughput loops: the denominators of the roofline fractions that
// the benchmark reports for the dynamics kernels. Every thread runs 8
// independent multiply-add chains on registers (no memory traffic inside the
// loop), so the issue rate of the multiply-add pipe is the only limit.
#include <cuda_runtime.h>

#include "grid_internal.h"

namespace {

constexpr int kChains = 8;

__global__ void peak_ffma(int iters, float b, float c, float* out) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = b * (float)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Paired form: one instruction performs two independent FP32 multiply-adds.
__global__ void peak_ffma2(int iters, float b, float c, float* out) {
  float2 a[kChains];
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = make_float2(b * (float)(threadIdx.x + k), b * (float)(k + 1));
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b2, c2);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void peak_dfma(int iters, double b, double c, double* out) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = b * (double)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" grid_status grid_peak_loop(int kind, int blocks, int threads, int iters, void* out, double* flops,
                                      void* stream) {
  if (kind < 0 || kind > 2 || blocks < 1 || threads < 32 || threads > 1024 || threads % 32 || iters < 1 || !out ||
      !flops) {
    grid_set_error("grid_peak_loop: bad argument");
    return GRID_E_ARG;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // b slightly below 1 and c small keep every chain bounded for any length
  if (kind == 0) peak_ffma<<<blocks, threads, 0, st>>>(iters, 0.999f, 1e-3f, static_cast<float*>(out));
  else if (kind == 1) peak_ffma2<<<blocks, threads, 0, st>>>(iters, 0.999f, 1e-3f, static_cast<float*>(out));
  else peak_dfma<<<blocks, threads, 0, st>>>(iters, 0.999, 1e-3, static_cast<double*>(out));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    grid_set_error("grid_peak_loop: launch: %s", cudaGetErrorString(e));
    return GRID_E_CUDA;
  }
  *flops = 2.0 * (double)blocks * threads * (double)iters * kChains * (kind == 1 ? 2 : 1);
  return GRID_OK;
}
