// fei_peaks.cu -- measured peaks of the CUDA-core pipes that bound the
// CUDA-core paths: FP64 FMA (the plain FP64 path and the FP64 Jacobian work
// of every path), FP32 FMA and packed FP32x2 FMA (the FP32 contraction and
// the operand production of the tensor-core path).  A roofline fraction is
// only as good as its denominator, so these are measured on the part rather
// than derived from unit counts and clocks.
//
// Each thread runs NCH independent multiply-add chains in registers (enough
// to cover the pipe latency with a few warps per scheduler) for `iters`
// rounds; the result is folded into one store per thread so that nothing is
// optimised away.  The caller times a launch with CUDA events and counts
// 2 * NCH * iters * threads flops (4 per lane and step for the packed form).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int NCH = 8;

__global__ void __launch_bounds__(256) fma64_probe(double *out, int iters, double a, double b) {
  double x[NCH];
#pragma unroll
  for (int k = 0; k < NCH; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < NCH; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < NCH; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma32_probe(float *out, int iters, float a, float b) {
  float x[NCH];
#pragma unroll
  for (int k = 0; k < NCH; ++k) x[k] = 1.0f + 1e-3f * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < NCH; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < NCH; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma32x2_probe(float *out, int iters, float a, float b) {
  float2 x[NCH];
#pragma unroll
  for (int k = 0; k < NCH; ++k) x[k] = make_float2(1.0f + 1e-3f * (threadIdx.x + k), 1.0f - 1e-3f * k);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < NCH; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < NCH; ++k) s += x[k].x + x[k].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// kind 0: FP64 FMA, 1: FP32 FMA, 2: packed FP32x2 FMA.  out: device buffer
// of blocks * 256 elements of the kind's type (8 bytes suffice for both).
// Returns the flops the launch performs, or -1 for a bad argument or a
// failed launch.
extern "C" double fei_peak_probe_launch(int kind, int blocks, int iters, void *out, void *stream) {
  if (blocks < 1 || iters < 1 || !out) return -1.0;
  cudaStream_t s = (cudaStream_t)stream;
  const double threads = (double)blocks * 256.0;
  double flops = 0.0;
  switch (kind) {
    case 0:
      fma64_probe<<<blocks, 256, 0, s>>>((double *)out, iters, 0.999999, 1e-7);
      flops = 2.0 * NCH * iters * threads;
      break;
    case 1:
      fma32_probe<<<blocks, 256, 0, s>>>((float *)out, iters, 0.9999f, 1e-4f);
      flops = 2.0 * NCH * iters * threads;
      break;
    case 2:
      fma32x2_probe<<<blocks, 256, 0, s>>>((float *)out, iters, 0.9999f, 1e-4f);
      flops = 4.0 * NCH * iters * threads;
      break;
    default:
      return -1.0;
  }
  return cudaGetLastError() == cudaSuccess ? flops : -1.0;
}
