// Issue-rate microbenchmarks for the roofline of the interpreter kernels:
// long chains of independent FP32 fused multiply-adds (scalar FFMA and the
// packed two-row FFMA2 of sm_100 and later) and of SFU instructions
// (reciprocal square root, base-2 exponential and logarithm, sine), with
// enough independent chains per thread and enough warps per SM that the
// pipe, not latency, bounds them.  The benchmark divides the operations by
// the time and by the SM clock it samples, giving FP32 and SFU operations
// per SM per clock: the denominators of the algorithmic roofline.
#include <cuda_runtime.h>

#include <cstdio>

#include "ggeval.h"

namespace {

constexpr int CHAINS = 8;  // independent chains per thread

template <int K>
__device__ __forceinline__ float sfu_op(float x) {
  float r;
  if constexpr (K == 0) asm volatile("rsqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  if constexpr (K == 1) asm volatile("ex2.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  if constexpr (K == 2) asm volatile("lg2.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  if constexpr (K == 3) asm volatile("sin.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// kind 0: scalar FFMA, 1: packed FFMA2, 2..5: SFU (rsqrt, ex2, lg2, sin).
// Every operation's result feeds the next one of its chain; the sums are
// written so that nothing is dead code.
template <int KIND>
__global__ void __launch_bounds__(256) pipe_kernel(int iters, float seed, float* out) {
  constexpr int kind = KIND;
  float v[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) v[c] = seed + 1e-3f * (threadIdx.x + c);
  if constexpr (kind == 0) {
    const float m = 0.999999f, a = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) v[c] = fmaf(v[c], m, a);
    }
  } else if constexpr (kind == 1) {
    float2 w[CHAINS / 2];
#pragma unroll
    for (int c = 0; c < CHAINS / 2; ++c) w[c] = make_float2(v[2 * c], v[2 * c + 1]);
    const float2 m = make_float2(0.999999f, 0.999999f), a = make_float2(1e-7f, 1e-7f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < CHAINS / 2; ++c) w[c] = __ffma2_rn(w[c], m, a);
    }
#pragma unroll
    for (int c = 0; c < CHAINS / 2; ++c) {
      v[2 * c] = w[c].x;
      v[2 * c + 1] = w[c].y;
    }
  } else {
    // each chain stays finite: 2^-|v| lies in (0, 1], log2(1 + |v|) tends
    // to 1, rsqrt(v) to 1 and sin(v) to 0 (the one FP32 operation next to
    // each SFU operation costs nothing against the narrower SFU pipe)
    constexpr int k = kind - 2;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) {
        const float x = k == 1 ? -fabsf(v[c]) : k == 2 ? 1.0f + fabsf(v[c]) : v[c];
        v[c] = sfu_op<k>(x);
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += v[c];
  if (s == 12345.678f) out[blockIdx.x] = s;  // never true; keeps the chains live
}

}  // namespace

extern "C" ggeval_status ggeval_pipe_rates(int32_t device, int32_t iters, double* ops_per_s) {
  if (!ops_per_s || iters < 1) return GGEVAL_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return GGEVAL_ERR_ARG;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ggeval_status st = GGEVAL_OK;
  const int blocks = sms * 8, threads = 256;  // 64 warps per SM
  if (cudaMalloc(&out, sizeof(float) * blocks) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = GGEVAL_ERR_CUDA;
  }
  void (*kernels[6])(int, float, float*) = {pipe_kernel<0>, pipe_kernel<1>, pipe_kernel<2>,
                                            pipe_kernel<3>, pipe_kernel<4>, pipe_kernel<5>};
  for (int kind = 0; kind < 6 && st == GGEVAL_OK; ++kind) {
    // SFU chains run 8x fewer iterations (the pipe is narrower)
    const int it = kind >= 2 ? (iters + 7) / 8 : iters;
    kernels[kind]<<<blocks, threads>>>(it, 0.5f, out);  // warm-up
    cudaEventRecord(e0);
    kernels[kind]<<<blocks, threads>>>(it, 0.5f, out);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = GGEVAL_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double ops = (double)blocks * threads * it * CHAINS;  // an FFMA2 does 2
    ops_per_s[kind] = ops / (ms * 1e-3);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}
