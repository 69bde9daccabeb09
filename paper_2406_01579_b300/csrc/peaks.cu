// ALU peak microbenchmarks for the roofline of the blend kernels (which are
// bound by FP32 arithmetic and by the special-function unit, not by a dense
// contraction or by HBM).  Built as libtets_peaks.so beside libtets.so; the
// benchmark times these launches with CUDA events and divides the operation
// counts they report by the time.
//
//   tts_peak_fma   FP32 fused multiply-adds: every thread runs NCH
//                  independent dependency chains x = fma(x, a, b), unrolled,
//                  so each warp scheduler always has independent FMAs to
//                  issue.  2 flop per FMA.
//   tts_peak_mufu  special-function-unit operations: NCH independent chains
//                  of ex2.approx (kind 0: x = 2^(-x), which stays in [0.5, 1])
//                  or rcp.approx (kind 1: x = 1 / x + 0.5, one FP32 add per
//                  reciprocal, x near 1.28), the two MUFU operations the blend
//                  kernels use
//                  (Eq. 1's exponentials and the reciprocals of the chord and
//                  the backward's 1 / (1 - alpha)).
//
// Both take the launch shape from the caller (blocks x threads, iterations)
// and write one float per thread so that no chain is dead code.  *ops
// receives the operations the launch performs.
#include <cstdint>

#include <cuda_runtime.h>

namespace {

constexpr int NCH = 8;        // independent chains per thread
constexpr int UNROLL = 16;    // chain steps per loop iteration

__global__ void k_peak_fma(float* __restrict__ out, int iters, float a, float b) {
  float x[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) x[c] = 1e-3f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
      for (int c = 0; c < NCH; ++c) x[c] = __fmaf_rn(x[c], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < NCH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_neg(float x) {
  float r;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-x));
  return r;
}

__device__ __forceinline__ float rcp(float x) {
  float r;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <int KIND>
__global__ void k_peak_mufu(float* __restrict__ out, int iters) {
  float x[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) x[c] = 0.5f + 1e-4f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
      for (int c = 0; c < NCH; ++c) x[c] = (KIND == 0) ? ex2_neg(x[c]) : __fadd_rn(rcp(x[c]), 0.5f);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < NCH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One launch; its own launch status (an error pending from earlier calls is
// neither reported nor cleared).
template <typename... KArgs, typename... Args>
cudaError_t launch(void (*kernel)(KArgs...), int blocks, int threads, void* stream,
                   Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.stream = static_cast<cudaStream_t>(stream);
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

extern "C" {

// out: device float[blocks * threads].  Returns 0, or 1 on a bad argument
// or a failed launch.
int tts_peak_fma(int blocks, int threads, int iters, float* out, double* ops, void* stream) {
  if (blocks < 1 || threads < 32 || threads > 1024 || iters < 1 || !out || !ops) return 1;
  *ops = 2.0 * (double)blocks * threads * iters * UNROLL * NCH;   // flop
  return launch(k_peak_fma, blocks, threads, stream, out, iters, 0.999999f, 1e-7f) == cudaSuccess
             ? 0 : 1;
}

int tts_peak_mufu(int kind, int blocks, int threads, int iters, float* out, double* ops,
                  void* stream) {
  if (kind < 0 || kind > 1 || blocks < 1 || threads < 32 || threads > 1024 || iters < 1 || !out ||
      !ops)
    return 1;
  *ops = (double)blocks * threads * iters * UNROLL * NCH;
  const cudaError_t e = (kind == 0) ? launch(k_peak_mufu<0>, blocks, threads, stream, out, iters)
                                    : launch(k_peak_mufu<1>, blocks, threads, stream, out, iters);
  return e == cudaSuccess ? 0 : 1;
}

}  // extern "C"
