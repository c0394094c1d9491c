// Arithmetic-pipe microbenchmarks that give the roofline denominators the fit's kernels
// are bounded by: FP32 fused multiply-add (scalar and packed float2), the special-function
// unit's 2^x, and FP64 fused multiply-add. Each thread runs independent dependency chains
// for a fixed iteration count; the result feeds a store so nothing is optimised away.
#include <cuda_runtime.h>

#include "prism.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_ub_ffma(float* out, int iters) {
  float x[kChains];
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
  const float a = 0.999f, b = 1e-3f;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  float s = 0.f;
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_ub_ffma2(float* out, int iters) {
  float2 x[kChains];
  for (int c = 0; c < kChains; ++c) x[c] = make_float2(threadIdx.x * 1e-3f + c, c * 0.5f);
  const float2 a = make_float2(0.999f, 0.998f), b = make_float2(1e-3f, 2e-3f);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a, b);
  float s = 0.f;
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  if (s == 12345.f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_ub_ex2(float* out, int iters) {
  float x[kChains];
  for (int c = 0; c < kChains; ++c) x[c] = -1e-3f * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      float y;
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
      x[c] = y - 1.0f;   // stays in (-1, 0]: one extra FADD per 2^x
    }
  float s = 0.f;
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_ub_dfma(float* out, int iters) {
  double x[kChains];
  for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
  const double a = 0.999, b = 1e-3;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  double s = 0.0;
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.0) out[blockIdx.x] = static_cast<float>(s);
}

}  // namespace

int prism_record_error(int code, const char* msg);

extern "C" int prism_microbench(int32_t kind, double* ops_per_s, void* stream) {
  if (!ops_per_s || kind < 0 || kind > 3) return prism_record_error(PRISM_E_INVALID_ARG, "prism_microbench: bad argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return prism_record_error(PRISM_E_CUDA, "prism_microbench: device query failed");
  const int blocks = sms * 8, threads = 256;
  const int iters = (kind == 3) ? 256 : 4096;
  float* sink = nullptr;
  if (cudaMalloc(&sink, blocks * sizeof(float)) != cudaSuccess)
    return prism_record_error(PRISM_E_OOM, "prism_microbench: cudaMalloc failed");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&]() {
    switch (kind) {
      case 0: k_ub_ffma<<<blocks, threads, 0, st>>>(sink, iters); break;
      case 1: k_ub_ffma2<<<blocks, threads, 0, st>>>(sink, iters); break;
      case 2: k_ub_ex2<<<blocks, threads, 0, st>>>(sink, iters); break;
      default: k_ub_dfma<<<blocks, threads, 0, st>>>(sink, iters); break;
    }
  };
  launch();   // warm-up
  cudaEventRecord(e0, st);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1, st);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) return prism_record_error(PRISM_E_CUDA, cudaGetErrorString(err));
  // operations: FMA counts 2 (flops), packed FMA 4, 2^x 1
  const double per = (kind == 0 || kind == 3) ? 2.0 : (kind == 1 ? 4.0 : 1.0);
  const double ops = static_cast<double>(blocks) * threads * iters * kChains * per * reps;
  *ops_per_s = ops / (ms * 1e-3);
  return PRISM_OK;
}
