// Per-SM issue rates of the SFU approximations (ex2, lg2, rcp, rsqrt) and of FFMA on the
// GPU it runs on: the denominators of the likelihood kernels' SFU and FP32 rooflines.
//
// Each thread runs 8 independent chains of one PTX instruction (plus one FP32 operation
// that keeps the chain from folding), 4096 iterations, two blocks of 1024 threads per SM.
// The total rate is instructions / CUDA-event time; test_gpu_pipe_rates.py divides it by
// the SM count and the SM clock sampled during the run.  Bounded loops, no waits.  Prints
// one JSON object.  Test infrastructure: not part of the library.
#include <cuda_runtime.h>

#include <cstdio>

namespace {

__device__ __forceinline__ float op_ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float op_lg2(float x) {
  float y;
  asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float op_rcp(float x) {
  float y;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float op_rsqrt(float x) {
  float y;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr int kChains = 8;
constexpr int kThreads = 1024;
constexpr int kIters = 4096;

template <int OP>
__global__ void __launch_bounds__(kThreads) chains(float* out) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 0.5f + 0.01f * (float)(threadIdx.x + i);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      if (OP == 0) a[i] = op_ex2(a[i]) * 0.5f;
      if (OP == 1) a[i] = op_lg2(a[i] + 1.5f);
      if (OP == 2) a[i] = op_rcp(a[i] + 1.0f);
      if (OP == 3) a[i] = op_rsqrt(a[i] + 1.0f);
      if (OP == 4) a[i] = fmaf(a[i], 0.999f, 0.001f);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
void launch(int blocks, float* out) {
  chains<OP><<<blocks, kThreads>>>(out);
}

}  // namespace

int main() {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || sms <= 0) {
    std::printf("{\"error\": \"no device\"}\n");
    return 1;
  }
  const int blocks = 2 * sms;
  float* out = nullptr;
  if (cudaMalloc(&out, sizeof(float) * (size_t)blocks * kThreads) != cudaSuccess) {
    std::printf("{\"error\": \"allocation failed\"}\n");
    return 1;
  }
  const char* names[] = {"ex2.approx.ftz.f32", "lg2.approx.ftz.f32", "rcp.approx.ftz.f32",
                         "rsqrt.approx.ftz.f32", "fma.rn.f32"};
  void (*launchers[])(int, float*) = {launch<0>, launch<1>, launch<2>, launch<3>, launch<4>};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::printf("{\"sms\": %d, \"total_gops\": {", sms);
  for (int op = 0; op < 5; ++op) {
    float best = 0.f;
    for (int rep = 0; rep < 4; ++rep) {   // the first launch warms up; keep the fastest of the rest
      cudaEventRecord(e0);
      launchers[op](blocks, out);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep == 1 || (rep > 1 && ms < best)) best = ms;
    }
    const double total = (double)blocks * kThreads * kChains * kIters;
    std::printf("%s\"%s\": %.1f", op ? ", " : "", names[op], total / (best * 1e6));
  }
  const cudaError_t err = cudaGetLastError();
  std::printf("}, \"status\": \"%s\"}\n", cudaGetErrorString(err));
  cudaFree(out);
  return err == cudaSuccess ? 0 : 1;
}
