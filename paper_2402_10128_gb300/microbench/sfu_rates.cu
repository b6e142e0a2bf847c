// Throughput of the special-function unit (MUFU) instructions the compositing kernels use:
// ex2.approx.ftz.f32, lg2.approx.ftz.f32 and rcp.approx.ftz.f32, each on 8 independent chains per
// thread, 8 CTAs of 256 threads per SM.  Prints one JSON object: results per SM per clock at the
// device's reported maximum clock, so that a rate measured under a lower clock reads lower.
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ float ex2(float x) { float y; asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float lg2(float x) { float y; asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float rcp(float x) { float y; asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }

template <int MODE>
__global__ void chains(float* out, int iters) {
  float a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = 0.5f + 1e-3f * (float)(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (MODE == 0) a[j] = ex2(a[j] - 1.0f);        // stays in [0.5, 1]
      else if (MODE == 1) a[j] = lg2(a[j] + 1.5f);   // stays in [0.6, 1.5]
      else a[j] = rcp(a[j] + 1.0f);                  // stays in [0.4, 0.7]
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == 12345.0f) out[threadIdx.x] = s;  // keeps the chains live; never true
}

int main() {
  int sms = 0, khz = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, 0);
  float* out = nullptr;
  if (cudaMalloc(&out, 256 * sizeof(float)) != cudaSuccess) return 1;
  const int iters = 4096, threads = 256, blocks = sms * 8;
  const char* names[3] = {"ex2", "lg2", "rcp"};
  double rate[3] = {0, 0, 0};
  for (int mode = 0; mode < 3; ++mode) {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a);
      if (mode == 0) chains<0><<<blocks, threads>>>(out, iters);
      else if (mode == 1) chains<1><<<blocks, threads>>>(out, iters);
      else chains<2><<<blocks, threads>>>(out, iters);
      cudaEventRecord(b);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0 && ms < best) best = ms;
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
    const double ops = (double)blocks * threads * iters * 8;
    rate[mode] = ops / (best * 1e-3) / sms / (khz * 1e3);
  }
  cudaError_t e = cudaGetLastError();
  printf("{\"sms\": %d, \"max_clock_mhz\": %.0f, \"per_sm_per_clk\": {\"%s\": %.2f, \"%s\": %.2f, \"%s\": %.2f}, \"error\": \"%s\"}\n",
         sms, khz / 1e3, names[0], rate[0], names[1], rate[1], names[2], rate[2], cudaGetErrorString(e));
  cudaFree(out);
  return e == cudaSuccess ? 0 : 1;
}
