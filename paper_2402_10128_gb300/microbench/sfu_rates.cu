// Throughput of the special-function unit (MUFU) instructions the compositing kernels use:
// ex2.approx.ftz.f32, lg2.approx.ftz.f32 and rcp.approx.ftz.f32, each on 8 independent chains per
// thread, 8 CTAs of 256 threads per SM.  Also the FP32 FMA rate issued as scalar fma.rn.f32 and as
// packed fma.rn.f32x2, alone and interleaved one-to-one with integer xors (which share the
// warp schedulers' issue slots but not the FMA pipe).  Prints one JSON object: results per SM per
// clock at the device's reported maximum clock, so that a rate measured under a lower clock reads
// lower.
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ float ex2(float x) { float y; asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float lg2(float x) { float y; asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float rcp(float x) { float y; asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ float fma1(float a, float b, float c) {
  float d;
  asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ unsigned ixor(unsigned a, unsigned b) {
  unsigned d;
  asm volatile("xor.b32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// FMA modes, 8 FP32 FMAs per iteration and chain group: 0 scalar, 1 packed, 2 scalar + 8 integer
// xors, 3 packed + 8 integer xors (each xor mixes two integer chains, so it cannot be folded away)
template <int MODE>
__global__ void fma_chains(float* out, int iters) {
  float a[8];
  unsigned b[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    a[j] = 1e-3f * (float)(threadIdx.x + j);
    b[j] = threadIdx.x + j;
  }
  const float m = 0.999f, c = 1e-4f;
  const unsigned long long m2 = pack2(m, m), c2 = pack2(c, c);
  for (int i = 0; i < iters; ++i) {
    if (MODE == 0 || MODE == 2) {
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = fma1(a[j], m, c);
    } else {
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        const float2 r = unpack2(fma2(pack2(a[j], a[j + 1]), m2, c2));
        a[j] = r.x;
        a[j + 1] = r.y;
      }
    }
    if (MODE >= 2) {
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = ixor(b[j], b[(j + 1) & 7]);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j] + (float)(b[j] & 1u);
  if (s == 12345.0f) out[threadIdx.x] = s;
}

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
  const char* fnames[4] = {"fma", "fma_f32x2", "fma_with_ixor", "fma_f32x2_with_ixor"};
  double frate[4] = {0, 0, 0, 0};
  for (int mode = 0; mode < 4; ++mode) {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a);
      if (mode == 0) fma_chains<0><<<blocks, threads>>>(out, iters);
      else if (mode == 1) fma_chains<1><<<blocks, threads>>>(out, iters);
      else if (mode == 2) fma_chains<2><<<blocks, threads>>>(out, iters);
      else fma_chains<3><<<blocks, threads>>>(out, iters);
      cudaEventRecord(b);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0 && ms < best) best = ms;
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
    const double ops = (double)blocks * threads * iters * 8;  // FP32 FMAs
    frate[mode] = ops / (best * 1e-3) / sms / (khz * 1e3);
  }
  cudaError_t e = cudaGetLastError();
  printf("{\"sms\": %d, \"max_clock_mhz\": %.0f, \"per_sm_per_clk\": {\"%s\": %.2f, \"%s\": %.2f, \"%s\": %.2f, "
         "\"%s\": %.2f, \"%s\": %.2f, \"%s\": %.2f, \"%s\": %.2f}, \"error\": \"%s\"}\n",
         sms, khz / 1e3, names[0], rate[0], names[1], rate[1], names[2], rate[2], fnames[0], frate[0], fnames[1], frate[1],
         fnames[2], frate[2], fnames[3], frate[3], cudaGetErrorString(e));
  cudaFree(out);
  return e == cudaSuccess ? 0 : 1;
}
