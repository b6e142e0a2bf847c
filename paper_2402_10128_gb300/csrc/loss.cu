// The training image loss that consumes the rendered image (Sec. 4.3 and Eq. final):
//   L = lambda_L1 L1 + lambda_ssim (1 - SSIM) + lambda_omega L_omega,  lambda_L1 = 1 - lambda_ssim - lambda_omega,
//   L_omega = mean |(I - I_gt) M_omega|                                               (Eq. laplace)
//   M_omega = 1(|DoG_omega(I_gt)| / max |DoG_omega(I_gt)| > threshold)                (Eq. mask)
//   DoG_omega = G(., 0.2 + 20 omega) - G(., 0.1 + 10 omega) on the ground truth's channel mean,
//   downsampled by the image-frequency scale (implementation details of the appendix); for
//   omega <= 1/2 the mask is 1 - M_(1 - omega).
// Readings where the paper is open: separable Gaussian blurs truncated at ceil(3 sigma), zero
// outside the image; box downsampling by f = round(1/scale) and nearest upsampling; the response
// normalised by its maximum; L1, L_omega and SSIM are means over the 3 H W values; SSIM with the
// 11 x 11 window of sigma 1.5 and C1 = 0.01^2, C2 = 0.03^2.
//
// Mask: four small kernels on the downsampled image (gray box average, row blurs, column blurs
// with |DoG| and its maximum, threshold and nearest upsampling).  Loss: two tiled kernels, one CTA
// per 32 x 16 tile and channel.  The first stages the tile of I and I_gt with a 5-pixel halo in
// shared memory and blurs x, y,
// x^2, y^2, x y separably.  It then writes, per pixel, the SSIM value's derivatives with respect
// to the blurred x, x^2 and x y, and accumulates L1, L_omega and SSIM.  The second blurs those
// derivative maps the same way (the blur is its own adjoint) and forms dL/dI.
#include <cmath>
#include <cstring>

#include "api_internal.h"

namespace ges {
namespace {

constexpr int kMaxTaps = 127;   // blur radius <= 63
constexpr int kSsimR = 5;       // SSIM window radius (11 taps)
constexpr int kTX = 32, kTY = 16;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct Weights {
  int r1, r2;
  float w1[kMaxTaps], w2[kMaxTaps];
};

struct SsimWeights {
  float w[2 * kSsimR + 1];
};

// normalised Gaussian weights on [-r, r], r = ceil(3 sigma) unless given
int gauss_weights(double sigma, int r, float* w) {
  if (r < 0) r = (int)std::ceil(3.0 * sigma);
  double s = 0.0;
  double tmp[kMaxTaps];
  for (int k = -r; k <= r; ++k) {
    tmp[k + r] = std::exp(-(double)k * k / (2.0 * sigma * sigma));
    s += tmp[k + r];
  }
  for (int k = 0; k <= 2 * r; ++k) w[k] = (float)(tmp[k] / s);
  return r;
}

// ---- mask
__global__ void k_gray_down(const float* __restrict__ gt, int W, int H, int f, int w, int h, float* __restrict__ low) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= w * h) return;
  const int x0 = (i % w) * f, y0 = (i / w) * f;
  const int x1 = min(x0 + f, W), y1 = min(y0 + f, H);
  const int64_t plane = (int64_t)W * H;
  float s = 0.f;
  for (int c = 0; c < 3; ++c)
    for (int y = y0; y < y1; ++y)
      for (int x = x0; x < x1; ++x) s += gt[c * plane + (int64_t)y * W + x];
  low[i] = s / (float)(3 * (x1 - x0) * (y1 - y0));
}

__global__ void k_rows2(const __grid_constant__ Weights wt, const float* __restrict__ low, int w, int h,
                        float* __restrict__ a, float* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= w * h) return;
  const int x = i % w, y = i / w;
  const float* row = low + (int64_t)y * w;
  float s1 = 0.f, s2 = 0.f;
  for (int k = -wt.r1; k <= wt.r1; ++k) {
    const int xx = x + k;
    if (xx >= 0 && xx < w) s1 += wt.w1[k + wt.r1] * row[xx];
  }
  for (int k = -wt.r2; k <= wt.r2; ++k) {
    const int xx = x + k;
    if (xx >= 0 && xx < w) s2 += wt.w2[k + wt.r2] * row[xx];
  }
  a[i] = s1;
  b[i] = s2;
}

__global__ void k_cols_dog(const __grid_constant__ Weights wt, const float* __restrict__ a, const float* __restrict__ b,
                           int w, int h, float* __restrict__ d, unsigned int* __restrict__ dmax) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float v = 0.f;
  if (i < w * h) {
    const int x = i % w, y = i / w;
    float s1 = 0.f, s2 = 0.f;
    for (int k = -wt.r1; k <= wt.r1; ++k) {
      const int yy = y + k;
      if (yy >= 0 && yy < h) s1 += wt.w1[k + wt.r1] * a[(int64_t)yy * w + x];
    }
    for (int k = -wt.r2; k <= wt.r2; ++k) {
      const int yy = y + k;
      if (yy >= 0 && yy < h) s2 += wt.w2[k + wt.r2] * b[(int64_t)yy * w + x];
    }
    v = fabsf(s1 - s2);
    d[i] = v;
  }
  // block maximum, then one atomic (non-negative floats order like their bit patterns)
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dmax, __float_as_uint(v));
}

__global__ void k_mask_up(const float* __restrict__ d, const unsigned int* __restrict__ dmax, int W, int H, int f, int w,
                          float threshold, int flip, uint8_t* __restrict__ mask) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)W * H) return;
  const int x = (int)(i % W), y = (int)(i / W);
  const float m = __uint_as_float(*dmax);
  const float r = m > 0.f ? __fdiv_rn(d[(int64_t)(y / f) * w + x / f], m) : 0.f;
  const bool on = r > threshold;
  mask[i] = (uint8_t)((on != (flip != 0)) ? 1 : 0);
}

// ---- loss: tile with halo, separable SSIM window
struct LossArgs {
  const float* img;
  const float* gt;
  const uint8_t* mask;
  int W, H;
  float lam_l1, lam_ssim, lam_w, inv_n;
  float* P;          // [3 maps][3 channels][H][W]: dS/dm_x, dS/dm_xx, dS/dm_xy
  double* sums;      // L1, SSIM, L_omega (sums over the 3 H W values)
  float* grad;       // dL/dI [3,H,W]
  float* loss;       // L, L1, SSIM, L_omega (means)
};

constexpr int kHX = kTX + 2 * kSsimR, kHY = kTY + 2 * kSsimR;

__device__ __forceinline__ float block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0)
    for (int k = 0; k < nw; ++k) s += red[k];
  return s;  // valid in thread 0
}

__global__ void __launch_bounds__(kTX * kTY) k_ssim_stats(const __grid_constant__ LossArgs A,
                                                          const __grid_constant__ SsimWeights sw) {
  __shared__ float sx[kHY][kHX], sy[kHY][kHX];
  __shared__ float hs[5][kHY][kTX];
  __shared__ float red[kTX * kTY / 32];
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int x = x0 + tx, y = y0 + ty;
  const bool inside = x < A.W && y < A.H;
  const int64_t plane = (int64_t)A.W * A.H;
  float acc_ssim = 0.f, acc_l1 = 0.f, acc_w = 0.f;
  const float m = inside ? (float)A.mask[(int64_t)y * A.W + x] : 0.f;
  const int c = blockIdx.z;
  {
    for (int k = threadIdx.x; k < kHX * kHY; k += blockDim.x) {
      const int hx = k % kHX, hy = k / kHX;
      const int gx = x0 + hx - kSsimR, gy = y0 + hy - kSsimR;
      float vx = 0.f, vy = 0.f;
      if (gx >= 0 && gx < A.W && gy >= 0 && gy < A.H) {
        const int64_t o = c * plane + (int64_t)gy * A.W + gx;
        vx = A.img[o];
        vy = A.gt[o];
      }
      sx[hy][hx] = vx;
      sy[hy][hx] = vy;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kTX * kHY; k += blockDim.x) {
      const int cx = k % kTX, cy = k / kTX;
      float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
      for (int t = 0; t <= 2 * kSsimR; ++t) {
        const float wv = sw.w[t], p = sx[cy][cx + t], q = sy[cy][cx + t];
        a = fmaf(wv, p, a);
        b = fmaf(wv, q, b);
        aa = fmaf(wv, p * p, aa);
        bb = fmaf(wv, q * q, bb);
        ab = fmaf(wv, p * q, ab);
      }
      hs[0][cy][cx] = a; hs[1][cy][cx] = b; hs[2][cy][cx] = aa; hs[3][cy][cx] = bb; hs[4][cy][cx] = ab;
    }
    __syncthreads();
    float mx = 0.f, my = 0.f, mxx = 0.f, myy = 0.f, mxy = 0.f;
#pragma unroll
    for (int t = 0; t <= 2 * kSsimR; ++t) {
      const float wv = sw.w[t];
      mx = fmaf(wv, hs[0][ty + t][tx], mx);
      my = fmaf(wv, hs[1][ty + t][tx], my);
      mxx = fmaf(wv, hs[2][ty + t][tx], mxx);
      myy = fmaf(wv, hs[3][ty + t][tx], myy);
      mxy = fmaf(wv, hs[4][ty + t][tx], mxy);
    }
    if (inside) {
      const float vx = mxx - mx * mx, vy = myy - my * my, cxy = mxy - mx * my;
      const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cxy + kC2;
      const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
      const float S = (A1 * A2) / (B1 * B2);
      // derivatives of S with respect to the blurred x, x^2 and x y
      const float dS_dvx = -S / B2, dS_dcxy = 2.f * S / A2;
      const float dS_dmx = S * (2.f * my / A1 - 2.f * mx / B1) + dS_dvx * (-2.f * mx) + dS_dcxy * (-my);
      const int64_t o = c * plane + (int64_t)y * A.W + x;
      A.P[o] = dS_dmx;
      A.P[3 * plane + o] = dS_dvx;
      A.P[6 * plane + o] = dS_dcxy;
      const float dxy = sx[ty + kSsimR][tx + kSsimR] - sy[ty + kSsimR][tx + kSsimR];
      acc_ssim += S;
      acc_l1 += fabsf(dxy);
      acc_w += fabsf(dxy * m);
    }
  }
  const float s0 = block_sum(acc_l1, red);
  if (threadIdx.x == 0) atomicAdd(&A.sums[0], (double)s0);
  const float s1 = block_sum(acc_ssim, red);
  if (threadIdx.x == 0) atomicAdd(&A.sums[1], (double)s1);
  const float s2 = block_sum(acc_w, red);
  if (threadIdx.x == 0) atomicAdd(&A.sums[2], (double)s2);
}

__global__ void __launch_bounds__(kTX * kTY) k_ssim_grad(const __grid_constant__ LossArgs A,
                                                         const __grid_constant__ SsimWeights sw) {
  __shared__ float sp[3][kHY][kHX];
  __shared__ float hs[3][kHY][kTX];
  const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int x = x0 + tx, y = y0 + ty;
  const bool inside = x < A.W && y < A.H;
  const int64_t plane = (int64_t)A.W * A.H;
  const float m = inside ? (float)A.mask[(int64_t)y * A.W + x] : 0.f;
  const int c = blockIdx.z;
  {
    for (int k = threadIdx.x; k < kHX * kHY; k += blockDim.x) {
      const int hx = k % kHX, hy = k / kHX;
      const int gx = x0 + hx - kSsimR, gy = y0 + hy - kSsimR;
      float v0 = 0.f, v1 = 0.f, v2 = 0.f;
      if (gx >= 0 && gx < A.W && gy >= 0 && gy < A.H) {
        const int64_t o = c * plane + (int64_t)gy * A.W + gx;
        v0 = A.P[o];
        v1 = A.P[3 * plane + o];
        v2 = A.P[6 * plane + o];
      }
      sp[0][hy][hx] = v0;
      sp[1][hy][hx] = v1;
      sp[2][hy][hx] = v2;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kTX * kHY; k += blockDim.x) {
      const int cx = k % kTX, cy = k / kTX;
      float a = 0.f, b = 0.f, d = 0.f;
#pragma unroll
      for (int t = 0; t <= 2 * kSsimR; ++t) {
        const float wv = sw.w[t];
        a = fmaf(wv, sp[0][cy][cx + t], a);
        b = fmaf(wv, sp[1][cy][cx + t], b);
        d = fmaf(wv, sp[2][cy][cx + t], d);
      }
      hs[0][cy][cx] = a; hs[1][cy][cx] = b; hs[2][cy][cx] = d;
    }
    __syncthreads();
    if (inside) {
      float g0 = 0.f, g1 = 0.f, g2 = 0.f;
#pragma unroll
      for (int t = 0; t <= 2 * kSsimR; ++t) {
        const float wv = sw.w[t];
        g0 = fmaf(wv, hs[0][ty + t][tx], g0);
        g1 = fmaf(wv, hs[1][ty + t][tx], g1);
        g2 = fmaf(wv, hs[2][ty + t][tx], g2);
      }
      const int64_t o = c * plane + (int64_t)y * A.W + x;
      const float xv = A.img[o], yv = A.gt[o];
      const float dS = g0 + 2.f * xv * g1 + yv * g2;  // d(sum of S)/dx
      const float dlt = xv - yv;
      const float sg = dlt > 0.f ? 1.f : (dlt < 0.f ? -1.f : 0.f);
      A.grad[o] = A.inv_n * (A.lam_l1 * sg + A.lam_w * sg * m - A.lam_ssim * dS);
    }
  }
}

__global__ void k_loss_final(const __grid_constant__ LossArgs A) {
  const double n = 1.0 / (double)A.inv_n;
  const double l1 = A.sums[0] / n, ssim = A.sums[1] / n, lw = A.sums[2] / n;
  A.loss[0] = (float)(A.lam_l1 * l1 + A.lam_ssim * (1.0 - ssim) + A.lam_w * lw);
  A.loss[1] = (float)l1;
  A.loss[2] = (float)ssim;
  A.loss[3] = (float)lw;
}

}  // namespace
}  // namespace ges

using namespace ges;

extern "C" {

ges_status ges_freq_mask(ges_ctx* ctx, const float* gt, int32_t width, int32_t height, float omega, float scale,
                         float threshold, uint8_t* mask, void* stream) {
  if (!ctx || !gt || !mask) return fail(GES_ERR_INVALID_ARG, "NULL argument");
  if (width < 1 || height < 1 || width > 16384 || height > 16384)
    return fail(GES_ERR_INVALID_ARG, "image size %dx%d out of range", width, height);
  if (!(omega >= 0.f && omega <= 1.f)) return fail(GES_ERR_INVALID_ARG, "omega must lie in [0,1]");
  if (!(scale > 0.f && scale <= 1.f)) return fail(GES_ERR_INVALID_ARG, "scale must lie in (0,1]");
  ges_status st = use_device(ctx->device);
  if (st != GES_OK) return st;
  const bool flip = omega <= 0.5f;
  const double om = flip ? 1.0 - (double)omega : (double)omega;
  const double s2 = 0.1 + 10.0 * om, s1 = 2.0 * s2;
  Weights wt;
  std::memset(&wt, 0, sizeof(wt));
  if ((int)std::ceil(3.0 * s1) > (kMaxTaps - 1) / 2) return fail(GES_ERR_INVALID_ARG, "blur radius too large");
  wt.r1 = gauss_weights(s1, -1, wt.w1);
  wt.r2 = gauss_weights(s2, -1, wt.w2);
  int f = (int)std::lround(1.0 / (double)scale);
  if (f < 1) f = 1;
  const int w = (width + f - 1) / f, h = (height + f - 1) / f;
  const size_t n = (size_t)w * h;
  void* buf = nullptr;
  if ((st = ctx_scratch(ctx, 0, 256 + sizeof(float) * 4 * n, &buf)) != GES_OK) return st;
  unsigned int* dmax = reinterpret_cast<unsigned int*>(buf);
  float* low = reinterpret_cast<float*>(static_cast<char*>(buf) + 256);
  float* a = low + n;
  float* b = a + n;
  float* d = b + n;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(dmax, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "memset");
  const int T = 256;
  const unsigned gb = (unsigned)((n + T - 1) / T);
  k_gray_down<<<gb, T, 0, s>>>(gt, width, height, f, w, h, low);
  k_rows2<<<gb, T, 0, s>>>(wt, low, w, h, a, b);
  k_cols_dog<<<gb, T, 0, s>>>(wt, a, b, w, h, d, dmax);
  const int64_t np = (int64_t)width * height;
  k_mask_up<<<(unsigned)((np + T - 1) / T), T, 0, s>>>(d, dmax, width, height, f, w, threshold, flip ? 1 : 0, mask);
  count_launches(4);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "freq mask launch");
  return GES_OK;
}

ges_status ges_image_loss(ges_ctx* ctx, const float* img, const float* gt, const uint8_t* mask, int32_t width,
                          int32_t height, float lambda_ssim, float lambda_omega, float* loss, float* dL_dimg,
                          void* stream) {
  if (!ctx || !img || !gt || !mask || !loss || !dL_dimg) return fail(GES_ERR_INVALID_ARG, "NULL argument");
  if (width < 1 || height < 1 || width > 16384 || height > 16384)
    return fail(GES_ERR_INVALID_ARG, "image size %dx%d out of range", width, height);
  if (!(lambda_ssim >= 0.f && lambda_omega >= 0.f && lambda_ssim + lambda_omega <= 1.f))
    return fail(GES_ERR_INVALID_ARG, "need lambda_ssim, lambda_omega >= 0 and lambda_ssim + lambda_omega <= 1");
  ges_status st = use_device(ctx->device);
  if (st != GES_OK) return st;
  const int64_t plane = (int64_t)width * height;
  void* buf = nullptr;
  if ((st = ctx_scratch(ctx, 1, 256 + sizeof(float) * 9 * (size_t)plane, &buf)) != GES_OK) return st;
  LossArgs A;
  A.img = img;
  A.gt = gt;
  A.mask = mask;
  A.W = width;
  A.H = height;
  A.lam_ssim = lambda_ssim;
  A.lam_w = lambda_omega;
  A.lam_l1 = 1.f - lambda_ssim - lambda_omega;
  A.inv_n = 1.f / (float)(3 * plane);
  A.sums = reinterpret_cast<double*>(buf);
  A.P = reinterpret_cast<float*>(static_cast<char*>(buf) + 256);
  A.grad = dL_dimg;
  A.loss = loss;
  SsimWeights sw;
  gauss_weights(1.5, kSsimR, sw.w);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(A.sums, 0, 3 * sizeof(double), s)) != cudaSuccess) return cuda_fail(e, "memset");
  const dim3 grid((unsigned)((width + kTX - 1) / kTX), (unsigned)((height + kTY - 1) / kTY), 3);  // z: channel
  k_ssim_stats<<<grid, kTX * kTY, 0, s>>>(A, sw);
  k_ssim_grad<<<grid, kTX * kTY, 0, s>>>(A, sw);
  k_loss_final<<<1, 1, 0, s>>>(A);
  count_launches(3);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "image loss launch");
  return GES_OK;
}

}  // extern "C"
