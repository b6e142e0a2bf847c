// Shared device-side definitions of libges: view descriptors, parameter block,
// projected-primitive record, and the fixed-order FP32 arithmetic of the key path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ges {

constexpr int kTile = 16;           // tile edge in pixels (16x16 tiles)
constexpr int kTilePixels = kTile * kTile;
constexpr int kServeMaxViews = 32;  // views per batched (serving) launch
constexpr uint32_t kCulledKey = 0xffffffffu;

// One view of one scene inside a batched launch.  Global primitive ids of the
// view are [prim_base, prim_base + n); global tile ids [tile_base, tile_base + tiles_x*tiles_y).
struct ViewDesc {
  float V[12];                 // world -> camera, rows of the 3x4 upper block
  float fx, fy, cx, cy;
  float campos[3];
  float znear;
  float bg[3];
  int32_t W, H, tiles_x, tiles_y;
  int32_t tile_base;
  int32_t sh_degree;
  int64_t prim_base;
  int64_t n;
  const float* means;          // [n,3]
  const float* scales;         // [n,3]
  const float* quats;          // [n,4]
  const float* betas;          // [n]
  const float* opac;           // [n]
  const float* shs;            // [n,(d+1)^2,3]
  float* img;                  // [3,H,W]
  float* final_T;              // [H,W]
  uint32_t* n_contrib;         // [H,W]
  const float* dL_dimg;        // [3,H,W] (backward)
  float* g_means;              // backward outputs (same shapes as the scene)
  float* g_scales;
  float* g_quats;
  float* g_betas;
  float* g_opac;
  float* g_shs;
};

// Views of one launch, passed by value as a __grid_constant__ kernel parameter so that a
// launch carries everything it needs (no host staging buffer; capturable in a CUDA graph).
// Views are ordered by prim_base and by tile_base.
template <int MAXV>
struct ViewTable {
  int32_t n;
  int32_t pad;
  unsigned long long total_prims;  // sum of the views' n
  long long total_tiles;           // sum of the views' tiles
  ViewDesc v[MAXV];
};

// Where a kernel finds its view table: passed by value as a __grid_constant__ parameter (a single
// frame), or read from device memory (serving batches, whose captured graphs replay unchanged
// while the table is rewritten between replays).
template <int MAXV>
struct ViewsByValue {
  static constexpr int kMax = MAXV;
  ViewTable<MAXV> t;
  __device__ __forceinline__ const ViewTable<MAXV>& get() const { return t; }
};
template <int MAXV>
struct ViewsInMemory {
  static constexpr int kMax = MAXV;
  const ViewTable<MAXV>* p;
  __device__ __forceinline__ const ViewTable<MAXV>& get() const { return *p; }
};
using FrameViews = ViewsByValue<1>;
using BatchViews = ViewsInMemory<kServeMaxViews>;

template <int MAXV>
__device__ __forceinline__ int view_of_prim(const ViewTable<MAXV>& vt, int64_t g) {
  if (MAXV == 1) return 0;
  int lo = 0, hi = vt.n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (vt.v[mid].prim_base <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int MAXV>
__device__ __forceinline__ int view_of_tile(const ViewTable<MAXV>& vt, int64_t tile) {
  if (MAXV == 1) return 0;
  int lo = 0, hi = vt.n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (vt.v[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct Params {
  float rho, dilation, alpha_max, alpha_min, t_min, margin_rel, margin_abs, clamp_fov;
  int32_t mode;                // 0 GEF falloff, 1 Gaussian-form (paper's rasterizer)
};

// Projected primitive as the compositing kernels read it (48 bytes, gathered by id).
//   a = (mean x, mean y, q limit, beta exponent hb)    hb = beta/2 (GEF) or 1
//   b = (conic a, conic b, conic c, opacity)            q = a dx^2 + 2 b dx dy + c dy^2
//   c = (r, g, b, 0)
struct __align__(16) Rec {
  float4 a, b, c;
};

// ------------------------------------------------------------------------------------------
// Compositing arithmetic shared by the forward and backward kernels.  Both must take the
// same decisions (skip, clamp, stop) bit for bit, so the sequence is written with explicit
// intrinsics: the compiler has no freedom to contract it differently in the two kernels.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float mufu_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr float kNegHalfLog2e = -0.72134752044448170f;  // -1/2 log2(e): exp(-p/2) = 2^(kNegHalfLog2e p)

struct FragEval {
  float dx, dy, q, p, G, alpha, lq;  // lq = log2 q (GEF exponent path only)
  bool in_range, clamped;
};

// q = d^T conic d with d = pixel - mean; p = q^hb; G = exp(-p/2); alpha = min(alpha_max, kappa G)
__device__ __forceinline__ void eval_fragment(const Rec& r, float px, float py, float alpha_max, FragEval& f) {
  f.dx = __fsub_rn(px, r.a.x);
  f.dy = __fsub_rn(py, r.a.y);
  // q = (a dx + 2 b dy) dx + c dy dy
  float t = __fmaf_rn(__fmul_rn(2.0f, r.b.y), f.dy, __fmul_rn(r.b.x, f.dx));
  f.q = __fmaf_rn(__fmul_rn(r.b.z, f.dy), f.dy, __fmul_rn(t, f.dx));
  f.q = fmaxf(f.q, 0.0f);
  f.in_range = f.q <= r.a.z;  // beyond the extent alpha < alpha_min; decided without the MUFU work
  if (!f.in_range) {
    f.p = f.G = f.alpha = f.lq = 0.0f;
    f.clamped = false;
    return;
  }
  if (r.a.w == 1.0f) {
    f.p = f.q;
    f.lq = 0.f;
  } else {
    f.lq = mufu_lg2(f.q);
    f.p = mufu_ex2(__fmul_rn(r.a.w, f.lq));
  }
  f.G = mufu_ex2(__fmul_rn(kNegHalfLog2e, f.p));
  float a = __fmul_rn(r.b.w, f.G);
  f.clamped = a > alpha_max;
  f.alpha = f.clamped ? alpha_max : a;
}

// Real SH basis (l-major, m = -l..l, Condon-Shortley phase), Cartesian polynomial forms on
// the unit direction; normalisations K_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times
// sqrt 2 for m != 0) folded into the constants below.
struct SHConst {
  // degree 0
  static constexpr double kPi = 3.14159265358979323846;
};

__host__ __device__ constexpr double sh_fact(int n) { return n <= 1 ? 1.0 : n * sh_fact(n - 1); }
__host__ __device__ constexpr double sh_sqrt_newton(double x, double g, int it) {
  return it == 0 ? g : sh_sqrt_newton(x, 0.5 * (g + x / g), it - 1);
}
__host__ __device__ constexpr double sh_csqrt(double x) { return sh_sqrt_newton(x, x > 1 ? x : 1.0, 60); }
// K_lm (times sqrt(2) for m != 0)
__host__ __device__ constexpr double sh_norm(int l, int m) {
  return (m == 0 ? 1.0 : sh_csqrt(2.0)) *
         sh_csqrt((2.0 * l + 1.0) / (4.0 * SHConst::kPi) * sh_fact(l - (m < 0 ? -m : m)) / sh_fact(l + (m < 0 ? -m : m)));
}

}  // namespace ges
