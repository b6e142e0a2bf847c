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
// view are [prim_base, prim_base + n); global tile ids [tile_base, tile_base + tiles_x*tiles_y);
// global segment ids [seg_base, seg_base + segs_x*tiles_y), where a segment is a run of
// 2^seg_log2 tiles of one tile row (segs_x = ceil(tiles_x / 2^seg_log2)).
struct ViewDesc {
  float V[12];                 // world -> camera, rows of the 3x4 upper block
  float fx, fy, cx, cy;
  float campos[3];
  float znear;
  float bg[3];
  int32_t W, H, tiles_x, tiles_y;
  int32_t tile_base;
  int32_t seg_base, segs_x;
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
  long long total_segs;            // sum of the views' segments
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
  int32_t seg_log2;            // log2 of the tiles per segment
  int32_t seg_bits;            // bits of a global segment id (the radix sort's key width)
  int32_t phi_mode;            // 0 phi_bar_rho, 1 phi_n on the scale vector, 2 phi_n on the variance
  int32_t id_bits;             // > 0: the depth sort's values are id | list entries << id_bits
};

// A list entry's key: the global segment id in the low seg_bits bits, then the first and last
// tile of the primitive's span inside the segment, relative to the segment's first tile
// (seg_log2 bits each).  The sort orders by the segment bits only.
__device__ __forceinline__ uint32_t seg_key(uint32_t seg, uint32_t off0, uint32_t off1, const Params& P) {
  return seg | (off0 << P.seg_bits) | (off1 << (P.seg_bits + P.seg_log2));
}
// does the entry's span contain tile offset `to` (0 .. 2^seg_log2 - 1) of its segment?
__device__ __forceinline__ bool seg_key_covers(uint32_t key, uint32_t to, const Params& P) {
  const uint32_t m = (1u << P.seg_log2) - 1u;
  const uint32_t off0 = (key >> P.seg_bits) & m, off1 = (key >> (P.seg_bits + P.seg_log2)) & m;
  return off0 <= to && to <= off1;
}

// Projected primitive as the compositing kernels read it (48 bytes, gathered by id).
//   a = (mean x, mean y, q limit, beta exponent hb)    hb = beta/2 (GEF) or 1
//   b = (conic a, conic b, conic c, opacity)            q = a dx^2 + 2 b dx dy + c dy^2
//   c = (r, g, b, 0)
struct __align__(16) Rec {
  float4 a, b, c;
};

// What the key generation reads of a primitive, in one 32-byte sector: the extent's shape (2D
// covariance with dilation, and the q limit), the 2D mean, and the bounding box in tiles.
struct __align__(32) KeyShape {
  float4 ext;    // a, b, c, q limit
  float2 mean;   // u, v
  ushort4 box;   // x0, y0, x1, y1 (end-exclusive)
};

// ------------------------------------------------------------------------------------------
// Key path: FP32 with every operation rounded separately (no contraction), in a fixed order.
// These values decide integers (visibility, depth order, tile rectangles), so the oracle
// evaluates the same sequence.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float kadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float ksub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float kmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float kdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float ksqrt(float a) { return __fsqrt_rn(a); }


// Tiles of row ty that the ellipse {d : d^T cov^-1 d <= qlim} around the 2D mean (u, v) meets, on
// the key path.  ext = (a, b, c, qlim) with (a, b, c) the 2D covariance (with dilation).  The row
// band is y in [16 ty, 16 ty + 16); inside it the ellipse's x-extent runs from its leftmost to its
// rightmost point, x(dy) = (b/c) dy +- sqrt((qlim - dy^2/c) det/c), whose extremes over the whole
// ellipse lie at dy = +-b sqrt(qlim/a); over the band they lie at that dy clamped into the band.
// The span, widened by margin_abs, is intersected with the bounding box's columns [r.x, r.z).
struct RowSpan {
  float u, v, ql, mabs;  // 2D mean, q limit, absolute margin
  float Y, sl, g, ic, dys;
  float r0, r1;          // first and last column of the bounding box
};

__device__ __forceinline__ RowSpan make_row_span(const float4 ext, float u, float v, float mabs, const ushort4 r) {
  const float a = ext.x, b = ext.y, c = ext.z, ql = ext.w;
  RowSpan s;
  s.u = u;
  s.v = v;
  s.ql = ql;
  s.mabs = mabs;
  s.Y = ksqrt(kmul(ql, c));
  const float det = ksub(kmul(a, c), kmul(b, b));
  s.sl = kdiv(b, c);
  s.g = kdiv(det, c);
  s.ic = kdiv(1.0f, c);
  s.dys = kmul(b, ksqrt(kdiv(ql, a)));
  s.r0 = (float)r.x;
  s.r1 = (float)(r.z - 1);
  return s;
}

__device__ __forceinline__ bool tile_row_span(const RowSpan& s, int ty, int& tx0, int& tx1) {
  const float lo = ksub((float)(16 * ty), s.v);
  const float hi = ksub((float)(16 * ty + 16), s.v);
  const float lo2 = fmaxf(lo, -s.Y), hi2 = fminf(hi, s.Y);
  if (!(lo2 <= hi2)) return false;
  const float dmax = fminf(fmaxf(s.dys, lo2), hi2);
  const float dmin = fminf(fmaxf(-s.dys, lo2), hi2);
  const float tr = fmaxf(ksub(s.ql, kmul(kmul(dmax, dmax), s.ic)), 0.0f);
  const float tl = fmaxf(ksub(s.ql, kmul(kmul(dmin, dmin), s.ic)), 0.0f);
  const float wr = ksqrt(kmul(tr, s.g)), wl = ksqrt(kmul(tl, s.g));
  const float xr = kadd(kadd(kadd(s.u, kmul(s.sl, dmax)), wr), s.mabs);
  const float xl = ksub(ksub(kadd(s.u, kmul(s.sl, dmin)), wl), s.mabs);
  float f0 = floorf(kmul(xl, 0.0625f)), f1 = floorf(kmul(xr, 0.0625f));
  // a span wholly outside the box's columns (the row's part of the ellipse is off the image) is empty
  if (!(f1 >= s.r0 && f0 <= s.r1)) return false;
  f0 = fmaxf(f0, s.r0);
  f1 = fminf(f1, s.r1);
  tx0 = (int)f0;
  tx1 = (int)f1;
  return tx1 >= tx0;
}

// ------------------------------------------------------------------------------------------
// Warp-cooperative row walk.  The warp's primitives, h[i] tile rows each, are laid out as one list
// of (primitive, row) slots in lane order; the slots are taken 32 at a time, one per lane, so that
// every lane evaluates a row span whatever the mix of large and small primitives.
// ------------------------------------------------------------------------------------------
// exclusive prefix sum over the warp's lanes; total receives the sum of all lanes
__device__ __forceinline__ unsigned warp_excl_scan(unsigned v, unsigned& total) {
  const unsigned lane = threadIdx.x & 31u;
  unsigned x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= (unsigned)d) x += y;
  }
  total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

// the last lane i whose key[i] <= s, for keys nondecreasing over the lanes with key[0] = 0
__device__ __forceinline__ int warp_last_le(unsigned key, unsigned s) {
  int lo = 0;
#pragma unroll
  for (int step = 16; step; step >>= 1) {
    const unsigned kv = __shfl_sync(0xffffffffu, key, lo + step);
    if (kv <= s) lo += step;
  }
  return lo;
}

__device__ __forceinline__ RowSpan shfl_row_span(const RowSpan& s, int src) {
  RowSpan q;
  q.u = __shfl_sync(0xffffffffu, s.u, src);
  q.v = __shfl_sync(0xffffffffu, s.v, src);
  q.ql = __shfl_sync(0xffffffffu, s.ql, src);
  q.mabs = __shfl_sync(0xffffffffu, s.mabs, src);
  q.Y = __shfl_sync(0xffffffffu, s.Y, src);
  q.sl = __shfl_sync(0xffffffffu, s.sl, src);
  q.g = __shfl_sync(0xffffffffu, s.g, src);
  q.ic = __shfl_sync(0xffffffffu, s.ic, src);
  q.dys = __shfl_sync(0xffffffffu, s.dys, src);
  q.r0 = __shfl_sync(0xffffffffu, s.r0, src);
  q.r1 = __shfl_sync(0xffffffffu, s.r1, src);
  return q;
}

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
