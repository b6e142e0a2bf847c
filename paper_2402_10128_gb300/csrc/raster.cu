// Tile compositing: forward (K6) and backward (K7).
//
// Discrete front-to-back form of the volume-rendering integral (Sec. 3.2, Eq. transmittance):
//   C = sum_i c_i alpha_i T_i + T_final bg,   T_i = prod_{j<i} (1 - alpha_j),
// with alpha_i = min(alpha_max, kappa_i G_i) and the GES falloff G = exp(-1/2 q^(beta/2))
// (Sec. 3.1, Eq. ges) or the paper's Gaussian-form rasterizer G = exp(-1/2 q).
// One CTA per 16x16 tile, 256 threads, one pixel per thread.  A warp covers an 8x4 pixel
// block (spatially compact, so a primitive tends to be in or out for the whole warp).
// The tile's list is staged in shared memory 256 records at a time.
#include "common.cuh"
#include "kernels.cuh"

namespace ges {

namespace {

constexpr int kBatch = 256;

__device__ __forceinline__ void pixel_of(int lt, int tiles_x, int& x, int& y) {
  const int tx = lt % tiles_x, ty = lt / tiles_x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  x = tx * kTile + (w & 1) * 8 + (lane & 7);
  y = ty * kTile + (w >> 1) * 4 + (lane >> 3);
}

template <int MAXV, bool STATS>
__global__ void __launch_bounds__(kBatch) k_render_fwd(const __grid_constant__ ViewTable<MAXV> vt,
                                                       const uint2* __restrict__ ranges,
                                                       const uint32_t* __restrict__ vals, const Rec* __restrict__ rec,
                                                       const Params P, unsigned long long* __restrict__ stats) {
  __shared__ Rec batch[kBatch];
  const int64_t tile = blockIdx.x;
  const ViewDesc& vd = vt.v[view_of_tile(vt, tile)];
  int x, y;
  pixel_of((int)(tile - vd.tile_base), vd.tiles_x, x, y);
  const bool inside = x < vd.W && y < vd.H;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const uint2 rg = ranges[tile];

  float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  uint32_t last = 0;
  uint32_t n_eval = 0, n_range = 0;
  bool done = !inside;
  for (uint32_t base = rg.x; base < rg.y; base += kBatch) {
    if (__syncthreads_count(done) == kBatch) break;
    const uint32_t idx = base + threadIdx.x;
    if (idx < rg.y) batch[threadIdx.x] = rec[vals[idx]];
    __syncthreads();
    const int cnt = (int)min((uint32_t)kBatch, rg.y - base);
    if (!__all_sync(0xffffffffu, done)) {
      for (int j = 0; j < cnt; ++j) {
        if (done) break;
        const Rec r = batch[j];
        FragEval f;
        eval_fragment(r, px, py, P.alpha_max, f);
        if (STATS) {
          ++n_eval;
          n_range += f.in_range ? 1u : 0u;
        }
        if (f.alpha < P.alpha_min) continue;
        const float Tn = T * (1.0f - f.alpha);
        if (Tn < P.t_min) {
          done = true;
          break;
        }
        const float w = f.alpha * T;
        C0 = fmaf(r.c.x, w, C0);
        C1 = fmaf(r.c.y, w, C1);
        C2 = fmaf(r.c.z, w, C2);
        T = Tn;
        last = base - rg.x + (uint32_t)j + 1u;
      }
    }
  }
  if (inside) {
    const int64_t pix = (int64_t)y * vd.W + x, plane = (int64_t)vd.W * vd.H;
    vd.img[pix] = C0 + T * vd.bg[0];
    vd.img[plane + pix] = C1 + T * vd.bg[1];
    vd.img[2 * plane + pix] = C2 + T * vd.bg[2];
    vd.final_T[pix] = T;
    vd.n_contrib[pix] = last;
  }
  if (STATS) {
    unsigned long long a = n_eval, b = n_range;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(stats, a);
      atomicAdd(stats + 1, b);
    }
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Backward.  Per pixel, walks its contributors back to front, recovering T_i = T_{i+1}/(1-alpha_i)
// from the saved final transmittance; S is the colour composited behind the current fragment.
//   dC/dalpha_i = c_i T_i - S_i / (1 - alpha_i)
//   dalpha/dkappa = G, dalpha/dG = kappa (0 where alpha is clamped)
//   dG/dp = -G/2,  p = q^hb:  dp/dq = hb p / q,  dp/dhb = p ln q  (0 for q < 1e-12)
//   q = a dx^2 + 2 b dx dy + c dy^2, dx = px - mx
// Per-pixel terms are summed over the warp by shuffles, then one vector atomic per field group.
template <int MAXV>
__global__ void __launch_bounds__(kBatch) k_render_bwd(const __grid_constant__ ViewTable<MAXV> vt,
                                                       const uint2* __restrict__ ranges,
                                                       const uint32_t* __restrict__ vals, const Rec* __restrict__ rec,
                                                       const Params P, float4* __restrict__ g2d) {
  __shared__ Rec batch[kBatch];
  __shared__ uint32_t ids[kBatch];
  __shared__ uint32_t s_max_last;
  const int64_t tile = blockIdx.x;
  const ViewDesc& vd = vt.v[view_of_tile(vt, tile)];
  int x, y;
  pixel_of((int)(tile - vd.tile_base), vd.tiles_x, x, y);
  const bool inside = x < vd.W && y < vd.H;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const uint2 rg = ranges[tile];
  const int64_t pix = (int64_t)y * vd.W + x, plane = (int64_t)vd.W * vd.H;

  float T = 0.f, gC0 = 0.f, gC1 = 0.f, gC2 = 0.f;
  uint32_t last = 0;
  if (inside) {
    T = vd.final_T[pix];
    last = vd.n_contrib[pix];
    gC0 = vd.dL_dimg[pix];
    gC1 = vd.dL_dimg[plane + pix];
    gC2 = vd.dL_dimg[2 * plane + pix];
  }
  float S0 = T * vd.bg[0], S1 = T * vd.bg[1], S2 = T * vd.bg[2];
  if (threadIdx.x == 0) s_max_last = 0;
  __syncthreads();
  atomicMax(&s_max_last, last);
  __syncthreads();
  const uint32_t max_last = s_max_last;
  const bool gef = P.mode == 0;
  const float ln2 = 0.69314718055994531f;

  for (uint32_t end = rg.x + max_last; end > rg.x;) {
    const uint32_t start = (end - rg.x > (uint32_t)kBatch) ? end - kBatch : rg.x;
    __syncthreads();
    const uint32_t idx = start + threadIdx.x;
    if (idx < end) {
      const uint32_t g = vals[idx];
      ids[threadIdx.x] = g;
      batch[threadIdx.x] = rec[g];
    }
    __syncthreads();
    for (int j = (int)(end - start) - 1; j >= 0; --j) {
      const uint32_t k = start - rg.x + (uint32_t)j + 1u;  // 1-based position in the tile's list
      float g[10];
#pragma unroll
      for (int t = 0; t < 10; ++t) g[t] = 0.f;
      bool contrib = false;
      if (k <= last) {
        const Rec r = batch[j];
        FragEval f;
        eval_fragment(r, px, py, P.alpha_max, f);
        if (f.alpha >= P.alpha_min) {
          contrib = true;
          const float oma = 1.0f - f.alpha;
          T = T / oma;
          const float w = f.alpha * T;
          const float dLda = gC0 * (r.c.x * T - S0 / oma) + gC1 * (r.c.y * T - S1 / oma) + gC2 * (r.c.z * T - S2 / oma);
          S0 = fmaf(r.c.x, w, S0);
          S1 = fmaf(r.c.y, w, S1);
          S2 = fmaf(r.c.z, w, S2);
          g[7] = gC0 * w;
          g[8] = gC1 * w;
          g[9] = gC2 * w;
          const float dG = f.clamped ? 0.f : dLda * r.b.w;
          g[5] = f.clamped ? 0.f : dLda * f.G;
          const float dp = dG * (-0.5f * f.G);
          float dq;
          if (gef) {
            if (f.q > 1e-12f) {
              dq = dp * r.a.w * f.p / f.q;
              g[6] = dp * f.p * (mufu_lg2(f.q) * ln2);
            } else {
              dq = 0.f;
            }
          } else {
            dq = dp;
          }
          g[0] = dq * (-2.f) * (r.b.x * f.dx + r.b.y * f.dy);
          g[1] = dq * (-2.f) * (r.b.y * f.dx + r.b.z * f.dy);
          g[2] = dq * f.dx * f.dx;
          g[3] = dq * 2.f * f.dx * f.dy;
          g[4] = dq * f.dy * f.dy;
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
        for (int t = 0; t < 10; ++t) g[t] = warp_sum(g[t]);
        if ((threadIdx.x & 31) == 0) {
          float4* dst = g2d + 3 * (int64_t)ids[j];
          atomicAdd(dst + 0, make_float4(g[0], g[1], g[2], g[3]));
          atomicAdd(dst + 1, make_float4(g[4], g[5], g[6], g[7]));
          atomicAdd(reinterpret_cast<float2*>(dst + 2), make_float2(g[8], g[9]));
        }
      }
    }
    end = start;
  }
}

}  // namespace

template <int MAXV>
void launch_render_fwd(const ViewTable<MAXV>& vt, int64_t total_tiles, const uint2* ranges, const uint32_t* vals,
                       const Rec* rec, const Params& P, cudaStream_t s, unsigned long long* stats) {
  if (total_tiles <= 0) return;
  if (stats)
    k_render_fwd<MAXV, true><<<(unsigned)total_tiles, kBatch, 0, s>>>(vt, ranges, vals, rec, P, stats);
  else
    k_render_fwd<MAXV, false><<<(unsigned)total_tiles, kBatch, 0, s>>>(vt, ranges, vals, rec, P, nullptr);
  count_launches(1);
}

template <int MAXV>
void launch_render_bwd(const ViewTable<MAXV>& vt, int64_t total_tiles, const uint2* ranges, const uint32_t* vals,
                       const Rec* rec, const Params& P, float4* g2d, cudaStream_t s) {
  if (total_tiles <= 0) return;
  k_render_bwd<MAXV><<<(unsigned)total_tiles, kBatch, 0, s>>>(vt, ranges, vals, rec, P, g2d);
  count_launches(1);
}

template void launch_render_fwd<1>(const ViewTable<1>&, int64_t, const uint2*, const uint32_t*, const Rec*,
                                   const Params&, cudaStream_t, unsigned long long*);
template void launch_render_fwd<kServeMaxViews>(const ViewTable<kServeMaxViews>&, int64_t, const uint2*,
                                                const uint32_t*, const Rec*, const Params&, cudaStream_t,
                                                unsigned long long*);
template void launch_render_bwd<1>(const ViewTable<1>&, int64_t, const uint2*, const uint32_t*, const Rec*,
                                   const Params&, float4*, cudaStream_t);

}  // namespace ges
