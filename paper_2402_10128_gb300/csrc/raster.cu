// Tile compositing: forward (K6) and backward (K7).
//
// Discrete front-to-back form of the volume-rendering integral (Sec. 3.2, Eq. transmittance):
//   C = sum_i c_i alpha_i T_i + T_final bg,   T_i = prod_{j<i} (1 - alpha_j),
// with alpha_i = min(alpha_max, kappa_i G_i) and the GES falloff G = exp(-1/2 q^(beta/2))
// (Sec. 3.1, Eq. ges) or the paper's Gaussian-form rasterizer G = exp(-1/2 q).
//
// Forward: one CTA of 256 threads per 16x16 tile, one pixel per thread, warps on 8x4 blocks.
// Backward: one CTA of 128 threads per tile, two pixels per thread, (x, y) and (x, y + 4), so a
// warp covers an 8x8 block and its per-fragment gradient sum is shared by 64 pixels.  The tile's
// list is staged in shared memory one record per thread per round.  Both kernels evaluate every
// (fragment, pixel) pair with eval_fragment, so they take the same skip / clamp / stop decisions
// bit for bit whatever their thread layout.
#include "common.cuh"
#include "kernels.cuh"

namespace ges {

namespace {

constexpr int kThreads = 128;  // backward, per tile
constexpr int kBatch = kThreads;
constexpr int kFwdThreads = 256;
constexpr int kFwdBatch = kFwdThreads;

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

struct WarpBlock {
  int x, y;  // first pixel of this thread (the second is at y + 4)
};

// backward layout: warp w of the tile covers the 8x8 block at ((w & 1) * 8, (w >> 1) * 8)
__device__ __forceinline__ WarpBlock warp_block(int lt, int tiles_x) {
  const int tx = lt % tiles_x, ty = lt / tiles_x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpBlock b;
  b.x = tx * kTile + (w & 1) * 8 + (lane & 7);
  b.y = ty * kTile + (w >> 1) * 8 + (lane >> 3);
  return b;
}

template <int MAXV, bool STATS>
__device__ __forceinline__ void render_tile_fwd(const ViewTable<MAXV>& vt, int64_t tile, Rec* batch,
                                                const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                                                const Rec* __restrict__ rec, const Params& P,
                                                unsigned long long* __restrict__ stats) {
  const ViewDesc& vd = vt.v[view_of_tile(vt, tile)];
  const int lt = (int)(tile - vd.tile_base);
  const int tx = lt % vd.tiles_x, ty = lt / vd.tiles_x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int x = tx * kTile + (w & 1) * 8 + (lane & 7);
  const int y = ty * kTile + (w >> 1) * 4 + (lane >> 3);
  const bool inside = x < vd.W && y < vd.H;
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const uint2 rg = ranges[tile];
  float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  uint32_t last = 0, n_eval = 0, n_range = 0, n_comp = 0;
  bool done = !inside;
  for (uint32_t base = rg.x; base < rg.y; base += kFwdBatch) {
    if (__syncthreads_count(done) == kFwdThreads) break;
    const uint32_t idx = base + threadIdx.x;
    if (idx < rg.y) batch[threadIdx.x] = rec[vals[idx]];
    __syncthreads();
    const int cnt = (int)min((uint32_t)kFwdBatch, rg.y - base);
    if (!__all_sync(0xffffffffu, done)) {
      for (int j = 0; j < cnt; ++j) {
        if (done) break;
        const Rec r = batch[j];
        FragEval f;
        eval_fragment(r, px, py, P.alpha_max, f);
        if (STATS) { ++n_eval; n_range += f.in_range ? 1u : 0u; }
        if (f.alpha < P.alpha_min) continue;
        const float Tn = T * (1.0f - f.alpha);
        if (Tn < P.t_min) { done = true; break; }
        const float wgt = f.alpha * T;
        C0 = fmaf(r.c.x, wgt, C0);
        C1 = fmaf(r.c.y, wgt, C1);
        C2 = fmaf(r.c.z, wgt, C2);
        T = Tn;
        last = base - rg.x + (uint32_t)j + 1u;
        if (STATS) ++n_comp;
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
    unsigned long long a = n_eval, b = n_range, c = n_comp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(stats, a);
      atomicAdd(stats + 1, b);
      atomicAdd(stats + 2, c);
    }
  }
}

template <class VS, bool STATS>
__global__ void __launch_bounds__(kFwdThreads) k_render_fwd(const __grid_constant__ VS vs, const uint2* __restrict__ ranges,
                                                         const uint32_t* __restrict__ vals, const Rec* __restrict__ rec,
                                                         const Params P, unsigned long long* __restrict__ stats) {
  __shared__ Rec batch[kFwdBatch];
  render_tile_fwd<VS::kMax, STATS>(vs.get(), (int64_t)blockIdx.x, batch, ranges, vals, rec, P, stats);
}

// Persistent form: CTAs take tiles from a work counter until the table's total_tiles are done, so
// a fixed grid serves batches of any size (the launch can be replayed from a captured graph).
template <class VS>
__global__ void __launch_bounds__(kFwdThreads) k_render_fwd_persistent(const __grid_constant__ VS vs,
                                                                    const uint2* __restrict__ ranges,
                                                                    const uint32_t* __restrict__ vals,
                                                                    const Rec* __restrict__ rec, const Params P,
                                                                    unsigned int* __restrict__ tile_counter) {
  __shared__ Rec batch[kFwdBatch];
  __shared__ unsigned int s_tile;
  const auto& vt = vs.get();
  const long long total = vt.total_tiles;
  for (;;) {
    __syncthreads();  // previous tile's readers of s_tile and batch are done
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const unsigned int tile = s_tile;
    if ((long long)tile >= total) break;
    render_tile_fwd<VS::kMax, false>(vt, (int64_t)tile, batch, ranges, vals, rec, P, nullptr);
  }
}

// Sums 16 per-lane values over the warp with a reduce-scatter butterfly (16 shuffles instead of
// 16 x 5): at each step a lane keeps half of its values and receives the partner's copy of that
// half.  On return lane L holds the full sum of value ((L >> 1) & 15) (L and L^1 hold the same).
__device__ __forceinline__ float warp_reduce_scatter16(float (&v)[16]) {
  const unsigned lane = threadIdx.x & 31u;
#pragma unroll
  for (int step = 0; step < 4; ++step) {
    const int half = 8 >> step;          // values kept after this step
    const int o = 16 >> step;            // partner distance
    const bool upper = (lane & (unsigned)o) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const float send = upper ? v[k] : v[k + half];
      const float keep = upper ? v[k + half] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Backward.  Per pixel, walks its contributors back to front, recovering T_i = T_{i+1}/(1-alpha_i)
// from the saved final transmittance; S is the colour composited behind the current fragment.
//   dC/dalpha_i = c_i T_i - S_i / (1 - alpha_i)
//   dalpha/dkappa = G, dalpha/dG = kappa (0 where alpha is clamped)
//   dG/dp = -G/2,  p = q^hb:  dp/dq = hb p / q,  dp/dhb = p ln q  (0 for q < 1e-12)
//   q = a dx^2 + 2 b dx dy + c dy^2, dx = px - mx
// A thread sums its two pixels' terms, the warp sums by a reduce-scatter butterfly, and ten lanes
// add the ten per-primitive sums with one atomic each.  Reciprocals use the approximate MUFU
// instruction (about 1 ulp); they only scale gradients, never decide a branch.
template <class VS>
__global__ void __launch_bounds__(kThreads) k_render_bwd(const __grid_constant__ VS vs, const uint2* __restrict__ ranges,
                                                         const uint32_t* __restrict__ vals, const Rec* __restrict__ rec,
                                                         const Params P, float4* __restrict__ g2d) {
  __shared__ Rec batch[kBatch];
  __shared__ uint32_t ids[kBatch];
  __shared__ uint32_t s_max_last;
  const auto& vt = vs.get();
  const int64_t tile = blockIdx.x;
  const ViewDesc& vd = vt.v[view_of_tile(vt, tile)];
  const WarpBlock wb = warp_block((int)(tile - vd.tile_base), vd.tiles_x);
  const uint2 rg = ranges[tile];
  const int64_t plane = (int64_t)vd.W * vd.H;

  float px[2], py[2], T[2], gC0[2], gC1[2], gC2[2], S0[2], S1[2], S2[2];
  uint32_t last[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int y = wb.y + 4 * k;
    const bool inside = wb.x < vd.W && y < vd.H;
    px[k] = (float)wb.x + 0.5f;
    py[k] = (float)y + 0.5f;
    T[k] = 0.f; gC0[k] = gC1[k] = gC2[k] = 0.f;
    last[k] = 0;
    if (inside) {
      const int64_t pix = (int64_t)y * vd.W + wb.x;
      T[k] = vd.final_T[pix];
      last[k] = vd.n_contrib[pix];
      gC0[k] = vd.dL_dimg[pix];
      gC1[k] = vd.dL_dimg[plane + pix];
      gC2[k] = vd.dL_dimg[2 * plane + pix];
    }
    S0[k] = T[k] * vd.bg[0];
    S1[k] = T[k] * vd.bg[1];
    S2[k] = T[k] * vd.bg[2];
  }
  if (threadIdx.x == 0) s_max_last = 0;
  __syncthreads();
  atomicMax(&s_max_last, max(last[0], last[1]));
  __syncthreads();
  const uint32_t max_last = s_max_last;
  const uint32_t wlast = __reduce_max_sync(0xffffffffu, max(last[0], last[1]));
  const bool gef = P.mode == 0;
  const float ln2 = 0.69314718055994531f;
  const unsigned lane = threadIdx.x & 31u;

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
      const uint32_t kpos = start - rg.x + (uint32_t)j + 1u;  // 1-based position in the tile's list
      if (kpos > wlast) continue;                             // beyond every pixel of this warp
      const Rec r = batch[j];
      float g[16];
#pragma unroll
      for (int t = 0; t < 16; ++t) g[t] = 0.f;
      bool contrib = false;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (kpos > last[k]) continue;
        FragEval f;
        eval_fragment(r, px[k], py[k], P.alpha_max, f);
        if (f.alpha < P.alpha_min) continue;
        contrib = true;
        const float inv = rcp_approx(1.0f - f.alpha);
        T[k] *= inv;
        const float w = f.alpha * T[k];
        const float dLda = gC0[k] * (r.c.x * T[k] - S0[k] * inv) + gC1[k] * (r.c.y * T[k] - S1[k] * inv) +
                           gC2[k] * (r.c.z * T[k] - S2[k] * inv);
        S0[k] = fmaf(r.c.x, w, S0[k]);
        S1[k] = fmaf(r.c.y, w, S1[k]);
        S2[k] = fmaf(r.c.z, w, S2[k]);
        g[7] += gC0[k] * w;
        g[8] += gC1[k] * w;
        g[9] += gC2[k] * w;
        const float dG = f.clamped ? 0.f : dLda * r.b.w;
        g[5] += f.clamped ? 0.f : dLda * f.G;
        const float dp = dG * (-0.5f * f.G);
        float dq;
        if (gef) {
          if (f.q > 1e-12f) {
            if (r.a.w == 1.0f) {
              dq = dp;
              g[6] += dp * f.q * (mufu_lg2(f.q) * ln2);
            } else {
              dq = dp * r.a.w * f.p * rcp_approx(f.q);
              g[6] += dp * f.p * (f.lq * ln2);
            }
          } else {
            dq = 0.f;
          }
        } else {
          dq = dp;
        }
        const float dqdx = dq * f.dx, dqdy = dq * f.dy;
        g[0] -= 2.f * (r.b.x * dqdx + r.b.y * dqdy);
        g[1] -= 2.f * (r.b.y * dqdx + r.b.z * dqdy);
        g[2] += dqdx * f.dx;
        g[3] += 2.f * dqdx * f.dy;
        g[4] += dqdy * f.dy;
      }
      if (__any_sync(0xffffffffu, contrib)) {
        const float sum = warp_reduce_scatter16(g);
        const unsigned slot = (lane >> 1) & 15u;
        if ((lane & 1u) == 0 && slot < 10u) atomicAdd(reinterpret_cast<float*>(g2d + 3 * (int64_t)ids[j]) + slot, sum);
      }
    }
    end = start;
  }
}

}  // namespace

template <class VS>
void launch_render_fwd(const VS& vs, int64_t total_tiles, const uint2* ranges, const uint32_t* vals, const Rec* rec,
                       const Params& P, cudaStream_t s, unsigned long long* stats, unsigned int* tile_counter,
                       int num_sms) {
  if (total_tiles <= 0) return;
  if (tile_counter) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_fwd_persistent<VS>, kFwdThreads, 0);
    const int64_t grid = (int64_t)num_sms * (per_sm > 0 ? per_sm : 1);
    k_render_fwd_persistent<VS><<<(unsigned)(grid < total_tiles ? grid : total_tiles), kFwdThreads, 0, s>>>(
        vs, ranges, vals, rec, P, tile_counter);
  } else if (stats) {
    k_render_fwd<VS, true><<<(unsigned)total_tiles, kFwdThreads, 0, s>>>(vs, ranges, vals, rec, P, stats);
  } else {
    k_render_fwd<VS, false><<<(unsigned)total_tiles, kFwdThreads, 0, s>>>(vs, ranges, vals, rec, P, nullptr);
  }
  count_launches(1);
}

template <class VS>
void launch_render_bwd(const VS& vs, int64_t total_tiles, const uint2* ranges, const uint32_t* vals, const Rec* rec,
                       const Params& P, float4* g2d, cudaStream_t s) {
  if (total_tiles <= 0) return;
  k_render_bwd<VS><<<(unsigned)total_tiles, kThreads, 0, s>>>(vs, ranges, vals, rec, P, g2d);
  count_launches(1);
}

template void launch_render_fwd<FrameViews>(const FrameViews&, int64_t, const uint2*, const uint32_t*, const Rec*,
                                            const Params&, cudaStream_t, unsigned long long*, unsigned int*, int);
template void launch_render_fwd<BatchViews>(const BatchViews&, int64_t, const uint2*, const uint32_t*, const Rec*,
                                            const Params&, cudaStream_t, unsigned long long*, unsigned int*, int);
template void launch_render_bwd<FrameViews>(const FrameViews&, int64_t, const uint2*, const uint32_t*, const Rec*,
                                            const Params&, float4*, cudaStream_t);

}  // namespace ges
