// Tile compositing: forward (K6) and backward (K7).
//
// Discrete front-to-back form of the volume-rendering integral (Sec. 4.2, Eq. transmittance):
//   C = sum_i c_i alpha_i T_i + T_final bg,   T_i = prod_{j<i} (1 - alpha_j),
// with alpha_i = min(alpha_max, kappa_i G_i) and the GES falloff G = exp(-1/2 q^(beta/2))
// (Sec. 4.1, Eq. ges) or the paper's Gaussian-form rasterizer G = exp(-1/2 q).
//
// Both kernels run one CTA of 128 threads per 16x16 tile, two pixels per thread, (x, y) and
// (x, y + 4), so a warp covers an 8x8 block (and, backward, its per-fragment gradient sum is shared
// by 64 pixels).  The two pixels share x and every fragment, so their arithmetic runs as packed
// float2 pairs, one instruction for both.  The tile's list is staged in shared memory one record
// per thread per round.  Both kernels evaluate every (fragment, pixel) pair with eval_pair, so
// they take the same skip / clamp / stop decisions bit for bit.
#include "common.cuh"
#include "kernels.cuh"

namespace ges {

namespace {

constexpr int kThreads = 128;  // backward, per tile
constexpr int kBatch = kThreads;
constexpr int kFwdThreads = 128;
constexpr int kFwdBatch = 2 * kFwdThreads;  // list positions per round: two per thread

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// A fragment's record as the composite kernels read it: every value the two pixels of a thread
// share is stored twice, so that one 16-byte shared load gives two ready float2 operands.  Five
// such loads per fragment (the q limit, read only when counting work, comes from the global
// record); the backward adds the conic's b pair.
struct RecPair {
  float4 m;    // -mx, -mx, -my, -my
  float4 c0;   // conic a x2, 2 conic b x2
  float4 c1;   // conic c x2, kappa x2
  float4 k0;   // r x2, g x2
  float4 k1;   // b x2, beta/2 x2
};
// the backward's copy adds the conic terms of the mean gradient
struct RecPairB : RecPair {
  float2 nb;   // conic b x2 (the mean gradient's cross term; a and c are in c0 and c1)
};

__device__ __forceinline__ void stage_pair(RecPair& d, const Rec& r) {
  d.m = make_float4(-r.a.x, -r.a.x, -r.a.y, -r.a.y);
  const float tb = __fmul_rn(2.0f, r.b.y);
  d.c0 = make_float4(r.b.x, r.b.x, tb, tb);
  d.c1 = make_float4(r.b.z, r.b.z, r.b.w, r.b.w);
  d.k0 = make_float4(r.c.x, r.c.x, r.c.y, r.c.y);
  d.k1 = make_float4(r.c.z, r.c.z, r.a.w, r.a.w);
}

__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 sel2(bool a, bool b, float2 v, float2 z) {
  return make_float2(a ? v.x : z.x, b ? v.y : z.y);
}

// The fragment test on a thread's two pixels (PX, PY; both share x), with explicit round-to-
// nearest intrinsics so that the compiler cannot contract it differently in the two kernels:
//   d = pixel - mean, q = max(0, (a dx + 2 b dy) dx + c dy dy),
//   p = q^hb = 2^(hb log2 q) (p = q at hb = 1), G = exp(-p/2) = 2^(-p log2(e)/2), a = kappa G;
// the caller takes alpha = min(alpha_max, a) and skips the fragment where alpha < alpha_min.
// No separate test against the extent's q limit is needed: beyond it kappa G < alpha_min by
// construction of the extent.
struct PairEval {
  float2 dx, dy, p, lq, G, a;
  float q0, q1;
};
__device__ __forceinline__ void eval_pair(const RecPair& r, float2 PX, float2 PY, PairEval& f) {
  const float4 m = r.m, c0 = r.c0, c1 = r.c1, e = r.k1;  // e.z, e.w: beta/2
  f.dx = __fadd2_rn(PX, lo2(m));
  f.dy = __fadd2_rn(PY, hi2(m));
  const float2 t = __ffma2_rn(hi2(c0), f.dy, __fmul2_rn(lo2(c0), f.dx));
  const float2 q2 = __ffma2_rn(__fmul2_rn(lo2(c1), f.dy), f.dy, __fmul2_rn(t, f.dx));
  f.q0 = fmaxf(q2.x, 0.0f);
  f.q1 = fmaxf(q2.y, 0.0f);
  if (e.z == 1.0f) {
    f.p = make_float2(f.q0, f.q1);
    f.lq = make_float2(0.f, 0.f);
  } else {
    f.lq = make_float2(mufu_lg2(f.q0), mufu_lg2(f.q1));
    const float2 hl = __fmul2_rn(hi2(e), f.lq);
    f.p = make_float2(mufu_ex2(hl.x), mufu_ex2(hl.y));
  }
  const float2 ge = __fmul2_rn(make_float2(kNegHalfLog2e, kNegHalfLog2e), f.p);
  f.G = make_float2(mufu_ex2(ge.x), mufu_ex2(ge.y));
  f.a = __fmul2_rn(hi2(c1), f.G);
}

// The shared memory a composite CTA stages one round of its segment's list in: the entries whose
// span covers the CTA's tile, in list order (rec pairs, 1-based list positions, primitive ids).
template <class RecT, int N>
struct Stage {
  RecT rec[N];
  uint32_t pos[N];
  uint32_t id[N];
  uint32_t warp_count[N / 32];
};

// Keeps, in order, the round's candidates (one per thread: list entry idx, valid if `keep`) into
// st.rec / st.pos / st.id [0, count) and returns count.  Every thread of the CTA calls it; it
// contains two barriers, the second after the staging writes.
template <int N, class RecT, class StageFn>
__device__ __forceinline__ int stage_kept(Stage<RecT, N>& st, bool keep, uint32_t idx, uint32_t list_start,
                                          const uint32_t* __restrict__ vals, StageFn stage_rec) {
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  if (lane == 0) st.warp_count[w] = (uint32_t)__popc(m);
  __syncthreads();
  uint32_t off = 0, total = 0;
#pragma unroll
  for (int k = 0; k < N / 32; ++k) {
    const uint32_t c = st.warp_count[k];
    off += k < (int)w ? c : 0u;
    total += c;
  }
  if (keep) {
    const uint32_t at = off + (uint32_t)__popc(m & ((1u << lane) - 1u));
    const uint32_t g = vals[idx];
    stage_rec(st.rec[at], g);
    st.pos[at] = idx - list_start + 1u;
    st.id[at] = g;
  }
  __syncthreads();
  return (int)total;
}

// The same for two candidates per thread (positions idx0 < idx1 of a round of 2 NT): the round's
// first half is kept in order, then the second.
template <int NT, class RecT, class StageFn>
__device__ __forceinline__ int stage_kept2(Stage<RecT, 2 * NT>& st, bool keep0, uint32_t idx0, bool keep1,
                                           uint32_t idx1, uint32_t list_start, const uint32_t* __restrict__ vals,
                                           StageFn stage_rec) {
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const unsigned m0 = __ballot_sync(0xffffffffu, keep0), m1 = __ballot_sync(0xffffffffu, keep1);
  if (lane == 0) {
    st.warp_count[w] = (uint32_t)__popc(m0);
    st.warp_count[NT / 32 + w] = (uint32_t)__popc(m1);
  }
  __syncthreads();
  uint32_t off0 = 0, off1 = 0, t0 = 0, t1 = 0;
#pragma unroll
  for (int k = 0; k < NT / 32; ++k) {
    const uint32_t c0 = st.warp_count[k], c1 = st.warp_count[NT / 32 + k];
    off0 += k < (int)w ? c0 : 0u;
    off1 += k < (int)w ? c1 : 0u;
    t0 += c0;
    t1 += c1;
  }
  const unsigned lt = (1u << lane) - 1u;
  if (keep0) {
    const uint32_t at = off0 + (uint32_t)__popc(m0 & lt);
    const uint32_t g = vals[idx0];
    stage_rec(st.rec[at], g);
    st.pos[at] = idx0 - list_start + 1u;
    st.id[at] = g;
  }
  if (keep1) {
    const uint32_t at = t0 + off1 + (uint32_t)__popc(m1 & lt);
    const uint32_t g = vals[idx1];
    stage_rec(st.rec[at], g);
    st.pos[at] = idx1 - list_start + 1u;
    st.id[at] = g;
  }
  __syncthreads();
  return (int)(t0 + t1);
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

using FwdStage = Stage<RecPair, kFwdBatch>;

template <int MAXV, bool STATS>
__device__ __forceinline__ void render_tile_fwd(const ViewTable<MAXV>& vt, int64_t tile, FwdStage& st,
                                                const uint2* __restrict__ ranges, const uint32_t* __restrict__ keys,
                                                const uint32_t* __restrict__ vals, const Rec* __restrict__ rec,
                                                const Params& P, unsigned long long* __restrict__ stats) {
  const ViewDesc& vd = vt.v[view_of_tile(vt, tile)];
  const int lt = (int)(tile - vd.tile_base);
  const int tx = lt % vd.tiles_x, ty = lt / vd.tiles_x;
  const WarpBlock wb = warp_block(lt, vd.tiles_x);
  const bool inside0 = wb.x < vd.W && wb.y < vd.H, inside1 = wb.x < vd.W && wb.y + 4 < vd.H;
  // this tile's list: the entries of its segment whose span covers tile offset `to`
  const uint2 rg = ranges[vd.seg_base + ty * vd.segs_x + (tx >> P.seg_log2)];
  const uint32_t to = (uint32_t)tx & ((1u << P.seg_log2) - 1u);
  const float2 PX = make_float2((float)wb.x + 0.5f, (float)wb.x + 0.5f);
  const float2 PY = make_float2((float)wb.y + 0.5f, (float)(wb.y + 4) + 0.5f);
  const float2 ONE = make_float2(1.0f, 1.0f), NEG1 = make_float2(-1.0f, -1.0f), ZERO = make_float2(0.f, 0.f);
  float2 T = ONE, C0 = ZERO, C1 = ZERO, C2 = ZERO;
  uint32_t last0 = 0, last1 = 0, n_eval = 0, n_range = 0, n_comp = 0;
  bool done0 = !inside0, done1 = !inside1;
  for (uint32_t base = rg.x; base < rg.y; base += kFwdBatch) {
    if (__syncthreads_count(done0 && done1) == kFwdThreads) break;
    const uint32_t idx0 = base + threadIdx.x, idx1 = idx0 + kFwdThreads;
    const bool keep0 = idx0 < rg.y && seg_key_covers(keys[idx0], to, P);
    const bool keep1 = idx1 < rg.y && seg_key_covers(keys[idx1], to, P);
    const int cnt = stage_kept2<kFwdThreads>(st, keep0, idx0, keep1, idx1, rg.x, vals,
                                             [&](RecPair& d, uint32_t g) { stage_pair(d, rec[g]); });
    if (!__all_sync(0xffffffffu, done0 && done1)) {
      // full groups of eight staged fragments with one done-test each (a pixel finished inside a group
      // composites nothing more: c0/c1 stay false), then the rest one by one.  At the scene-scale
      // view 0.706 -> 0.579 ms (0.647 with the same loop unrolled but tested per fragment); padding
      // the rounds to whole groups instead cost the cube view 13%, whose rounds stage few entries.
      const int n8 = cnt & ~7;
      for (int j0 = 0; j0 < n8; j0 += 8) {
        if (done0 && done1) break;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int j = j0 + jj;
          PairEval f;
          eval_pair(st.rec[j], PX, PY, f);
          if (STATS) {
            const float ql = rec[st.id[j]].a.z;
            n_eval += (done0 ? 0u : 1u) + (done1 ? 0u : 1u);
            n_range += (!done0 && f.q0 <= ql ? 1u : 0u) + (!done1 && f.q1 <= ql ? 1u : 0u);
          }
          const float2 al = make_float2(fminf(f.a.x, P.alpha_max), fminf(f.a.y, P.alpha_max));
          const float2 Tn = __fmul2_rn(T, __ffma2_rn(al, NEG1, ONE));
          bool c0 = !done0 && al.x >= P.alpha_min;
          bool c1 = !done1 && al.y >= P.alpha_min;
          const bool s0 = c0 && Tn.x < P.t_min, s1 = c1 && Tn.y < P.t_min;
          done0 = done0 || s0;
          done1 = done1 || s1;
          c0 = c0 && !s0;
          c1 = c1 && !s1;
          // composite: alpha is zero for a pixel that does not take this fragment, so T and C stay
          const float2 alpha = make_float2(c0 ? al.x : 0.f, c1 ? al.y : 0.f);
          const float2 wgt = __fmul2_rn(alpha, T);
          T = __fmul2_rn(T, __ffma2_rn(alpha, NEG1, ONE));
          const float4 k0 = st.rec[j].k0, k1 = st.rec[j].k1;
          C0 = __ffma2_rn(lo2(k0), wgt, C0);
          C1 = __ffma2_rn(hi2(k0), wgt, C1);
          C2 = __ffma2_rn(lo2(k1), wgt, C2);
          const uint32_t kpos = st.pos[j];
          last0 = c0 ? kpos : last0;
          last1 = c1 ? kpos : last1;
          if (STATS) n_comp += (c0 ? 1u : 0u) + (c1 ? 1u : 0u);
        }
      }
#pragma unroll 4
      for (int j = n8; j < cnt; ++j) {
        if (done0 && done1) break;
        PairEval f;
        eval_pair(st.rec[j], PX, PY, f);
        if (STATS) {
          const float ql = rec[st.id[j]].a.z;
          n_eval += (done0 ? 0u : 1u) + (done1 ? 0u : 1u);
          n_range += (!done0 && f.q0 <= ql ? 1u : 0u) + (!done1 && f.q1 <= ql ? 1u : 0u);
        }
        const float2 al = make_float2(fminf(f.a.x, P.alpha_max), fminf(f.a.y, P.alpha_max));
        const float2 Tn = __fmul2_rn(T, __ffma2_rn(al, NEG1, ONE));
        bool c0 = !done0 && al.x >= P.alpha_min;
        bool c1 = !done1 && al.y >= P.alpha_min;
        const bool s0 = c0 && Tn.x < P.t_min, s1 = c1 && Tn.y < P.t_min;
        done0 = done0 || s0;
        done1 = done1 || s1;
        c0 = c0 && !s0;
        c1 = c1 && !s1;
        // composite: alpha is zero for a pixel that does not take this fragment, so T and C stay
        const float2 alpha = make_float2(c0 ? al.x : 0.f, c1 ? al.y : 0.f);
        const float2 wgt = __fmul2_rn(alpha, T);
        T = __fmul2_rn(T, __ffma2_rn(alpha, NEG1, ONE));
        const float4 k0 = st.rec[j].k0, k1 = st.rec[j].k1;
        C0 = __ffma2_rn(lo2(k0), wgt, C0);
        C1 = __ffma2_rn(hi2(k0), wgt, C1);
        C2 = __ffma2_rn(lo2(k1), wgt, C2);
        const uint32_t kpos = st.pos[j];
        last0 = c0 ? kpos : last0;
        last1 = c1 ? kpos : last1;
        if (STATS) n_comp += (c0 ? 1u : 0u) + (c1 ? 1u : 0u);
      }
    }
  }
  const int64_t plane = (int64_t)vd.W * vd.H;
  if (inside0) {
    const int64_t pix = (int64_t)wb.y * vd.W + wb.x;
    vd.img[pix] = C0.x + T.x * vd.bg[0];
    vd.img[plane + pix] = C1.x + T.x * vd.bg[1];
    vd.img[2 * plane + pix] = C2.x + T.x * vd.bg[2];
    vd.final_T[pix] = T.x;
    vd.n_contrib[pix] = last0;
  }
  if (inside1) {
    const int64_t pix = (int64_t)(wb.y + 4) * vd.W + wb.x;
    vd.img[pix] = C0.y + T.y * vd.bg[0];
    vd.img[plane + pix] = C1.y + T.y * vd.bg[1];
    vd.img[2 * plane + pix] = C2.y + T.y * vd.bg[2];
    vd.final_T[pix] = T.y;
    vd.n_contrib[pix] = last1;
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
// seven CTAs per SM: at 72 registers the forward keeps its values in registers (eight CTAs
// capped it at 64 with spills: 0.566 against 0.555 ms at the scene-scale view)
__global__ void __launch_bounds__(kFwdThreads, 7) k_render_fwd(const __grid_constant__ VS vs, const uint2* __restrict__ ranges,
                                                            const uint32_t* __restrict__ keys,
                                                            const uint32_t* __restrict__ vals, const Rec* __restrict__ rec,
                                                            const Params P, unsigned long long* __restrict__ stats) {
  __shared__ FwdStage st;
  render_tile_fwd<VS::kMax, STATS>(vs.get(), (int64_t)blockIdx.x, st, ranges, keys, vals, rec, P, stats);
}

// Persistent form: CTAs take tiles from a work counter until the table's total_tiles are done, so
// a fixed grid serves batches of any size (the launch can be replayed from a captured graph).
template <class VS>
__global__ void __launch_bounds__(kFwdThreads, 7) k_render_fwd_persistent(const __grid_constant__ VS vs,
                                                                    const uint2* __restrict__ ranges,
                                                                    const uint32_t* __restrict__ keys,
                                                                    const uint32_t* __restrict__ vals,
                                                                    const Rec* __restrict__ rec, const Params P,
                                                                    unsigned int* __restrict__ tile_counter) {
  __shared__ FwdStage st;
  __shared__ unsigned int s_tile;
  const auto& vt = vs.get();
  const long long total = vt.total_tiles;
  for (;;) {
    __syncthreads();  // previous tile's readers of s_tile and the staged list are done
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const unsigned int tile = s_tile;
    if ((long long)tile >= total) break;
    render_tile_fwd<VS::kMax, false>(vt, (int64_t)tile, st, ranges, keys, vals, rec, P, nullptr);
  }
}

// Sums 10 per-lane values over the warp with a reduce-scatter butterfly: at each step a lane keeps
// half of its values (the odd one out padded with a zero) and receives the partner's copy of that
// half, 12 shuffles in all.  On return the lane holds the full sum of value reduce10_slot(lane), or
// of a padding zero where that is -1; lanes L and L^1 hold the same.
__device__ __forceinline__ float warp_reduce_scatter10(float (&v)[10]) {
  const unsigned lane = threadIdx.x & 31u;
  const bool u16 = lane & 16u, u8 = lane & 8u, u4 = lane & 4u, u2 = lane & 2u;
#pragma unroll
  for (int k = 0; k < 5; ++k) {  // 10 -> 5: lower half keeps 0..4, upper keeps 5..9
    const float send = u16 ? v[k] : v[k + 5];
    const float keep = u16 ? v[k + 5] : v[k];
    v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {  // 5 (+1 zero) -> 3
    const float hi = k + 3 < 5 ? v[k + 3] : 0.0f;
    const float send = u8 ? v[k] : hi;
    const float keep = u8 ? hi : v[k];
    w[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float x[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {  // 3 (+1 zero) -> 2
    const float hi = k + 2 < 3 ? w[k + 2] : 0.0f;
    const float send = u4 ? w[k] : hi;
    const float keep = u4 ? hi : w[k];
    x[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  const float send = u2 ? x[0] : x[1];
  const float keep = u2 ? x[1] : x[0];
  const float y = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  return y + __shfl_xor_sync(0xffffffffu, y, 1);
}

// which of the 10 values warp_reduce_scatter10 leaves on a lane (-1: a padding zero)
__device__ __forceinline__ int reduce10_slot(unsigned lane) {
  const int t3 = ((lane & 4u) ? 2 : 0) + ((lane & 2u) ? 1 : 0);  // position among the kept three
  if (t3 > 2) return -1;
  const int p6 = ((lane & 8u) ? 3 : 0) + t3;                      // position among the kept five
  if (p6 > 4) return -1;
  return ((lane & 16u) ? 5 : 0) + p6;
}

// Backward.  Per pixel, walks its contributors back to front, recovering T_i = T_{i+1}/(1-alpha_i)
// from the saved final transmittance; S is the colour composited behind the current fragment.
//   dC/dalpha_i = c_i T_i - S_i / (1 - alpha_i)   (summed over the channels against dL/dC)
//   dalpha/dkappa = G, dalpha/dG = kappa (0 where alpha is clamped)
//   dG/dp = -G/2,  p = q^hb:  dp/dq = hb p / q,  dp/dhb = p ln q  (0 for q < 1e-12)
//   q = a dx^2 + 2 b dx dy + c dy^2, dx = px - mx
// A thread's two pixels share x and the fragment, so their arithmetic runs as float2 pairs (one
// packed instruction for both).  The fragment test is eval_pair, as in the forward, so the skip /
// clamp / stop decisions equal the forward's bit for bit.  A thread sums
// its two pixels' terms, the warp sums by a reduce-scatter butterfly, and ten lanes add the ten
// per-primitive sums with one predicated atomic each.  Reciprocals use the approximate MUFU
// instruction (about 1 ulp); they only scale gradients, never decide a branch.  The falloff mode is
// a template parameter, so the Gaussian form carries no exponent path and no mode branch.
template <class VS, bool GEF>
__global__ void __launch_bounds__(kThreads) k_render_bwd(const __grid_constant__ VS vs, const uint2* __restrict__ ranges,
                                                         const uint32_t* __restrict__ keys,
                                                         const uint32_t* __restrict__ vals, const Rec* __restrict__ rec,
                                                         const Params P, float4* __restrict__ g2d,
                                                         const uint32_t* __restrict__ order) {
  __shared__ Stage<RecPairB, kBatch> st;
  __shared__ uint32_t s_max_last;
  const auto& vt = vs.get();
  const int64_t tile = order ? (int64_t)order[blockIdx.x] : (int64_t)blockIdx.x;
  if (tile >= (int64_t)vt.total_tiles) return;  // (order is a permutation of the tiles)
  const ViewDesc& vd = vt.v[view_of_tile(vt, tile)];
  const int lt = (int)(tile - vd.tile_base);
  const int tx = lt % vd.tiles_x, ty = lt / vd.tiles_x;
  const WarpBlock wb = warp_block(lt, vd.tiles_x);
  const uint2 rg = ranges[vd.seg_base + ty * vd.segs_x + (tx >> P.seg_log2)];
  const uint32_t to = (uint32_t)tx & ((1u << P.seg_log2) - 1u);
  const int64_t plane = (int64_t)vd.W * vd.H;

  float Tk[2], gc[3][2];
  uint32_t last[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int y = wb.y + 4 * k;
    const bool inside = wb.x < vd.W && y < vd.H;
    Tk[k] = 0.f;
    gc[0][k] = gc[1][k] = gc[2][k] = 0.f;
    last[k] = 0;
    if (inside) {
      const int64_t pix = (int64_t)y * vd.W + wb.x;
      Tk[k] = vd.final_T[pix];
      last[k] = vd.n_contrib[pix];
      gc[0][k] = vd.dL_dimg[pix];
      gc[1][k] = vd.dL_dimg[plane + pix];
      gc[2][k] = vd.dL_dimg[2 * plane + pix];
    }
  }
  const float2 PX = make_float2((float)wb.x + 0.5f, (float)wb.x + 0.5f);
  const float2 PY = make_float2((float)wb.y + 0.5f, (float)(wb.y + 4) + 0.5f);
  const float2 GC0 = make_float2(gc[0][0], gc[0][1]), GC1 = make_float2(gc[1][0], gc[1][1]),
               GC2 = make_float2(gc[2][0], gc[2][1]);
  float2 T = make_float2(Tk[0], Tk[1]);
  // U = sum_c dL/dC_c S_c, S_c the colour composited behind the current fragment (at the start,
  // T_final bg_c): dL/dalpha_i needs S only through this sum, so one float2 carries it.
  float2 U = __fmul2_rn(T, __ffma2_rn(GC2, make_float2(vd.bg[2], vd.bg[2]),
                                      __ffma2_rn(GC1, make_float2(vd.bg[1], vd.bg[1]),
                                                 __fmul2_rn(GC0, make_float2(vd.bg[0], vd.bg[0])))));
  if (threadIdx.x == 0) s_max_last = 0;
  __syncthreads();
  atomicMax(&s_max_last, max(last[0], last[1]));
  __syncthreads();
  const uint32_t max_last = s_max_last;
  const uint32_t wlast = __reduce_max_sync(0xffffffffu, max(last[0], last[1]));
  constexpr bool gef = GEF;
  const unsigned lane = threadIdx.x & 31u;
  const int slot = reduce10_slot(lane);
  const bool adder = (lane & 1u) == 0 && slot >= 0;
  // the constant factor each summed value still lacks (see the loop)
  const float kSlotScale[10] = {1.0f, 1.0f, -0.5f, -1.0f, -0.5f, 1.0f, -0.34657359027997264f, 1.0f, 1.0f, 1.0f};
  float slot_scale = 1.0f;
#pragma unroll
  for (int k = 0; k < 10; ++k) slot_scale = slot == k ? kSlotScale[k] : slot_scale;
  const float2 ONE = make_float2(1.0f, 1.0f), NEG1 = make_float2(-1.0f, -1.0f), ZERO = make_float2(0.f, 0.f);

  for (uint32_t end = rg.x + max_last; end > rg.x;) {
    const uint32_t start = (end - rg.x > (uint32_t)kBatch) ? end - kBatch : rg.x;
    __syncthreads();  // the previous round's readers of the staged list are done
    const uint32_t idx = start + threadIdx.x;
    const bool keep = idx < end && seg_key_covers(keys[idx], to, P);
    const int cnt = stage_kept<kBatch>(st, keep, idx, rg.x, vals, [&](RecPairB& d, uint32_t g) {
      const Rec r = rec[g];
      stage_pair(d, r);
      d.nb = make_float2(r.b.y, r.b.y);
    });
    for (int j = cnt - 1; j >= 0; --j) {
      const uint32_t kpos = st.pos[j];  // 1-based position in the segment's list
      if (kpos > wlast) continue;       // beyond every pixel of this warp
      PairEval f;
      eval_pair(st.rec[j], PX, PY, f);
      const bool cl0 = f.a.x > P.alpha_max, cl1 = f.a.y > P.alpha_max;
      const float al0 = cl0 ? P.alpha_max : f.a.x, al1 = cl1 ? P.alpha_max : f.a.y;
      const bool act0 = kpos <= last[0] && al0 >= P.alpha_min;
      const bool act1 = kpos <= last[1] && al1 >= P.alpha_min;
      if (!__any_sync(0xffffffffu, act0 || act1)) continue;
      // gradient terms of both pixels (zero for an inactive one, whose T and S stay as they are).
      // Constant factors are left out here and applied to the warp's sums (slot_scale): the
      // derivative of G = 2^(-p log2(e)/2) w.r.t. p is taken as G (true: -G/2), the record's conic
      // terms as (a, b, c) (true: -2 (a, b, c)), 2 dx dy as dx dy, and ln q as log2 q.
      const float4 c0 = st.rec[j].c0, k0 = st.rec[j].k0, k1 = st.rec[j].k1;
      const float2 nb = st.rec[j].nb;
      const float4 e = st.rec[j].k1, c1 = st.rec[j].c1;  // e.z, e.w: beta/2
      const float2 dx = f.dx, dy = f.dy, p = f.p, lq = f.lq, G = f.G;
      const float q0 = f.q0, q1 = f.q1, hb = e.z;
      const float2 alpha = make_float2(act0 ? al0 : 0.f, act1 ? al1 : 0.f);
      const float2 om = __ffma2_rn(alpha, NEG1, ONE);
      // an inactive pixel has alpha = 0, om = 1 and rcp(1) = 1: its T stays as it is
      const float2 inv = make_float2(rcp_approx(om.x), rcp_approx(om.y));
      T = __fmul2_rn(T, inv);
      const float2 w = __fmul2_rn(alpha, T);
      // D = sum_c dL/dC_c c_c;  dL/dalpha = D T_i - U / (1 - alpha_i);  U += D alpha_i T_i
      const float2 D = __ffma2_rn(GC2, lo2(k1), __ffma2_rn(GC1, hi2(k0), __fmul2_rn(GC0, lo2(k0))));
      const float2 dLda_all = __ffma2_rn(U, make_float2(-inv.x, -inv.y), __fmul2_rn(D, T));
      // dalpha/dG = kappa and dalpha/dkappa = G, both 0 where alpha is clamped or the pixel inactive
      const float2 dLdaG = sel2(act0 && !cl0, act1 && !cl1, dLda_all, ZERO);
      U = __ffma2_rn(D, w, U);
      const float2 gr = __fmul2_rn(GC0, w), gg = __fmul2_rn(GC1, w), gbl = __fmul2_rn(GC2, w);
      const float2 gk = __fmul2_rn(dLdaG, G);
      const float2 dp = __fmul2_rn(gk, hi2(c1));  // x (-1/2)
      float2 dq, gbeta = ZERO;
      if (gef) {
        // only where the pixel takes the fragment (elsewhere p may overflow) and q > 1e-12
        const bool m0 = act0 && q0 > 1e-12f, m1 = act1 && q1 > 1e-12f;
        if (hb == 1.0f) {
          dq = sel2(m0, m1, dp, ZERO);
          const float2 l2 = make_float2(m0 ? mufu_lg2(q0) : 0.f, m1 ? mufu_lg2(q1) : 0.f);
          gbeta = __fmul2_rn(__fmul2_rn(dq, make_float2(q0, q1)), l2);  // x (-ln 2 / 2)
        } else {
          const float2 rq = make_float2(rcp_approx(q0), rcp_approx(q1));
          const float2 dpp = __fmul2_rn(dp, p);
          dq = sel2(m0, m1, __fmul2_rn(__fmul2_rn(dpp, hi2(e)), rq), ZERO);
          gbeta = sel2(m0, m1, __fmul2_rn(dpp, lq), ZERO);                // x (-ln 2 / 2)
        }
      } else {
        dq = dp;
      }
      const float2 dqdx = __fmul2_rn(dq, dx), dqdy = __fmul2_rn(dq, dy);
      const float2 gmx = __ffma2_rn(dqdy, nb, __fmul2_rn(dqdx, lo2(c0)));
      const float2 gmy = __ffma2_rn(dqdy, lo2(c1), __fmul2_rn(dqdx, nb));
      const float2 ga = __fmul2_rn(dqdx, dx);   // x (-1/2)
      const float2 gb = __fmul2_rn(dqdx, dy);   // x (-1)
      const float2 gcc = __fmul2_rn(dqdy, dy);  // x (-1/2)
      float v[10] = {gmx.x + gmx.y, gmy.x + gmy.y, ga.x + ga.y,   gb.x + gb.y,   gcc.x + gcc.y,
                     gk.x + gk.y,   gbeta.x + gbeta.y, gr.x + gr.y, gg.x + gg.y, gbl.x + gbl.y};
      const float sum = warp_reduce_scatter10(v);
      {  // ten lanes add their sums: a predicated reduction, no divergent branch
        float* dst = reinterpret_cast<float*>(g2d + 3 * (int64_t)st.id[j]) + slot;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n @p red.global.add.f32 [%0], %1;\n}"
                     :: "l"(dst), "f"(sum * slot_scale), "r"((int)adder) : "memory");
      }
    }
    end = start;
  }
}

// The backward's tiles, heaviest first.  Tiles run in launch order as CTA slots free up, so with
// the row-major order the heavy tiles of the image's middle meet the last wave and the kernel ends
// on a few of them; longest-first keeps the SMs busy to the end.  A tile's cost is the sum over its
// four 8x8 warp blocks of the block's largest n_contrib (each warp walks the list that far), plus
// a constant for the staging; classes of 8 per octave are ordered by a counting sort (the order
// inside a class follows the atomics, which changes nothing but the order of the gradient sums).
template <class VS>
__global__ void __launch_bounds__(kThreads) k_tile_cost(const __grid_constant__ VS vs, uint32_t* __restrict__ bucket,
                                                        uint32_t* __restrict__ counts) {
  __shared__ uint32_t s_cost;
  const auto& vt = vs.get();
  const int64_t tile = blockIdx.x;
  const ViewDesc& vd = vt.v[view_of_tile(vt, tile)];
  const WarpBlock wb = warp_block((int)(tile - vd.tile_base), vd.tiles_x);
  uint32_t m = 0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int y = wb.y + 4 * k;
    if (wb.x < vd.W && y < vd.H) m = max(m, vd.n_contrib[(int64_t)y * vd.W + wb.x]);
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if (threadIdx.x == 0) s_cost = 0;
  __syncthreads();
  if ((threadIdx.x & 31u) == 0) atomicAdd(&s_cost, m);
  __syncthreads();
  if (threadIdx.x == 0) {
    const float c = (float)s_cost + 16.0f;
    const int b = min(kOrderBuckets - 1, (int)(log2f(c) * 8.0f));
    bucket[tile] = (uint32_t)b;
    atomicAdd(&counts[b], 1u);
  }
}

// order[start(b) + i] = the i-th tile of class b to arrive, start(b) = the tiles of heavier classes
__global__ void __launch_bounds__(kThreads) k_tile_order(int64_t total, const uint32_t* __restrict__ bucket,
                                                         uint32_t* __restrict__ counts, uint32_t* __restrict__ order) {
  __shared__ uint32_t start[kOrderBuckets];
  for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) start[b] = counts[b];
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive scan from the heaviest class down, 8 classes per lane
    const unsigned lane = threadIdx.x;
    uint32_t v[kOrderBuckets / 32], sum = 0;
#pragma unroll
    for (int k = 0; k < kOrderBuckets / 32; ++k) {
      v[k] = start[kOrderBuckets - 1 - (int)(lane * (kOrderBuckets / 32) + k)];
      sum += v[k];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if ((int)lane >= o) inc += y;
    }
    uint32_t run = inc - sum;
    __syncwarp();
#pragma unroll
    for (int k = 0; k < kOrderBuckets / 32; ++k) {
      start[kOrderBuckets - 1 - (int)(lane * (kOrderBuckets / 32) + k)] = run;
      run += v[k];
    }
  }
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < total) {
    const uint32_t b = bucket[t];
    const uint32_t pos = start[b] + atomicAdd(&counts[kOrderBuckets + b], 1u);
    if ((int64_t)pos < total) order[pos] = (uint32_t)t;
  }
}

}  // namespace

template <class VS>
void launch_tile_order(const VS& vs, int64_t total_tiles, uint32_t* bucket, uint32_t* counts, uint32_t* order,
                       cudaStream_t s) {
  if (total_tiles <= 0) return;
  cudaMemsetAsync(counts, 0, sizeof(uint32_t) * 2 * kOrderBuckets, s);
  k_tile_cost<VS><<<(unsigned)total_tiles, kThreads, 0, s>>>(vs, bucket, counts);
  k_tile_order<<<(unsigned)((total_tiles + kThreads - 1) / kThreads), kThreads, 0, s>>>(total_tiles, bucket, counts,
                                                                                          order);
  count_launches(2);
}

template <class VS>
void launch_render_fwd(const VS& vs, int64_t total_tiles, const uint2* ranges, const uint32_t* keys,
                       const uint32_t* vals, const Rec* rec, const Params& P, cudaStream_t s,
                       unsigned long long* stats, unsigned int* tile_counter, int num_sms) {
  if (total_tiles <= 0) return;
  if (tile_counter) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_fwd_persistent<VS>, kFwdThreads, 0);
    const int64_t grid = (int64_t)num_sms * (per_sm > 0 ? per_sm : 1);
    k_render_fwd_persistent<VS><<<(unsigned)(grid < total_tiles ? grid : total_tiles), kFwdThreads, 0, s>>>(
        vs, ranges, keys, vals, rec, P, tile_counter);
  } else if (stats) {
    k_render_fwd<VS, true><<<(unsigned)total_tiles, kFwdThreads, 0, s>>>(vs, ranges, keys, vals, rec, P, stats);
  } else {
    k_render_fwd<VS, false><<<(unsigned)total_tiles, kFwdThreads, 0, s>>>(vs, ranges, keys, vals, rec, P, nullptr);
  }
  count_launches(1);
}

template <class VS>
void launch_render_bwd(const VS& vs, int64_t total_tiles, const uint2* ranges, const uint32_t* keys,
                       const uint32_t* vals, const Rec* rec, const Params& P, float4* g2d, cudaStream_t s,
                       const uint32_t* order) {
  if (total_tiles <= 0) return;
  if (P.mode == 0)
    k_render_bwd<VS, true><<<(unsigned)total_tiles, kThreads, 0, s>>>(vs, ranges, keys, vals, rec, P, g2d, order);
  else
    k_render_bwd<VS, false><<<(unsigned)total_tiles, kThreads, 0, s>>>(vs, ranges, keys, vals, rec, P, g2d, order);
  count_launches(1);
}

template void launch_render_fwd<FrameViews>(const FrameViews&, int64_t, const uint2*, const uint32_t*, const uint32_t*,
                                            const Rec*, const Params&, cudaStream_t, unsigned long long*, unsigned int*,
                                            int);
template void launch_render_fwd<BatchViews>(const BatchViews&, int64_t, const uint2*, const uint32_t*, const uint32_t*,
                                            const Rec*, const Params&, cudaStream_t, unsigned long long*, unsigned int*,
                                            int);
template void launch_render_bwd<FrameViews>(const FrameViews&, int64_t, const uint2*, const uint32_t*, const uint32_t*,
                                            const Rec*, const Params&, float4*, cudaStream_t, const uint32_t*);
template void launch_tile_order<FrameViews>(const FrameViews&, int64_t, uint32_t*, uint32_t*, uint32_t*, cudaStream_t);

}  // namespace ges
