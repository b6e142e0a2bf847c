// Training-side updates over the primitives' SoA parameters (Sec. 4.4; App. B.2): the fused Adam
// step, the densification statistics, density control (clone, split, prune) and the opacity and
// shape resets.  The paper keeps Gaussian splatting's optimisation and density control and adds
// the shape reset and shape pruning; App. B.2 lists the constants.
//
// The optimizer's variables (group: activation): means (identity), log-scales (exp), quaternions
// (identity; the rasterizer normalises), shapes shifted by -2 (beta = p + 2), opacity logits
// (sigmoid), SH coefficients (identity).
//
// Adam: one launch over all six groups, four elements per thread (16-byte loads and stores), with
// the activation's chain rule in front and the new physical value written behind, so each element
// costs one pass: read p, m, v, g and write p, m, v, phys (32 bytes).  HBM-bound.
// Density control: a classification kernel (one thread per row), three exclusive scans of the
// keep / clone / child flags, one host read of the totals, a copy kernel per group (one thread per
// element, coalesced reads) and a kernel that places the split children.
#include <cmath>
#include <cstring>

#include "api_internal.h"

namespace ges {
namespace {

constexpr int kG = 6;
constexpr int kThreads = 256;

// activation per group: 0 identity, 1 exp, 2 shift by 2, 3 sigmoid
__host__ __device__ constexpr int group_act(int g) { return g == 1 ? 1 : (g == 3 ? 2 : (g == 4 ? 3 : 0)); }

__device__ __forceinline__ float act(int a, float x) {
  if (a == 1) return expf(x);
  if (a == 2) return x + 2.0f;
  if (a == 3) return 1.0f / (1.0f + expf(-x));
  return x;
}
// d act / dx; the sigmoid's as e^-|x| / (1 + e^-|x|)^2, which does not cancel for large |x|
__device__ __forceinline__ float dact(int a, float x) {
  if (a == 1) return expf(x);
  if (a == 3) {
    const float t = expf(-fabsf(x));
    return t / ((1.0f + t) * (1.0f + t));
  }
  return 1.0f;
}

struct AdamArgs {
  float* p[kG];
  float* m[kG];
  float* v[kG];
  const float* g[kG];
  float* phys[kG];
  int64_t count[kG];          // elements per group
  int64_t quad0[kG + 1];      // first 4-element chunk of each group (prefix sums); quad0[kG] = total
  float lr[kG];               // lr[5]: SH DC terms
  float lr_rest;              // SH terms of degree >= 1
  int32_t sh_row;             // SH values per primitive (3 (d+1)^2)
  float b1, b2, eps;
  float ic1, isc2;            // 1 / (1 - b1^step), 1 / sqrt(1 - b2^step)
  int32_t adam;               // 0: only write phys = act(p) (ges_activate)
};

// x <- x - lr m^ / (sqrt(v^) + eps) with m^ = m / (1 - b1^t), sqrt(v^) = sqrt(v) / sqrt(1 - b2^t)
__device__ __forceinline__ void adam_one(const AdamArgs& A, int a, float lr, float& p, float& m, float& v, float g,
                                         float& out) {
  if (A.adam) {
    const float gr = g * dact(a, p);
    m = A.b1 * m + (1.0f - A.b1) * gr;
    v = A.b2 * v + (1.0f - A.b2) * (gr * gr);
    p = p - (lr * A.ic1) * m / (sqrtf(v) * A.isc2 + A.eps);
  }
  out = act(a, p);
}

// the learning rate of element e0 + j of group grp; col0 = e0 mod (values per SH row) for the SH group
__device__ __forceinline__ float lr_of(const AdamArgs& A, int grp, int col0, int j) {
  if (grp != 5) return A.lr[grp];
  int c = col0 + j;
  if (c >= A.sh_row) c -= A.sh_row;  // col0 + j < 2 sh_row, as j <= 3 <= sh_row
  return c < 3 ? A.lr[5] : A.lr_rest;
}

__global__ void __launch_bounds__(kThreads) k_adam(const __grid_constant__ AdamArgs A) {
  const int64_t total = A.quad0[kG];
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int grp = 0;
    while (grp < kG - 1 && q >= A.quad0[grp + 1]) ++grp;
    const int a = group_act(grp);
    const int64_t e0 = (q - A.quad0[grp]) * 4;
    const int64_t rem = A.count[grp] - e0;
    int col0 = 0;
    if (grp == 5) col0 = e0 < 0x7fffffffLL ? (int)((uint32_t)e0 % (uint32_t)A.sh_row) : (int)(e0 % A.sh_row);
    if (rem >= 4) {
      float4 p = *reinterpret_cast<const float4*>(A.p[grp] + e0);
      float4 m = make_float4(0.f, 0.f, 0.f, 0.f), v = m, g = m, o;
      if (A.adam) {
        m = *reinterpret_cast<const float4*>(A.m[grp] + e0);
        v = *reinterpret_cast<const float4*>(A.v[grp] + e0);
        g = *reinterpret_cast<const float4*>(A.g[grp] + e0);
      }
      adam_one(A, a, lr_of(A, grp, col0, 0), p.x, m.x, v.x, g.x, o.x);
      adam_one(A, a, lr_of(A, grp, col0, 1), p.y, m.y, v.y, g.y, o.y);
      adam_one(A, a, lr_of(A, grp, col0, 2), p.z, m.z, v.z, g.z, o.z);
      adam_one(A, a, lr_of(A, grp, col0, 3), p.w, m.w, v.w, g.w, o.w);
      if (A.adam) {
        *reinterpret_cast<float4*>(A.p[grp] + e0) = p;
        *reinterpret_cast<float4*>(A.m[grp] + e0) = m;
        *reinterpret_cast<float4*>(A.v[grp] + e0) = v;
      }
      *reinterpret_cast<float4*>(A.phys[grp] + e0) = o;
    } else {
      for (int64_t e = e0; e < A.count[grp]; ++e) {
        float p = A.p[grp][e], m = 0.f, v = 0.f, g = 0.f, o;
        if (A.adam) {
          m = A.m[grp][e];
          v = A.v[grp][e];
          g = A.g[grp][e];
        }
        adam_one(A, a, lr_of(A, grp, col0, (int)(e - e0)), p, m, v, g, o);
        if (A.adam) {
          A.p[grp][e] = p;
          A.m[grp][e] = m;
          A.v[grp][e] = v;
        }
        A.phys[grp][e] = o;
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_densify_stats(const uint32_t* __restrict__ depth_key,
                                                            const float4* __restrict__ g2d, int64_t n, float sx,
                                                            float sy, float* __restrict__ acc,
                                                            int32_t* __restrict__ cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (depth_key[i] == kCulledKey) continue;
    const float4 a = g2d[3 * i];
    const float gx = a.x * sx, gy = a.y * sy;
    acc[i] += sqrtf(gx * gx + gy * gy);
    cnt[i] += 1;
  }
}

struct DensArgs {
  int64_t n;
  int32_t width[kG];
  const float* in[kG];
  const float* in_m[kG];
  const float* in_v[kG];
  float* out[kG];
  float* out_m[kG];
  float* out_v[kG];
  const float* acc;
  const int32_t* cnt;
  const float* xi;
  float t_grad, t_small, t_opac, t_beta, t_big, t_split;
  uint8_t* kind;              // bit 0 keep, bit 1 clone, bit 2 children
  uint32_t* pos[3];           // 0/1 flags, then their exclusive scans
  int64_t base[4];            // first output row of the kept rows, clones, first and second children
};

__global__ void __launch_bounds__(kThreads) k_density_classify(const __grid_constant__ DensArgs D) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float* ls = D.in[1] + 3 * i;
    const float l0 = ls[0], l1 = ls[1], l2 = ls[2];
    const float lmax = fmaxf(fmaxf(l0, l1), l2);
    const int32_t c = D.cnt[i] > 1 ? D.cnt[i] : 1;
    const float g = __fdiv_rn(D.acc[i], (float)c);
    const bool sel = g >= D.t_grad;
    const bool small = lmax <= D.t_small;
    const bool prune = D.in[4][i] < D.t_opac || D.in[3][i] < D.t_beta;
    const bool big = lmax > D.t_big;
    const float lc = fmaxf(fmaxf(__fsub_rn(l0, D.t_split), __fsub_rn(l1, D.t_split)), __fsub_rn(l2, D.t_split));
    const bool big_child = lc > D.t_big;
    const bool split = sel && !small;
    const bool clone = sel && small && !prune && !big;
    const bool keep = !split && !prune && !big;
    const bool child = split && !prune && !big_child;
    D.kind[i] = (uint8_t)((keep ? 1 : 0) | (clone ? 2 : 0) | (child ? 4 : 0));
    D.pos[0][i] = keep ? 1u : 0u;
    D.pos[1][i] = clone ? 1u : 0u;
    D.pos[2][i] = child ? 1u : 0u;
  }
}

// copies group `grp` (w values per row) into its places; new rows get zero moments
__global__ void __launch_bounds__(kThreads) k_density_copy(const __grid_constant__ DensArgs D, int grp) {
  const int w = D.width[grp];
  const int64_t total = D.n * w;
  const float* in = D.in[grp];
  const float* im = D.in_m[grp];
  const float* iv = D.in_v[grp];
  float* out = D.out[grp];
  float* om = D.out_m[grp];
  float* ov = D.out_v[grp];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / w;
    const int c = (int)(e - i * w);
    const unsigned k = D.kind[i];
    if (!k) continue;
    const float x = in[e];
    if (k & 1u) {
      const int64_t o = (D.base[0] + D.pos[0][i]) * w + c;
      out[o] = x;
      om[o] = im[e];
      ov[o] = iv[e];
    }
    if (k & 2u) {
      const int64_t o = (D.base[1] + D.pos[1][i]) * w + c;
      out[o] = x;
      om[o] = 0.f;
      ov[o] = 0.f;
    }
    if (k & 4u) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int64_t o = (D.base[2 + j] + D.pos[2][i]) * w + c;
        out[o] = x;
        om[o] = 0.f;
        ov[o] = 0.f;
      }
    }
  }
}

// the split children's means mu + R(q)(s * xi_j) and log-scales l - log 1.6 (after k_density_copy)
__global__ void __launch_bounds__(kThreads) k_density_children(const __grid_constant__ DensArgs D) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D.n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!(D.kind[i] & 4u)) continue;
    const float* mu = D.in[0] + 3 * i;
    const float* ls = D.in[1] + 3 * i;
    const float4 q4 = *reinterpret_cast<const float4*>(D.in[2] + 4 * i);
    const float rn = 1.0f / sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float w = q4.x * rn, x = q4.y * rn, y = q4.z * rn, z = q4.w * rn;
    const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                        2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                        2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    const float s[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float* xi = D.xi + (2 * i + j) * 3;
      const float d[3] = {s[0] * xi[0], s[1] * xi[1], s[2] * xi[2]};
      const int64_t o = D.base[2 + j] + D.pos[2][i];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        D.out[0][3 * o + r] = mu[r] + (R[3 * r] * d[0] + R[3 * r + 1] * d[1] + R[3 * r + 2] * d[2]);
        D.out[1][3 * o + r] = __fsub_rn(ls[r], D.t_split);
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_reset(float* __restrict__ p, float* __restrict__ m,
                                                    float* __restrict__ v, int64_t n, int clamp, float val) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    p[i] = clamp ? fminf(p[i], val) : val;
    m[i] = 0.f;
    v[i] = 0.f;
  }
}

// ---------------------------------------------------------------- host helpers
int64_t group_width(int g, int sh_degree) {
  static const int w[5] = {3, 3, 4, 1, 1};
  return g < 5 ? w[g] : 3 * (int64_t)(sh_degree + 1) * (sh_degree + 1);
}

bool aligned16(const void* p) { return (((uintptr_t)p) & 15u) == 0; }

ges_status check_set(const ges_train_set* t, const char* what) {
  if (!t) return fail(GES_ERR_INVALID_ARG, "%s is NULL", what);
  if (t->n < 0 || t->n > 0x7fffffffLL) return fail(GES_ERR_INVALID_ARG, "%s: n = %lld out of range", what, (long long)t->n);
  if (t->sh_degree < 0 || t->sh_degree > 3) return fail(GES_ERR_INVALID_ARG, "%s: sh_degree %d", what, t->sh_degree);
  if (t->n == 0) return GES_OK;
  for (int g = 0; g < kG; ++g) {
    if (!t->param[g] || !t->m[g] || !t->v[g]) return fail(GES_ERR_INVALID_ARG, "%s: group %d pointer is NULL", what, g);
    if (!aligned16(t->param[g]) || !aligned16(t->m[g]) || !aligned16(t->v[g]))
      return fail(GES_ERR_INVALID_ARG, "%s: group %d pointer is not 16-byte aligned", what, g);
  }
  return GES_OK;
}

// blocks for a grid-stride kernel over `items`: at most one wave of resident blocks, so that every
// block gets the same share and none waits for a second wave
template <class Kernel>
unsigned grid_for(const ges_ctx* ctx, Kernel kernel, int64_t items) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int64_t cap = (int64_t)ctx->num_sms * per_sm;
  const int64_t b = (items + kThreads - 1) / kThreads;
  return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap));
}

ges_status run_adam(ges_ctx* ctx, const ges_train_set* set, const ges_grads* grads, const ges_scene_out* phys,
                    const ges_adam_params* hp, int64_t step, void* stream, bool adam) {
  if (!ctx || !phys) return fail(GES_ERR_INVALID_ARG, "NULL argument");
  ges_status st;
  if ((st = check_set(set, "set")) != GES_OK) return st;
  float* ph[kG] = {phys->means, phys->scales, phys->quats, phys->betas, phys->opacities, phys->shs};
  const float* gp[kG] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (adam) {
    if (!grads || !hp) return fail(GES_ERR_INVALID_ARG, "NULL argument");
    if (step < 1) return fail(GES_ERR_INVALID_ARG, "step must be >= 1");
    if (!(hp->beta1 >= 0.f && hp->beta1 < 1.f && hp->beta2 >= 0.f && hp->beta2 < 1.f) || !(hp->eps >= 0.f))
      return fail(GES_ERR_INVALID_ARG, "need beta1, beta2 in [0,1) and eps >= 0");
    const float* gg[kG] = {grads->means, grads->scales, grads->quats, grads->betas, grads->opacities, grads->shs};
    std::memcpy(gp, gg, sizeof(gg));
  }
  if (set->n == 0) return GES_OK;
  AdamArgs A;
  std::memset(&A, 0, sizeof(A));
  int64_t q = 0;
  for (int g = 0; g < kG; ++g) {
    if (!ph[g] || !aligned16(ph[g])) return fail(GES_ERR_INVALID_ARG, "phys group %d pointer is NULL or misaligned", g);
    if (adam && (!gp[g] || !aligned16(gp[g])))
      return fail(GES_ERR_INVALID_ARG, "gradient group %d pointer is NULL or misaligned", g);
    A.p[g] = set->param[g];
    A.m[g] = set->m[g];
    A.v[g] = set->v[g];
    A.g[g] = gp[g];
    A.phys[g] = ph[g];
    A.count[g] = set->n * group_width(g, set->sh_degree);
    A.quad0[g] = q;
    q += (A.count[g] + 3) / 4;
  }
  A.quad0[kG] = q;
  A.sh_row = (int32_t)group_width(5, set->sh_degree);
  A.adam = adam ? 1 : 0;
  if (adam) {
    for (int g = 0; g < kG; ++g) A.lr[g] = hp->lr[g];
    A.lr_rest = hp->lr_sh_rest;
    A.b1 = hp->beta1;
    A.b2 = hp->beta2;
    A.ic1 = (float)(1.0 / (1.0 - std::pow((double)hp->beta1, (double)step)));
    A.isc2 = (float)(1.0 / std::sqrt(1.0 - std::pow((double)hp->beta2, (double)step)));
    A.eps = hp->eps;
  }
  if ((st = use_device(ctx->device)) != GES_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  {
    TraceScope tr(ctx, adam ? "k_adam" : "k_activate", s);
    k_adam<<<grid_for(ctx, k_adam, q), kThreads, 0, s>>>(A);
  }
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GES_OK : cuda_fail(e, adam ? "adam launch" : "activate launch");
}

ges_status run_reset(ges_ctx* ctx, const ges_train_set* set, int grp, int clamp, float val, void* stream) {
  if (!ctx) return fail(GES_ERR_INVALID_ARG, "ctx is NULL");
  ges_status st;
  if ((st = check_set(set, "set")) != GES_OK) return st;
  if (set->n == 0) return GES_OK;
  if ((st = use_device(ctx->device)) != GES_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  {
    TraceScope tr(ctx, "k_reset", s);
    k_reset<<<grid_for(ctx, k_reset, set->n), kThreads, 0, s>>>(set->param[grp], set->m[grp], set->v[grp], set->n, clamp, val);
  }
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GES_OK : cuda_fail(e, "reset launch");
}

}  // namespace
}  // namespace ges

using namespace ges;

extern "C" {

ges_status ges_adam_params_default(ges_adam_params* out) {
  if (!out) return fail(GES_ERR_INVALID_ARG, "out is NULL");
  const float lr[kG] = {1.6e-4f, 0.005f, 0.001f, 0.001f, 0.05f, 0.0025f};
  for (int g = 0; g < kG; ++g) out->lr[g] = lr[g];
  out->lr_sh_rest = (float)(0.0025 / 20.0);
  out->beta1 = 0.9f;
  out->beta2 = 0.999f;
  out->eps = 1e-15f;
  return GES_OK;
}

ges_status ges_density_params_default(ges_density_params* out) {
  if (!out) return fail(GES_ERR_INVALID_ARG, "out is NULL");
  out->grad_threshold = 0.0003f;
  out->percent_dense = 0.01f;
  out->scene_extent = 1.0f;
  out->min_opacity = 0.005f;
  out->min_beta = 0.0f;
  out->max_world_size = 0.0f;
  return GES_OK;
}

ges_status ges_position_lr(int64_t step, float lr_init, float lr_final, float delay_mult, int64_t delay_steps,
                           int64_t max_steps, float* out) {
  if (!out) return fail(GES_ERR_INVALID_ARG, "out is NULL");
  if (max_steps < 1 || !(lr_init > 0.f) || !(lr_final > 0.f))
    return fail(GES_ERR_INVALID_ARG, "need max_steps >= 1 and positive rates");
  if (step < 0) {
    *out = 0.f;
    return GES_OK;
  }
  double delay = 1.0;
  if (delay_steps > 0) {
    double r = (double)step / (double)delay_steps;
    r = r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
    delay = delay_mult + (1.0 - delay_mult) * std::sin(1.5707963267948966 * r);  // pi/2
  }
  double t = (double)step / (double)max_steps;
  t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  *out = (float)(delay * std::exp(std::log((double)lr_init) * (1.0 - t) + std::log((double)lr_final) * t));
  return GES_OK;
}

ges_status ges_adam_step(ges_ctx* ctx, const ges_train_set* set, const ges_grads* grads, const ges_scene_out* phys,
                         const ges_adam_params* hp, int64_t step, void* stream) {
  return run_adam(ctx, set, grads, phys, hp, step, stream, true);
}

ges_status ges_activate(ges_ctx* ctx, const ges_train_set* set, const ges_scene_out* phys, void* stream) {
  return run_adam(ctx, set, nullptr, phys, nullptr, 0, stream, false);
}

ges_status ges_densify_stats(ges_frame* f, float* grad_accum, int32_t* count, void* stream) {
  if (!f || !grad_accum || !count) return fail(GES_ERR_INVALID_ARG, "NULL argument");
  if (!f->have_bwd) return fail(GES_ERR_INVALID_ARG, "ges_densify_stats before ges_render_bwd");
  ges_status st = use_device(f->ctx->device);
  if (st != GES_OK) return st;
  if (f->n == 0) return GES_OK;
  cudaStream_t s = (cudaStream_t)stream;
  {
    TraceScope tr(f->ctx, "k_densify_stats", s);
    k_densify_stats<<<grid_for(f->ctx, k_densify_stats, f->n), kThreads, 0, s>>>(f->depth_key, f->g2d, f->n, 0.5f * (float)f->W,
                                                                0.5f * (float)f->H, grad_accum, count);
  }
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GES_OK : cuda_fail(e, "densify stats launch");
}

ges_status ges_density_control(ges_ctx* ctx, const ges_train_set* in, const float* grad_accum, const int32_t* count,
                               const float* xi, const ges_density_params* dp, const ges_train_set* out,
                               int64_t* n_out, void* stream) {
  if (!ctx || !dp || !n_out) return fail(GES_ERR_INVALID_ARG, "NULL argument");
  ges_status st;
  if ((st = check_set(in, "in")) != GES_OK) return st;
  if ((st = check_set(out, "out")) != GES_OK) return st;
  if (out->sh_degree != in->sh_degree) return fail(GES_ERR_INVALID_ARG, "out->sh_degree differs from in");
  if (in->n > 0 && (!grad_accum || !count || !xi)) return fail(GES_ERR_INVALID_ARG, "NULL statistics or xi");
  if (!(dp->grad_threshold >= 0.f) || !(dp->percent_dense > 0.f) || !(dp->scene_extent > 0.f) ||
      !(dp->min_opacity >= 0.f && dp->min_opacity < 1.f) || !(dp->min_beta >= 0.f) || !(dp->max_world_size >= 0.f))
    return fail(GES_ERR_INVALID_ARG, "density parameters out of range");
  if (in->n > 0 && out->n > 0)
    for (int g = 0; g < kG; ++g)
      if (in->param[g] == out->param[g] || in->m[g] == out->m[g] || in->v[g] == out->v[g])
        return fail(GES_ERR_INVALID_ARG, "in and out share group %d", g);
  const int64_t n = in->n;
  if (n == 0) {
    *n_out = 0;
    return GES_OK;
  }
  if ((st = use_device(ctx->device)) != GES_OK) return st;

  DensArgs D;
  std::memset(&D, 0, sizeof(D));
  D.n = n;
  for (int g = 0; g < kG; ++g) {
    D.width[g] = (int32_t)group_width(g, in->sh_degree);
    D.in[g] = in->param[g];
    D.in_m[g] = in->m[g];
    D.in_v[g] = in->v[g];
    D.out[g] = out->param[g];
    D.out_m[g] = out->m[g];
    D.out_v[g] = out->v[g];
  }
  D.acc = grad_accum;
  D.cnt = count;
  D.xi = xi;
  // thresholds mapped into the variables, in double, rounded once
  const double pd = dp->percent_dense, ext = dp->scene_extent;
  D.t_grad = dp->grad_threshold;
  D.t_small = (float)std::log(pd * ext);
  D.t_opac = dp->min_opacity > 0.f ? (float)std::log((double)dp->min_opacity / (1.0 - (double)dp->min_opacity))
                                   : -INFINITY;
  D.t_beta = dp->min_beta > 0.f ? (float)((double)dp->min_beta - 2.0) : -INFINITY;
  D.t_big = dp->max_world_size > 0.f ? (float)std::log((double)dp->max_world_size * ext) : INFINITY;
  D.t_split = (float)std::log(1.6);

  // scratch: totals | kind [n] | 3 position arrays [n] | scan scratch
  const size_t kind_bytes = ((size_t)n + 255) & ~(size_t)255;
  const size_t pos_bytes = (((size_t)n * 4) + 255) & ~(size_t)255;
  const size_t scan_bytes = ScanScratch::required(n);
  void* buf = nullptr;
  if ((st = ctx_scratch(ctx, 2, 256 + kind_bytes + 3 * pos_bytes + scan_bytes, &buf)) != GES_OK) return st;
  char* b = static_cast<char*>(buf);
  uint32_t* tot = reinterpret_cast<uint32_t*>(b);
  D.kind = reinterpret_cast<uint8_t*>(b + 256);
  for (int k = 0; k < 3; ++k) D.pos[k] = reinterpret_cast<uint32_t*>(b + 256 + kind_bytes + k * pos_bytes);
  ScanScratch sc;
  sc.buf = b + 256 + kind_bytes + 3 * pos_bytes;
  sc.bytes = scan_bytes;

  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  {
    TraceScope tr(ctx, "k_density_classify", s);
    k_density_classify<<<grid_for(ctx, k_density_classify, n), kThreads, 0, s>>>(D);
    count_launches(1);
    for (int k = 0; k < 3; ++k) scan_exclusive<uint32_t, uint32_t>(D.pos[k], D.pos[k], n, tot + k, sc, s);
  }
  uint32_t h[3] = {0, 0, 0};
  if ((e = cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "reading density counts");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "density control");
  const int64_t need = (int64_t)h[0] + h[1] + 2 * (int64_t)h[2];
  *n_out = need;
  if (need > out->n)
    return fail(GES_ERR_CAPACITY, "density control needs %lld rows, out holds %lld", (long long)need, (long long)out->n);
  D.base[0] = 0;
  D.base[1] = h[0];
  D.base[2] = (int64_t)h[0] + h[1];
  D.base[3] = D.base[2] + h[2];
  {
    TraceScope tr(ctx, "k_density_copy", s);
    for (int g = 0; g < kG; ++g) k_density_copy<<<grid_for(ctx, k_density_copy, n * D.width[g]), kThreads, 0, s>>>(D, g);
    count_launches(kG);
  }
  if (h[2] > 0) {
    TraceScope tr(ctx, "k_density_children", s);
    k_density_children<<<grid_for(ctx, k_density_children, n), kThreads, 0, s>>>(D);
    count_launches(1);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "density control launch");
  return GES_OK;
}

ges_status ges_reset_opacity(ges_ctx* ctx, const ges_train_set* set, float max_opacity, void* stream) {
  if (!(max_opacity > 0.f && max_opacity < 1.f)) return fail(GES_ERR_INVALID_ARG, "max_opacity must lie in (0,1)");
  const float lim = (float)std::log((double)max_opacity / (1.0 - (double)max_opacity));
  return run_reset(ctx, set, 4, 1, lim, stream);
}

ges_status ges_reset_shape(ges_ctx* ctx, const ges_train_set* set, float beta, void* stream) {
  if (!(beta > 0.f)) return fail(GES_ERR_INVALID_ARG, "beta must be > 0");
  return run_reset(ctx, set, 3, 0, (float)((double)beta - 2.0), stream);
}

}  // extern "C"
