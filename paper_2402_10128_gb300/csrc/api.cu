// C ABI of libges: contexts, per-frame workspaces, and the frame pipeline
//   ges_preprocess -> ges_bin_sort -> ges_render_fwd [-> ges_render_bwd].
// Every entry point validates its arguments on the host, enqueues on the caller's stream and
// returns a ges_status; no exception crosses the ABI.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "api_internal.h"

#include <nvtx3/nvToolsExt.h>

namespace ges {

static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

void count_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

ges_status fail(ges_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

ges_status cuda_fail(cudaError_t e, const char* what) {
  return fail(GES_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

ges_status ctx_alloc(ges_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return GES_OK;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->budget && ctx->used + bytes > ctx->budget)
      return fail(GES_ERR_OOM, "HBM budget exceeded: %zu used + %zu requested > %zu", ctx->used, bytes, ctx->budget);
    ctx->used += bytes;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->used -= bytes;
    *p = nullptr;
    return fail(GES_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  return GES_OK;
}

void ctx_free(ges_ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->used -= bytes;
}

ges_status use_device(int device) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != device) {
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  }
  return GES_OK;
}

Params to_params(const ges_params& p) {
  Params P;
  P.rho = p.rho;
  P.dilation = p.dilation;
  P.alpha_max = p.alpha_max;
  P.alpha_min = p.alpha_min;
  P.t_min = p.t_min;
  P.margin_rel = p.extent_margin_rel;
  P.margin_abs = p.extent_margin_abs;
  P.clamp_fov = p.clamp_fov;
  P.mode = p.falloff;
  int l = 0;
  while ((1 << l) < p.segment_tiles) ++l;
  P.seg_log2 = l;
  P.seg_bits = 0;  // set once the segment count is known
  P.phi_mode = p.phi_mode;
  P.id_bits = 0;  // set once the primitive and segment counts are known
  return P;
}

ges_status check_params(const ges_params* p) {
  if (!p) return fail(GES_ERR_INVALID_ARG, "params is NULL");
  if (p->falloff != GES_FALLOFF_GEF && p->falloff != GES_FALLOFF_PAPER_APPROX)
    return fail(GES_ERR_INVALID_ARG, "unknown falloff %d", p->falloff);
  if (!(p->alpha_min > 0.f && p->alpha_min < p->alpha_max && p->alpha_max < 1.f))
    return fail(GES_ERR_INVALID_ARG, "need 0 < alpha_min < alpha_max < 1");
  if (!(p->t_min > 0.f && p->t_min < 1.f)) return fail(GES_ERR_INVALID_ARG, "need 0 < t_min < 1");
  if (!(p->dilation >= 0.f) || !(p->rho >= 0.f) || !(p->extent_margin_rel >= 0.f) || !(p->extent_margin_abs >= 0.f) ||
      !(p->clamp_fov > 0.f))
    return fail(GES_ERR_INVALID_ARG, "dilation, rho and margins must be >= 0, clamp_fov > 0");
  if (p->segment_tiles < 1 || p->segment_tiles > 1024 || (p->segment_tiles & (p->segment_tiles - 1)))
    return fail(GES_ERR_INVALID_ARG, "segment_tiles %d is not a power of two in [1, 1024]", p->segment_tiles);
  if (p->phi_mode != GES_PHI_APPROX && p->phi_mode != GES_PHI_EXACT && p->phi_mode != GES_PHI_EXACT_VARIANCE)
    return fail(GES_ERR_INVALID_ARG, "unknown phi_mode %d", p->phi_mode);
  return GES_OK;
}

ges_status check_camera(const ges_camera* c) {
  if (!c) return fail(GES_ERR_INVALID_ARG, "camera is NULL");
  if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384)
    return fail(GES_ERR_INVALID_ARG, "image size %dx%d out of range", c->width, c->height);
  if (!(c->fx > 0.f) || !(c->fy > 0.f)) return fail(GES_ERR_INVALID_ARG, "focal lengths must be > 0");
  if (!(c->znear > 0.f)) return fail(GES_ERR_INVALID_ARG, "znear must be > 0");
  return GES_OK;
}

ges_status check_scene(const ges_scene* s) {
  if (!s) return fail(GES_ERR_INVALID_ARG, "scene is NULL");
  if (s->n < 0 || s->n > 0x7fffffffLL) return fail(GES_ERR_INVALID_ARG, "scene n=%lld out of range", (long long)s->n);
  if (s->sh_degree < 0 || s->sh_degree > 3) return fail(GES_ERR_INVALID_ARG, "sh_degree %d not in 0..3", s->sh_degree);
  if (s->n > 0 && (!s->means || !s->scales || !s->quats || !s->betas || !s->opacities || !s->shs))
    return fail(GES_ERR_INVALID_ARG, "scene array pointer is NULL");
  if (((uintptr_t)s->quats) & 15u) return fail(GES_ERR_INVALID_ARG, "quats must be 16-byte aligned");
  if ((s->sh_degree == 1 || s->sh_degree == 3) && (((uintptr_t)s->shs) & 15u))
    return fail(GES_ERR_INVALID_ARG, "shs must be 16-byte aligned for SH degree 1 and 3");
  return GES_OK;
}

void fill_view(ViewDesc& v, const ges_camera& c, const ges_scene& s, int64_t prim_base, int32_t tile_base,
               int32_t seg_base, int seg_log2) {
  std::memset(&v, 0, sizeof(v));
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 4; ++k) v.V[4 * r + k] = c.viewmat[4 * r + k];
  v.fx = c.fx; v.fy = c.fy; v.cx = c.cx; v.cy = c.cy;
  for (int k = 0; k < 3; ++k) { v.campos[k] = c.campos[k]; v.bg[k] = c.bg[k]; }
  v.znear = c.znear;
  v.W = c.width; v.H = c.height;
  v.tiles_x = (c.width + kTile - 1) / kTile;
  v.tiles_y = (c.height + kTile - 1) / kTile;
  v.tile_base = tile_base;
  v.seg_base = seg_base;
  v.segs_x = (v.tiles_x + (1 << seg_log2) - 1) >> seg_log2;
  v.sh_degree = s.sh_degree;
  v.prim_base = prim_base;
  v.n = s.n;
  v.means = s.means; v.scales = s.scales; v.quats = s.quats; v.betas = s.betas; v.opac = s.opacities; v.shs = s.shs;
}

int bits_for(int64_t count) {
  int b = 0;
  while (((int64_t)1 << b) < count) ++b;
  return b;
}

ges_status set_segment_bits(Params& P, int64_t total_segs) {
  P.seg_bits = bits_for(total_segs > 1 ? total_segs : 2);
  if (P.seg_bits + 2 * P.seg_log2 > 32)
    return fail(GES_ERR_INVALID_ARG, "%lld segments of %d tiles do not fit a 32-bit list key; use fewer tiles per segment",
                (long long)total_segs, 1 << P.seg_log2);
  return GES_OK;
}

// The depth sort's 32-bit value carries a primitive's list entries above its id when both fit: ids
// below n and entries at most the view's segment count (one entry per segment at most).
void set_pack_bits(Params& P, int64_t n, int64_t segs_per_view) {
  const int ib = bits_for(n > 1 ? n : 2);
  P.id_bits = ib + bits_for(segs_per_view + 1) <= 32 ? ib : 0;
}

// ---------------------------------------------------------------- frame buffers
static void frame_free_keys(ges_frame* f) {
  for (int i = 0; i < 2; ++i) {
    ctx_free(f->ctx, f->tk[i], sizeof(uint32_t) * f->key_cap);
    ctx_free(f->ctx, f->tv[i], sizeof(uint32_t) * f->key_cap);
    f->tk[i] = f->tv[i] = nullptr;
  }
  ctx_free(f->ctx, f->hist, sizeof(uint32_t) * f->hist_cap);
  ctx_free(f->ctx, f->scan.buf, f->scan.bytes);
  f->hist = nullptr;
  f->scan.buf = nullptr;
}

static ges_status frame_alloc_keys(ges_frame* f, int64_t key_cap) {
  f->key_cap = key_cap;
  ges_status st;
  for (int i = 0; i < 2; ++i) {
    if ((st = ctx_alloc(f->ctx, (void**)&f->tk[i], sizeof(uint32_t) * key_cap)) != GES_OK) return st;
    if ((st = ctx_alloc(f->ctx, (void**)&f->tv[i], sizeof(uint32_t) * key_cap)) != GES_OK) return st;
  }
  int64_t h1 = radix_hist_entries(f->n_cap, 32), h2 = radix_hist_entries(key_cap, bits_for(f->n_tiles));
  f->hist_cap = h1 > h2 ? h1 : h2;
  if ((st = ctx_alloc(f->ctx, (void**)&f->hist, sizeof(uint32_t) * f->hist_cap)) != GES_OK) return st;
  int64_t scan_n = f->hist_cap > f->n_cap ? f->hist_cap : f->n_cap;
  f->scan.bytes = ScanScratch::required(scan_n);
  if ((st = ctx_alloc(f->ctx, &f->scan.buf, f->scan.bytes)) != GES_OK) return st;
  return GES_OK;
}

// ---------------------------------------------------------------- tracing

cudaEvent_t trace_event(ges_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}


TraceScope::TraceScope(ges_ctx* c_, const char* name_, cudaStream_t s_) : c(c_), name(name_), s(s_) {
  nvtxRangePushA(name);
  if (!c->trace_on) return;
  std::lock_guard<std::mutex> lk(c->mu);
  a = trace_event(c);
  if (a && cudaEventRecord(a, s) != cudaSuccess) {
    c->event_pool.push_back(a);
    a = nullptr;
  }
}

TraceScope::~TraceScope() {
  nvtxRangePop();
  if (!a) return;
  std::lock_guard<std::mutex> lk(c->mu);
  cudaEvent_t b = trace_event(c);
  if (b && cudaEventRecord(b, s) == cudaSuccess) {
    c->trace.push_back({name, a, b});
  } else {
    c->event_pool.push_back(a);
    if (b) c->event_pool.push_back(b);
  }
}

// grow-only scratch of the context, one buffer per slot (0 mask, 1 loss, 2 density control)
ges_status ctx_scratch(ges_ctx* ctx, int slot, size_t bytes, void** out) {
  std::lock_guard<std::mutex> lk(ctx->scratch_mu);
  if (ctx->scratch_bytes[slot] < bytes) {
    if (ctx->scratch[slot]) {
      cudaDeviceSynchronize();  // kernels of an earlier call may still use it
      ctx_free(ctx, ctx->scratch[slot], ctx->scratch_bytes[slot]);
    }
    ctx->scratch[slot] = nullptr;
    ctx->scratch_bytes[slot] = 0;
    ges_status st = ctx_alloc(ctx, &ctx->scratch[slot], bytes);
    if (st != GES_OK) return st;
    ctx->scratch_bytes[slot] = bytes;
  }
  *out = ctx->scratch[slot];
  return GES_OK;
}

}  // namespace ges

using namespace ges;

// The per-tile lists of the last binning, expanded on the host from the segment lists: tiles in
// id order; for each, the entries of its segment whose span covers it, in list order.  Calls
// emit(tile, list entry index) for each (tile, entry) and returns the per-tile [start, end) in
// the expanded order through tile_ranges (optional, 2 per tile).
template <class Emit>
static ges_status walk_tile_lists(ges_frame* f, cudaStream_t s, std::vector<uint32_t>& tk, Emit emit,
                                  uint32_t* tile_ranges) {
  int64_t K = 0;
  ges_status st = ges_frame_status(f, s, &K);
  if (st != GES_OK) return st;
  tk.resize((size_t)K);
  std::vector<uint2> rg((size_t)f->n_segs);
  cudaError_t e;
  if (K && (e = cudaMemcpy(tk.data(), f->tile_keys, 4 * (size_t)K, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "copy list keys");
  if ((e = cudaMemcpy(rg.data(), f->ranges, sizeof(uint2) * f->n_segs, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "copy ranges");
  const int L = f->P.seg_log2, sb = f->P.seg_bits;
  const uint32_t m = (1u << L) - 1u;
  const int32_t sx = f->vt.t.v[0].segs_x;
  uint64_t pos = 0;
  for (int32_t ty = 0; ty < f->tiles_y; ++ty)
    for (int32_t tx = 0; tx < f->tiles_x; ++tx) {
      const int64_t tile = (int64_t)ty * f->tiles_x + tx;
      const uint2 r = rg[(size_t)ty * sx + (tx >> L)];
      const uint32_t to = (uint32_t)tx & m;
      const uint64_t start = pos;
      for (uint32_t i = r.x; i < r.y; ++i) {
        const uint32_t key = tk[i];
        if (((key >> sb) & m) <= to && to <= ((key >> (sb + L)) & m)) {
          emit(tile, i);
          ++pos;
        }
      }
      if (tile_ranges) {
        tile_ranges[2 * tile] = pos > start ? (uint32_t)start : 0u;
        tile_ranges[2 * tile + 1] = pos > start ? (uint32_t)pos : 0u;
      }
    }
  return GES_OK;
}

extern "C" {

const char* ges_last_error(void) { return g_last_error.c_str(); }

ges_status ges_params_default(ges_params* out) {
  if (!out) return fail(GES_ERR_INVALID_ARG, "out is NULL");
  out->rho = 0.1f;
  out->falloff = GES_FALLOFF_GEF;
  out->dilation = 0.3f;
  out->alpha_max = 0.99f;
  out->alpha_min = 1.0f / 255.0f;
  out->t_min = 1e-4f;
  out->extent_margin_rel = 1e-3f;
  out->extent_margin_abs = 1e-2f;
  out->clamp_fov = 1.3f;
  out->segment_tiles = 16;
  out->phi_mode = GES_PHI_APPROX;
  return GES_OK;
}

ges_status ges_ctx_create(int device, size_t hbm_budget_bytes, ges_ctx** out) {
  if (!out) return fail(GES_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(GES_ERR_INVALID_ARG, "device %d not in [0,%d)", device, ndev);
  ges_status st = use_device(device);
  if (st != GES_OK) return st;
  ges_ctx* c = new (std::nothrow) ges_ctx();
  if (!c) return fail(GES_ERR_OOM, "host allocation failed");
  c->device = device;
  c->budget = hbm_budget_bytes;
  c->used = 0;
  e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaDeviceGetAttribute"); }
  set_key_constants(0);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { delete c; return cuda_fail(e, "uploading key constants"); }
  *out = c;
  return GES_OK;
}

void ges_ctx_destroy(ges_ctx* ctx) {
  if (!ctx) return;
  bool any = false;
  for (int i = 0; i < kScratchSlots; ++i) any = any || ctx->scratch[i];
  if (any) cudaDeviceSynchronize();
  for (int i = 0; i < kScratchSlots; ++i) ctx_free(ctx, ctx->scratch[i], ctx->scratch_bytes[i]);
  for (auto& r : ctx->trace) {
    ctx->event_pool.push_back(r.a);
    ctx->event_pool.push_back(r.b);
  }
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  delete ctx;
}

ges_status ges_trace_enable(ges_ctx* ctx, int on) {
  if (!ctx) return fail(GES_ERR_INVALID_ARG, "ctx is NULL");
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (on) {
    for (auto& r : ctx->trace) {
      ctx->event_pool.push_back(r.a);
      ctx->event_pool.push_back(r.b);
    }
    ctx->trace.clear();
  }
  ctx->trace_on = on != 0;
  return GES_OK;
}

ges_status ges_trace_read(ges_ctx* ctx, int32_t capacity, char* names, int64_t* launches, double* total_ms,
                          int32_t* n_out) {
  if (!ctx || !n_out) return fail(GES_ERR_INVALID_ARG, "ctx/n_out is NULL");
  if (capacity < 0) return fail(GES_ERR_INVALID_ARG, "capacity < 0");
  if (capacity > 0 && (!names || !launches || !total_ms)) return fail(GES_ERR_INVALID_ARG, "output is NULL");
  ges_status st = use_device(ctx->device);
  if (st != GES_OK) return st;
  std::lock_guard<std::mutex> lk(ctx->mu);
  std::vector<const char*> order;
  std::vector<int64_t> cnt;
  std::vector<double> ms;
  ges_status result = GES_OK;
  for (auto& r : ctx->trace) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess && result == GES_OK) result = cuda_fail(e, "trace event");
    size_t k = 0;
    while (k < order.size() && std::strcmp(order[k], r.name) != 0) ++k;
    if (k == order.size()) {
      order.push_back(r.name);
      cnt.push_back(0);
      ms.push_back(0.0);
    }
    cnt[k] += 1;
    ms[k] += (double)t;
    ctx->event_pool.push_back(r.a);
    ctx->event_pool.push_back(r.b);
  }
  ctx->trace.clear();
  *n_out = (int32_t)order.size();
  for (size_t k = 0; k < order.size() && (int64_t)k < capacity; ++k) {
    std::strncpy(names + 32 * k, order[k], 31);
    names[32 * k + 31] = '\0';
    launches[k] = cnt[k];
    total_ms[k] = ms[k];
  }
  return result;
}

ges_status ges_frame_create(ges_ctx* ctx, int64_t n_capacity, int32_t width, int32_t height, int64_t key_capacity,
                            ges_frame** out) {
  if (!ctx || !out) return fail(GES_ERR_INVALID_ARG, "ctx/out is NULL");
  *out = nullptr;
  if (n_capacity < 0 || n_capacity > 0x7fffffffLL) return fail(GES_ERR_INVALID_ARG, "n_capacity out of range");
  if (width < 1 || height < 1 || width > 16384 || height > 16384) return fail(GES_ERR_INVALID_ARG, "image size out of range");
  if (key_capacity < 0 || key_capacity > 0x7fffffffLL) return fail(GES_ERR_INVALID_ARG, "key_capacity out of range");
  ges_status st = use_device(ctx->device);
  if (st != GES_OK) return st;
  ges_frame* f = new (std::nothrow) ges_frame();
  if (!f) return fail(GES_ERR_OOM, "host allocation failed");
  f->ctx = ctx;
  f->n_cap = n_capacity > 0 ? n_capacity : 1;
  f->W = width;
  f->H = height;
  f->tiles_x = (width + kTile - 1) / kTile;
  f->tiles_y = (height + kTile - 1) / kTile;
  f->n_tiles = (int64_t)f->tiles_x * f->tiles_y;
  f->auto_cap = key_capacity == 0;
  const int64_t N = f->n_cap;
  auto A = [&](void** p, size_t b) { return st == GES_OK ? (st = ctx_alloc(ctx, p, b)) : st; };
  A((void**)&f->depth_key, 4 * N);
  for (int i = 0; i < 2; ++i) {
    A((void**)&f->dk[i], 4 * N);
    A((void**)&f->pv[i], 4 * N);
  }
  A((void**)&f->rect, sizeof(ushort4) * N);
  A((void**)&f->rec, sizeof(Rec) * N);
  A((void**)&f->ks, sizeof(KeyShape) * N);
  A((void**)&f->tprim, 4 * N);
  A((void**)&f->touched, 4 * N);
  A((void**)&f->offsets, 8 * N);
  A((void**)&f->g2d, sizeof(float4) * 3 * N);
  A((void**)&f->ranges, sizeof(uint2) * f->n_tiles);
  A((void**)&f->tile_bucket, 4 * f->n_tiles);
  A((void**)&f->tile_order, 4 * f->n_tiles);
  A((void**)&f->order_count, 4 * 2 * kOrderBuckets);
  A((void**)&f->d_K, 8);
  A((void**)&f->d_flags, 4);
  if (st == GES_OK) {
    int64_t cap = key_capacity > 0 ? key_capacity : (N * 8 > 1024 ? N * 8 : 1024);
    st = frame_alloc_keys(f, cap);
  }
  if (st == GES_OK) {
    cudaError_t e = cudaMallocHost((void**)&f->h_K, 8);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMallocHost");
  }
  if (st != GES_OK) {
    std::string msg = g_last_error;
    ges_frame_destroy(f);
    g_last_error = msg;
    return st;
  }
  *out = f;
  return GES_OK;
}

void ges_frame_destroy(ges_frame* f) {
  if (!f) return;
  use_device(f->ctx->device);
  cudaDeviceSynchronize();
  const int64_t N = f->n_cap;
  ges_ctx* c = f->ctx;
  ctx_free(c, f->depth_key, 4 * N);
  for (int i = 0; i < 2; ++i) {
    ctx_free(c, f->dk[i], 4 * N);
    ctx_free(c, f->pv[i], 4 * N);
  }
  ctx_free(c, f->rect, sizeof(ushort4) * N);
  ctx_free(c, f->rec, sizeof(Rec) * N);
  ctx_free(c, f->ks, sizeof(KeyShape) * N);
  ctx_free(c, f->tprim, 4 * N);
  ctx_free(c, f->touched, 4 * N);
  ctx_free(c, f->offsets, 8 * N);
  ctx_free(c, f->g2d, sizeof(float4) * 3 * N);
  ctx_free(c, f->ranges, sizeof(uint2) * f->n_tiles);
  ctx_free(c, f->tile_bucket, 4 * f->n_tiles);
  ctx_free(c, f->tile_order, 4 * f->n_tiles);
  ctx_free(c, f->order_count, 4 * 2 * kOrderBuckets);
  ctx_free(c, f->d_K, 8);
  ctx_free(c, f->d_flags, 4);
  frame_free_keys(f);
  ctx_free(c, f->work_img, sizeof(float) * 5 * (size_t)f->W * f->H);
  ctx_free(c, f->work_stats, 32);
  if (f->h_K) cudaFreeHost(f->h_K);
  delete f;
}

ges_status ges_preprocess(ges_frame* f, const ges_scene* scene, const ges_camera* cam, const ges_params* params,
                          void* stream) {
  if (!f) return fail(GES_ERR_INVALID_ARG, "frame is NULL");
  ges_status st;
  if ((st = check_scene(scene)) != GES_OK || (st = check_camera(cam)) != GES_OK || (st = check_params(params)) != GES_OK)
    return st;
  if (scene->n > f->n_cap && !(scene->n == 0)) return fail(GES_ERR_INVALID_ARG, "scene n=%lld > frame capacity %lld",
                                                           (long long)scene->n, (long long)f->n_cap);
  if (cam->width != f->W || cam->height != f->H)
    return fail(GES_ERR_INVALID_ARG, "camera %dx%d != frame %dx%d", cam->width, cam->height, f->W, f->H);
  if ((st = use_device(f->ctx->device)) != GES_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  f->P = to_params(*params);
  f->vt.t.n = 1;
  fill_view(f->vt.t.v[0], *cam, *scene, 0, 0, 0, f->P.seg_log2);
  f->vt.t.total_prims = (unsigned long long)scene->n;
  f->vt.t.total_tiles = f->n_tiles;
  f->n_segs = (int64_t)f->vt.t.v[0].segs_x * f->tiles_y;
  f->vt.t.total_segs = f->n_segs;
  if ((st = set_segment_bits(f->P, f->n_segs)) != GES_OK) return st;
  set_pack_bits(f->P, scene->n, f->n_segs);
  f->n = scene->n;
  f->sh_degree = scene->sh_degree;
  {
    TraceScope tr(f->ctx, "k_preprocess", s);
    launch_preprocess<FrameViews>(f->vt, f->n, f->P, f->depth_key, f->dk[0], f->pv[0], f->rect, f->rec, f->ks,
                                  f->tprim, f->ctx->num_sms, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "preprocess launch");
  f->have_pre = true;
  f->have_sort = false;
  f->have_bwd = false;
  return GES_OK;
}

ges_status ges_bin_sort(ges_frame* f, void* stream) {
  if (!f) return fail(GES_ERR_INVALID_ARG, "frame is NULL");
  if (!f->have_pre) return fail(GES_ERR_INVALID_ARG, "ges_bin_sort before ges_preprocess");
  ges_status st = use_device(f->ctx->device);
  if (st != GES_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(f->d_flags, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "memset flags");
  // depth sort of the primitives (32-bit keys)
  int cur = 0;
  {
    TraceScope tr(f->ctx, "depth_sort", s);
    if (!radix_sort_pairs(f->dk, f->pv, cur, f->n, nullptr, f->n, 32, f->hist, f->hist_cap, f->scan, s, f->d_flags))
      return fail(GES_ERR_CUDA, "internal: depth-sort histogram exceeds its buffer");
  }
  f->sorted_prims = f->pv[cur];
  // list entries per primitive in depth order and their exclusive scan -> offsets, K
  {
    TraceScope tr(f->ctx, "scan_touched", s);
    if (f->P.id_bits)
      scan_unpack_onepass(f->sorted_prims, f->P.id_bits, f->offsets, f->n, f->d_K, f->scan, f->d_flags, s);
    else
      scan_gather_onepass(f->tprim, f->sorted_prims, f->touched, f->offsets, f->n, f->d_K, f->scan, f->d_flags, s);
  }
  if (f->auto_cap) {
    if ((e = cudaMemcpyAsync(f->h_K, f->d_K, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(e, "read K");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "sync for K");
    const int64_t K = (int64_t)*f->h_K;
    if (K > f->key_cap) {
      if (K > 0x7fffffffLL) return fail(GES_ERR_CAPACITY, "K=%lld duplicates exceed 2^31", (long long)K);
      frame_free_keys(f);
      int64_t cap = K + K / 4 + 1024;
      if (cap > 0x7fffffffLL) cap = 0x7fffffffLL;
      if ((st = frame_alloc_keys(f, cap)) != GES_OK) return st;
    }
  }
  {
    TraceScope tr(f->ctx, "k_keygen", s);
    launch_keygen<FrameViews>(f->vt, f->offsets, f->touched, f->d_K, f->n, f->sorted_prims, f->ks,
                              f->P, f->key_cap, f->tk[0], f->tv[0], f->d_flags, s);
  }
  int tcur = 0;
  bool ranges_done = false;
  {
    TraceScope tr(f->ctx, "list_sort", s);
    // a single-pass list sort also gives every segment's range, from its histogram
    if (!radix_sort_pairs(f->tk, f->tv, tcur, 0, f->d_K, f->key_cap, f->P.seg_bits, f->hist, f->hist_cap, f->scan, s,
                          f->d_flags, f->ranges, f->n_segs, &ranges_done))
      return fail(GES_ERR_CUDA, "internal: list-sort histogram exceeds its buffer");
  }
  f->tile_keys = f->tk[tcur];
  f->tile_vals = f->tv[tcur];
  if (!ranges_done) {
    if ((e = cudaMemsetAsync(f->ranges, 0, sizeof(uint2) * f->n_segs, s)) != cudaSuccess) return cuda_fail(e, "memset ranges");
    TraceScope tr(f->ctx, "k_ranges", s);
    launch_ranges(f->tile_keys, f->d_K, f->key_cap, (uint32_t)((1ull << f->P.seg_bits) - 1), f->ranges, f->ctx->num_sms,
                  s);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "bin_sort launch");
  f->have_sort = true;
  return GES_OK;
}

ges_status ges_render_fwd(ges_frame* f, float* img, float* final_T, uint32_t* n_contrib, void* stream) {
  if (!f || !img || !final_T || !n_contrib) return fail(GES_ERR_INVALID_ARG, "NULL argument");
  if (!f->have_sort) return fail(GES_ERR_INVALID_ARG, "ges_render_fwd before ges_bin_sort");
  ges_status st = use_device(f->ctx->device);
  if (st != GES_OK) return st;
  f->vt.t.v[0].img = img;
  f->vt.t.v[0].final_T = final_T;
  f->vt.t.v[0].n_contrib = n_contrib;
  {
    TraceScope tr(f->ctx, "k_render_fwd", (cudaStream_t)stream);
    launch_render_fwd<FrameViews>(f->vt, f->n_tiles, f->ranges, f->tile_keys, f->tile_vals, f->rec, f->P,
                                  (cudaStream_t)stream);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "render_fwd launch");
  return GES_OK;
}

ges_status ges_render_bwd(ges_frame* f, const ges_scene* scene, const float* final_T, const uint32_t* n_contrib,
                          const float* dL_dimg, const ges_grads* out, void* stream) {
  if (!f || !final_T || !n_contrib || !dL_dimg || !out) return fail(GES_ERR_INVALID_ARG, "NULL argument");
  if (!f->have_sort) return fail(GES_ERR_INVALID_ARG, "ges_render_bwd before ges_bin_sort");
  ges_status st;
  if ((st = check_scene(scene)) != GES_OK) return st;
  if (scene->n != f->n || scene->sh_degree != f->sh_degree)
    return fail(GES_ERR_INVALID_ARG, "scene differs from the one preprocessed");
  if (f->n > 0 && (!out->means || !out->scales || !out->quats || !out->betas || !out->opacities || !out->shs))
    return fail(GES_ERR_INVALID_ARG, "gradient pointer is NULL");
  if ((((uintptr_t)out->quats) & 15u) || (((uintptr_t)out->shs) & 15u))
    return fail(GES_ERR_INVALID_ARG, "gradient quats and shs must be 16-byte aligned");
  if ((st = use_device(f->ctx->device)) != GES_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  ViewDesc& v = f->vt.t.v[0];
  v.means = scene->means; v.scales = scene->scales; v.quats = scene->quats; v.betas = scene->betas;
  v.opac = scene->opacities; v.shs = scene->shs;
  v.final_T = const_cast<float*>(final_T);
  v.n_contrib = const_cast<uint32_t*>(n_contrib);
  v.dL_dimg = dL_dimg;
  v.g_means = out->means; v.g_scales = out->scales; v.g_quats = out->quats; v.g_betas = out->betas;
  v.g_opac = out->opacities; v.g_shs = out->shs;
  cudaError_t e;
  if (f->n > 0 && (e = cudaMemsetAsync(f->g2d, 0, sizeof(float4) * 3 * f->n, s)) != cudaSuccess)
    return cuda_fail(e, "memset g2d");
  {
    TraceScope tr(f->ctx, "tile_order", s);
    launch_tile_order<FrameViews>(f->vt, f->n_tiles, f->tile_bucket, f->order_count, f->tile_order, s);
  }
  {
    TraceScope tr(f->ctx, "k_render_bwd", s);
    launch_render_bwd<FrameViews>(f->vt, f->n_tiles, f->ranges, f->tile_keys, f->tile_vals, f->rec, f->P, f->g2d, s,
                                  f->tile_order);
  }
  {
    TraceScope tr(f->ctx, "k_preprocess_bwd", s);
    launch_preprocess_bwd<FrameViews>(f->vt, f->n, f->P, f->depth_key, f->g2d, f->ctx->num_sms, s);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "render_bwd launch");
  f->have_bwd = true;
  return GES_OK;
}

ges_status ges_frame_status(ges_frame* f, void* stream, int64_t* num_keys) {
  if (!f) return fail(GES_ERR_INVALID_ARG, "frame is NULL");
  ges_status st = use_device(f->ctx->device);
  if (st != GES_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stream sync");
  unsigned long long K = 0;
  uint32_t flags = 0;
  if ((e = cudaMemcpy(&K, f->d_K, 8, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e, "read K");
  if ((e = cudaMemcpy(&flags, f->d_flags, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_fail(e, "read flags");
  if (num_keys) *num_keys = (int64_t)K;
  if (flags & kFlagOverflow)
    return fail(GES_ERR_CAPACITY, "K=%llu duplicates exceed key capacity %lld", K, (long long)f->key_cap);
  if (flags & kFlagSortWait)
    return fail(GES_ERR_DEVICE_WAIT, "a radix sort's bounded look-back gave up; the frame's lists are invalid");
  return GES_OK;
}

ges_status ges_frame_keys(ges_frame* f, void* stream, uint64_t* keys, uint32_t* vals, int64_t max_keys, int64_t* num_keys) {
  if (!f) return fail(GES_ERR_INVALID_ARG, "frame is NULL");
  if (!f->have_sort) return fail(GES_ERR_INVALID_ARG, "no sorted keys yet");
  ges_status st = use_device(f->ctx->device);
  if (st != GES_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<uint32_t> tv, dk;
  const bool copy = (keys || vals) && max_keys > 0;
  if (copy) {
    int64_t K = 0;
    if ((st = ges_frame_status(f, stream, &K)) != GES_OK) return st;
    tv.resize((size_t)K);
    dk.resize((size_t)f->n);
    cudaError_t e;
    if (K && (e = cudaMemcpy(tv.data(), f->tile_vals, 4 * (size_t)K, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "copy list values");
    if (f->n && (e = cudaMemcpy(dk.data(), f->depth_key, 4 * (size_t)f->n, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "copy depth keys");
  }
  std::vector<uint32_t> tk;
  int64_t count = 0;
  st = walk_tile_lists(f, s, tk, [&](int64_t tile, uint32_t i) {
    if (copy && count < max_keys) {
      const uint32_t g = tv[i];
      if (keys) keys[count] = ((uint64_t)tile << 32) | dk[g];
      if (vals) vals[count] = g;
    }
    ++count;
  }, nullptr);
  if (num_keys) *num_keys = count;
  return st;
}

ges_status ges_frame_inspect(ges_frame* f, void* stream, uint32_t* depth_key, int32_t* rect, float* record,
                             uint32_t* ranges, float* grad2d) {
  if (!f) return fail(GES_ERR_INVALID_ARG, "frame is NULL");
  ges_status st = use_device(f->ctx->device);
  if (st != GES_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stream sync");
  const int64_t n = f->n;
  if (depth_key && n && (e = cudaMemcpy(depth_key, f->depth_key, 4 * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "copy depth keys");
  if (rect && n) {
    std::vector<ushort4> r((size_t)n);
    if ((e = cudaMemcpy(r.data(), f->rect, sizeof(ushort4) * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "copy rects");
    for (int64_t i = 0; i < n; ++i) {
      rect[4 * i] = r[i].x; rect[4 * i + 1] = r[i].y; rect[4 * i + 2] = r[i].z; rect[4 * i + 3] = r[i].w;
    }
  }
  if (record && n && (e = cudaMemcpy(record, f->rec, sizeof(Rec) * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "copy records");
  if (ranges) {
    if (!f->have_sort) {
      std::memset(ranges, 0, sizeof(uint32_t) * 2 * f->n_tiles);
    } else {
      std::vector<uint32_t> tk;
      if ((st = walk_tile_lists(f, s, tk, [](int64_t, uint32_t) {}, ranges)) != GES_OK) return st;
    }
  }
  if (grad2d && n && (e = cudaMemcpy(grad2d, f->g2d, sizeof(float4) * 3 * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "copy grad2d");
  return GES_OK;
}

uint64_t ges_kernel_launches(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

ges_status ges_frame_count_work(ges_frame* f, void* stream, int64_t* evaluated, int64_t* in_extent, int64_t* composited,
                                int64_t* num_keys) {
  if (!f) return fail(GES_ERR_INVALID_ARG, "frame is NULL");
  if (!f->have_sort) return fail(GES_ERR_INVALID_ARG, "no sorted keys yet");
  ges_status st = use_device(f->ctx->device);
  if (st != GES_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t npx = (size_t)f->W * f->H;
  if (!f->work_img) {
    if ((st = ctx_alloc(f->ctx, (void**)&f->work_img, sizeof(float) * 5 * npx)) != GES_OK) return st;
    if ((st = ctx_alloc(f->ctx, (void**)&f->work_stats, 32)) != GES_OK) return st;
  }
  FrameViews vt = f->vt;
  vt.t.v[0].img = f->work_img;
  vt.t.v[0].final_T = f->work_img + 3 * npx;
  vt.t.v[0].n_contrib = reinterpret_cast<uint32_t*>(f->work_img + 4 * npx);
  cudaError_t e;
  if ((e = cudaMemsetAsync(f->work_stats, 0, 32, s)) != cudaSuccess) return cuda_fail(e, "memset stats");
  launch_render_fwd<FrameViews>(vt, f->n_tiles, f->ranges, f->tile_keys, f->tile_vals, f->rec, f->P, s, f->work_stats);
  unsigned long long h[3] = {0, 0, 0};
  if ((e = cudaMemcpyAsync(h, f->work_stats, 24, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(e, "copy stats");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "sync");
  if (evaluated) *evaluated = (int64_t)h[0];
  if (in_extent) *in_extent = (int64_t)h[1];
  if (composited) *composited = (int64_t)h[2];
  return ges_frame_status(f, stream, num_keys);
}

}  // extern "C"
