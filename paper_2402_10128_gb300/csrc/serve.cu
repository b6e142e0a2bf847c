// Serving: several scenes resident on the device; render requests of mixed resolutions are
// admitted by memory into batches that run as one replay of a captured CUDA graph.
//
// A batch is a set of views (scene + camera) rendered together: the view table gives every
// view its range of global primitive ids and tile ids, so the preprocess, the depth sort, the
// keygen, the tile sort and the ranges run once over the whole batch, and one persistent
// compositing launch takes tiles of all views from a shared work counter.  Every kernel reads
// the view table and its counts from device memory and is sized by the workspace's fixed
// capacities, so the launch sequence is captured once per workspace and replayed for every batch;
// the host only rewrites the (pinned) table between replays.
//
// Continuous batching: a scheduler thread owns two workspaces.  While one batch runs, requests
// keep arriving; as soon as a workspace is free the next batch is formed from the queue (first in,
// first out, as many as fit the workspace's primitive, tile and pixel capacities and the slot
// limit) and launched, so consecutive batches overlap on the device.  A batch whose duplicate
// count overflows the key capacity is re-run with its requests one at a time.
#include <chrono>
#include <condition_variable>
#include <cstddef>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.h"

namespace ges {
namespace {

using Clock = std::chrono::steady_clock;

struct ResidentScene {
  ges_scene dev;   // device arrays owned by the server
  size_t bytes = 0;
};

enum ReqState { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Request {
  uint64_t ticket = 0;
  int32_t scene = 0;
  ges_camera cam{};
  float* out = nullptr;   // host [3,H,W]
  int64_t npix = 0, tiles = 0;
  Clock::time_point t_submit;
  float latency_ms = 0.f;
  ReqState state = kQueued;
  ges_status status = GES_OK;
  std::string err;
  bool solo = false;      // re-run alone after an overflow in a shared batch
};

using Table = ViewTable<kServeMaxViews>;

struct Workspace {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaGraphExec_t graph = nullptr;
  int64_t P_cap = 0, T_cap = 0, X_cap = 0, K_cap = 0, hist_cap = 0;
  size_t bytes = 0;
  Table* d_vt = nullptr;
  Table* h_vt = nullptr;  // pinned
  uint32_t* depth_key = nullptr;
  uint32_t* dk[2] = {nullptr, nullptr};
  uint32_t* pv[2] = {nullptr, nullptr};
  ushort4* rect = nullptr;
  Rec* rec = nullptr;
  KeyShape* ks = nullptr;
  uint32_t* tprim = nullptr;
  uint32_t* touched = nullptr;
  unsigned long long* offsets = nullptr;
  uint32_t* tk[2] = {nullptr, nullptr};
  uint32_t* tv[2] = {nullptr, nullptr};
  uint32_t* hist = nullptr;
  ScanScratch scan;
  uint2* ranges = nullptr;
  float* img = nullptr;
  float* T = nullptr;
  uint32_t* nc = nullptr;
  unsigned long long* stat = nullptr;  // [0] = K, [1] = flags (as u64), [2] = tile counter
  float* h_img = nullptr;              // pinned
  unsigned long long* h_stat = nullptr;  // pinned
  std::vector<Request*> reqs;
  std::vector<int64_t> pix_off;
  bool busy = false;
  std::vector<std::pair<void*, size_t>> owned;
};

}  // namespace
}  // namespace ges

struct ges_server {
  ges_ctx* ctx = nullptr;
  ges::Params P{};
  int32_t max_slots = 1;
  int num_sms = 0;
  std::vector<ges::ResidentScene> scenes;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<ges::Request*> queue;
  std::unordered_map<uint64_t, ges::Request*> reqs;
  uint64_t next_ticket = 1;
  size_t queue_cap = 1 << 16;
  ges::Workspace ws[2];
  bool ws_ready = false;
  ges_status ws_status = GES_OK;
  std::string ws_err;
  std::thread worker;
  bool stop = false;
};

namespace ges {
namespace {

// capacities of one workspace
constexpr int64_t kMaxPixelsPerView = 2048 * 1088;

ges_status ws_alloc(ges_server* S, Workspace& w, int64_t P_cap, int64_t T_cap, int64_t X_cap, int64_t K_cap) {
  ges_ctx* c = S->ctx;
  ges_status st = GES_OK;
  auto A = [&](void** p, size_t b) {
    if (st != GES_OK) return;
    st = ctx_alloc(c, p, b);
    if (st == GES_OK) {
      w.owned.emplace_back(*p, b);
      w.bytes += b;
    }
  };
  w.P_cap = P_cap;
  w.T_cap = T_cap;
  w.X_cap = X_cap;
  w.K_cap = K_cap;
  // segment ids of a batch stay below T_cap (a view has at most as many segments as tiles)
  ges_status sst = set_segment_bits(S->P, T_cap);
  if (sst != GES_OK) return sst;
  const int tile_bits = S->P.seg_bits;
  const int64_t h1 = radix_hist_entries(P_cap, 32), h2 = radix_hist_entries(K_cap, tile_bits);
  w.hist_cap = h1 > h2 ? h1 : h2;
  A((void**)&w.d_vt, sizeof(Table));
  A((void**)&w.depth_key, 4 * P_cap);
  for (int i = 0; i < 2; ++i) {
    A((void**)&w.dk[i], 4 * P_cap);
    A((void**)&w.pv[i], 4 * P_cap);
    A((void**)&w.tk[i], 4 * K_cap);
    A((void**)&w.tv[i], 4 * K_cap);
  }
  A((void**)&w.rect, sizeof(ushort4) * P_cap);
  A((void**)&w.rec, sizeof(Rec) * P_cap);
  A((void**)&w.ks, sizeof(KeyShape) * P_cap);
  A((void**)&w.tprim, 4 * P_cap);
  A((void**)&w.touched, 4 * P_cap);
  A((void**)&w.offsets, 8 * P_cap);
  A((void**)&w.hist, 4 * w.hist_cap);
  w.scan.bytes = ScanScratch::required(w.hist_cap > P_cap ? w.hist_cap : P_cap);
  A(&w.scan.buf, w.scan.bytes);
  A((void**)&w.ranges, sizeof(uint2) * T_cap);
  A((void**)&w.img, sizeof(float) * 3 * X_cap);
  A((void**)&w.T, sizeof(float) * X_cap);
  A((void**)&w.nc, sizeof(uint32_t) * X_cap);
  A((void**)&w.stat, 32);
  if (st != GES_OK) return st;
  cudaError_t e;
  if ((e = cudaMallocHost((void**)&w.h_vt, sizeof(Table))) != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
  if ((e = cudaMallocHost((void**)&w.h_img, sizeof(float) * 3 * X_cap)) != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
  if ((e = cudaMallocHost((void**)&w.h_stat, 32)) != cudaSuccess) return cuda_fail(e, "cudaMallocHost");
  std::memset(w.h_vt, 0, sizeof(Table));
  if ((e = cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "stream");
  if ((e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "event");

  // capture the batch pipeline once; every replay reads the table copied in by its first node
  cudaStream_t s = w.stream;
  if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return cuda_fail(e, "begin capture");
  BatchViews vs;
  vs.p = w.d_vt;
  const unsigned long long* n_dev =
      reinterpret_cast<const unsigned long long*>(reinterpret_cast<const char*>(w.d_vt) + offsetof(Table, total_prims));
  unsigned long long* dK = w.stat;
  uint32_t* flags = reinterpret_cast<uint32_t*>(w.stat + 1);
  unsigned int* counter = reinterpret_cast<unsigned int*>(w.stat + 2);
  cudaMemcpyAsync(w.d_vt, w.h_vt, sizeof(Table), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(w.stat + 1, 0, 16, s);
  cudaMemsetAsync(w.ranges, 0, sizeof(uint2) * T_cap, s);
  launch_preprocess<BatchViews>(vs, P_cap, S->P, w.depth_key, w.dk[0], w.pv[0], w.rect, w.rec, w.ks, w.tprim, S->num_sms,
                                s);
  int cur = 0;
  bool fits = radix_sort_pairs(w.dk, w.pv, cur, 0, n_dev, P_cap, 32, w.hist, w.hist_cap, w.scan, s, flags);
  scan_gather_onepass(w.tprim, w.pv[cur], w.touched, w.offsets, P_cap, dK, w.scan, flags, s, n_dev);
  launch_keygen<BatchViews>(vs, w.offsets, w.touched, dK, P_cap, w.pv[cur], w.ks, S->P, K_cap,
                            w.tk[0], w.tv[0], flags, s, n_dev);
  int tcur = 0;
  fits = radix_sort_pairs(w.tk, w.tv, tcur, 0, dK, K_cap, tile_bits, w.hist, w.hist_cap, w.scan, s, flags) && fits;
  launch_ranges(w.tk[tcur], dK, K_cap, (uint32_t)((1ull << tile_bits) - 1), w.ranges, S->num_sms, s);
  launch_render_fwd<BatchViews>(vs, T_cap, w.ranges, w.tk[tcur], w.tv[tcur], w.rec, S->P, s, nullptr, counter,
                                S->num_sms);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s, &g);
  if (e != cudaSuccess) return cuda_fail(e, "end capture");
  if (!fits) {
    cudaGraphDestroy(g);
    return fail(GES_ERR_CUDA, "internal: a radix histogram exceeds its buffer");
  }
  e = cudaGraphInstantiate(&w.graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
  return GES_OK;
}

void ws_free(ges_server* S, Workspace& w) {
  if (w.stream) cudaStreamSynchronize(w.stream);
  if (w.graph) cudaGraphExecDestroy(w.graph);
  for (auto& pb : w.owned) ctx_free(S->ctx, pb.first, pb.second);
  w.owned.clear();
  if (w.h_vt) cudaFreeHost(w.h_vt);
  if (w.h_img) cudaFreeHost(w.h_img);
  if (w.h_stat) cudaFreeHost(w.h_stat);
  if (w.done) cudaEventDestroy(w.done);
  if (w.stream) cudaStreamDestroy(w.stream);
  w = Workspace();
}

// Sizes the two workspaces from the memory this context may still use (its budget, else 60% of the
// device's free memory), at most 96 GB each, once the resident scenes are known.  Duplicates take
// what the primitive, tile and pixel arrays leave, up to 2^31 - 2^20 entries per batch.
ges_status setup_workspaces(ges_server* S) {
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
  size_t avail;
  {
    std::lock_guard<std::mutex> lk(S->ctx->mu);
    avail = S->ctx->budget ? (S->ctx->budget > S->ctx->used ? S->ctx->budget - S->ctx->used : 0) : (size_t)(0.6 * free_b);
  }
  size_t per_ws = avail / 2;
  const size_t cap_ws = (size_t)96 << 30;
  if (per_ws > cap_ws) per_ws = cap_ws;
  int64_t n_max = 1;
  for (auto& sc : S->scenes) n_max = sc.dev.n > n_max ? sc.dev.n : n_max;
  const int64_t slots = S->max_slots;
  const int64_t X_cap = slots * kMaxPixelsPerView;
  const int64_t T_cap = X_cap / 256 + slots * 256;
  int64_t P_cap = slots * n_max;
  // per primitive 124 B, per pixel 20 B (+ 12 B pinned), per tile 8 B; duplicates take the rest
  const size_t fixed_px = (size_t)X_cap * 20 + (size_t)T_cap * 8;
  if ((size_t)P_cap * 124 > per_ws / 3) P_cap = (int64_t)(per_ws / 3 / 124);
  if (P_cap < n_max)
    return fail(GES_ERR_OOM, "serving workspace of %zu bytes cannot hold the largest scene (%lld primitives)", per_ws,
                (long long)n_max);
  const size_t used = (size_t)P_cap * 124 + fixed_px;
  if (used >= per_ws) return fail(GES_ERR_OOM, "serving workspace budget %zu bytes is too small", per_ws);
  int64_t K_cap = (int64_t)((per_ws - used) / 17);
  const int64_t k_limit = ((int64_t)1 << 31) - ((int64_t)1 << 20);
  if (K_cap > k_limit) K_cap = k_limit;
  for (int i = 0; i < 2; ++i) {
    ges_status st = ws_alloc(S, S->ws[i], P_cap, T_cap, X_cap, K_cap);
    if (st != GES_OK) return st;
  }
  return GES_OK;
}

// Fills the workspace's table from the batch and launches it (graph replay + result copies).
ges_status ws_launch(ges_server* S, Workspace& w) {
  Table& t = *w.h_vt;
  std::memset(&t, 0, sizeof(Table));
  int64_t prim = 0, tile = 0, seg = 0, pix = 0;
  w.pix_off.clear();
  for (size_t i = 0; i < w.reqs.size(); ++i) {
    Request* r = w.reqs[i];
    const ResidentScene& sc = S->scenes[r->scene];
    fill_view(t.v[i], r->cam, sc.dev, prim, (int32_t)tile, (int32_t)seg, S->P.seg_log2);
    seg += (int64_t)t.v[i].segs_x * t.v[i].tiles_y;
    t.v[i].img = w.img + 3 * pix;
    t.v[i].final_T = w.T + pix;
    t.v[i].n_contrib = w.nc + pix;
    w.pix_off.push_back(pix);
    prim += sc.dev.n;
    tile += r->tiles;
    pix += r->npix;
  }
  t.n = (int32_t)w.reqs.size();
  t.total_prims = (unsigned long long)prim;
  t.total_tiles = tile;
  t.total_segs = seg;
  cudaError_t e;
  if ((e = cudaGraphLaunch(w.graph, w.stream)) != cudaSuccess) return cuda_fail(e, "graph launch");
  if ((e = cudaMemcpyAsync(w.h_img, w.img, sizeof(float) * 3 * pix, cudaMemcpyDeviceToHost, w.stream)) != cudaSuccess)
    return cuda_fail(e, "copy images");
  if ((e = cudaMemcpyAsync(w.h_stat, w.stat, 16, cudaMemcpyDeviceToHost, w.stream)) != cudaSuccess)
    return cuda_fail(e, "copy status");
  if ((e = cudaEventRecord(w.done, w.stream)) != cudaSuccess) return cuda_fail(e, "record");
  return GES_OK;
}

// Picks the next batch from the queue (caller holds the lock).  FIFO: stops at the first request
// that does not fit.  A request that cannot fit an empty workspace fails.
void take_batch(ges_server* S, Workspace& w) {
  w.reqs.clear();
  int64_t P = 0, T = 0, X = 0;
  const size_t slots = (size_t)(S->max_slots < kServeMaxViews ? S->max_slots : kServeMaxViews);
  while (!S->queue.empty() && w.reqs.size() < slots) {
    Request* r = S->queue.front();
    const int64_t n = S->scenes[r->scene].dev.n;
    if (n > w.P_cap || r->tiles > w.T_cap || r->npix > w.X_cap) {
      S->queue.pop_front();
      r->state = kFailed;
      r->status = GES_ERR_OOM;
      r->err = "request exceeds the serving workspace";
      continue;
    }
    if (r->solo && !w.reqs.empty()) break;
    if (P + n > w.P_cap || T + r->tiles > w.T_cap || X + r->npix > w.X_cap) break;
    S->queue.pop_front();
    r->state = kRunning;
    w.reqs.push_back(r);
    P += n;
    T += r->tiles;
    X += r->npix;
    if (r->solo) break;
  }
}

// Completes a finished batch (caller does not hold the lock).
void ws_finish(ges_server* S, Workspace& w) {
  const bool overflow = (w.h_stat[1] & kFlagOverflow) != 0;
  const bool sort_wait = (w.h_stat[1] & kFlagSortWait) != 0;
  const auto now = Clock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  if (sort_wait) {
    for (Request* r : w.reqs) {
      r->state = kFailed;
      r->status = GES_ERR_DEVICE_WAIT;
      r->err = "a radix sort's bounded look-back gave up";
    }
  } else if (overflow) {
    if (w.reqs.size() > 1) {
      for (auto it = w.reqs.rbegin(); it != w.reqs.rend(); ++it) {
        (*it)->solo = true;
        (*it)->state = kQueued;
        S->queue.push_front(*it);
      }
    } else {
      for (Request* r : w.reqs) {
        r->state = kFailed;
        r->status = GES_ERR_CAPACITY;
        r->err = "duplicate count exceeds the serving key capacity";
      }
    }
  } else {
    for (size_t i = 0; i < w.reqs.size(); ++i) {
      Request* r = w.reqs[i];
      std::memcpy(r->out, w.h_img + 3 * w.pix_off[i], sizeof(float) * 3 * r->npix);
      r->latency_ms = std::chrono::duration<float, std::milli>(now - r->t_submit).count();
      r->state = kDone;
    }
  }
  w.reqs.clear();
  w.busy = false;
  S->cv.notify_all();
}

void worker_main(ges_server* S) {
  use_device(S->ctx->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool any_busy = false;
    for (auto& w : S->ws) {
      if (!w.busy) continue;
      const cudaError_t q = cudaEventQuery(w.done);
      if (q == cudaSuccess) {
        lk.unlock();
        ws_finish(S, w);
        lk.lock();
      } else if (q == cudaErrorNotReady) {
        any_busy = true;
      } else {
        for (Request* r : w.reqs) {
          r->state = kFailed;
          r->status = GES_ERR_CUDA;
          r->err = cudaGetErrorString(q);
        }
        w.reqs.clear();
        w.busy = false;
        S->cv.notify_all();
      }
    }
    if (S->stop && S->queue.empty() && !any_busy) break;
    if (!S->queue.empty()) {
      if (!S->ws_ready && S->ws_status == GES_OK) {
        lk.unlock();
        ges_status st = setup_workspaces(S);
        std::string msg = st == GES_OK ? "" : ges_last_error();
        lk.lock();
        S->ws_status = st;
        S->ws_err = msg;
        S->ws_ready = st == GES_OK;
      }
      if (S->ws_status != GES_OK) {
        while (!S->queue.empty()) {
          Request* r = S->queue.front();
          S->queue.pop_front();
          r->state = kFailed;
          r->status = S->ws_status;
          r->err = S->ws_err;
        }
        S->cv.notify_all();
        continue;
      }
      Workspace* freew = nullptr;
      for (auto& w : S->ws)
        if (!w.busy) { freew = &w; break; }
      if (freew) {
        take_batch(S, *freew);
        S->cv.notify_all();
        if (!freew->reqs.empty()) {
          freew->busy = true;
          lk.unlock();
          ges_status st = ws_launch(S, *freew);
          std::string msg = st == GES_OK ? "" : ges_last_error();
          lk.lock();
          if (st != GES_OK) {
            for (Request* r : freew->reqs) {
              r->state = kFailed;
              r->status = st;
              r->err = msg;
            }
            freew->reqs.clear();
            freew->busy = false;
            S->cv.notify_all();
          }
          continue;
        }
      }
    }
    if (any_busy)
      S->cv.wait_for(lk, std::chrono::microseconds(50));
    else
      S->cv.wait(lk, [&] { return S->stop || !S->queue.empty(); });
  }
}

}  // namespace
}  // namespace ges

using namespace ges;

extern "C" {

ges_status ges_serve_create(ges_ctx* ctx, const ges_params* params, int32_t max_slots, ges_server** out) {
  if (!ctx || !out) return fail(GES_ERR_INVALID_ARG, "ctx/out is NULL");
  *out = nullptr;
  ges_status st;
  if ((st = check_params(params)) != GES_OK) return st;
  if (max_slots < 1 || max_slots > kServeMaxViews)
    return fail(GES_ERR_INVALID_ARG, "max_slots %d not in [1,%d]", max_slots, kServeMaxViews);
  if ((st = use_device(ctx->device)) != GES_OK) return st;
  ges_server* S = new (std::nothrow) ges_server();
  if (!S) return fail(GES_ERR_OOM, "host allocation failed");
  S->ctx = ctx;
  S->P = to_params(*params);
  S->max_slots = max_slots;
  S->num_sms = ctx->num_sms;
  S->worker = std::thread(worker_main, S);
  *out = S;
  return GES_OK;
}

ges_status ges_serve_add_scene(ges_server* S, const ges_scene* hs, int32_t* scene_id) {
  if (!S || !scene_id) return fail(GES_ERR_INVALID_ARG, "NULL argument");
  ges_status st;
  if ((st = check_scene(hs)) != GES_OK) return st;
  if (hs->n < 1) return fail(GES_ERR_INVALID_ARG, "empty scene");
  if ((st = use_device(S->ctx->device)) != GES_OK) return st;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->ws_ready) return fail(GES_ERR_BUSY, "scenes must be added before the first request");
  }
  ResidentScene rs;
  rs.dev = *hs;
  const int64_t n = hs->n;
  const int nb = (hs->sh_degree + 1) * (hs->sh_degree + 1);
  const size_t sizes[6] = {12 * (size_t)n, 12 * (size_t)n, 16 * (size_t)n, 4 * (size_t)n, 4 * (size_t)n,
                           12 * (size_t)nb * n};
  const float* src[6] = {hs->means, hs->scales, hs->quats, hs->betas, hs->opacities, hs->shs};
  float* dst[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  for (int k = 0; k < 6; ++k) {
    if ((st = ctx_alloc(S->ctx, (void**)&dst[k], sizes[k])) != GES_OK) {
      for (int j = 0; j < k; ++j) ctx_free(S->ctx, dst[j], sizes[j]);
      return st;
    }
    cudaError_t e = cudaMemcpy(dst[k], src[k], sizes[k], cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      for (int j = 0; j <= k; ++j) ctx_free(S->ctx, dst[j], sizes[j]);
      return cuda_fail(e, "scene upload");
    }
    rs.bytes += sizes[k];
  }
  rs.dev.means = dst[0]; rs.dev.scales = dst[1]; rs.dev.quats = dst[2];
  rs.dev.betas = dst[3]; rs.dev.opacities = dst[4]; rs.dev.shs = dst[5];
  std::lock_guard<std::mutex> lk(S->mu);
  S->scenes.push_back(rs);
  *scene_id = (int32_t)S->scenes.size() - 1;
  return GES_OK;
}

ges_status ges_serve_submit(ges_server* S, int32_t scene_id, const ges_camera* cam, float* out_img, uint64_t* ticket) {
  if (!S || !out_img || !ticket) return fail(GES_ERR_INVALID_ARG, "NULL argument");
  ges_status st;
  if ((st = check_camera(cam)) != GES_OK) return st;
  Request* r = new (std::nothrow) Request();
  if (!r) return fail(GES_ERR_OOM, "host allocation failed");
  r->cam = *cam;
  r->out = out_img;
  r->npix = (int64_t)cam->width * cam->height;
  r->tiles = (int64_t)((cam->width + kTile - 1) / kTile) * ((cam->height + kTile - 1) / kTile);
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  if (scene_id < 0 || scene_id >= (int32_t)S->scenes.size()) {
    delete r;
    return fail(GES_ERR_INVALID_ARG, "unknown scene id %d", scene_id);
  }
  if (S->queue.size() >= S->queue_cap) {
    delete r;
    return fail(GES_ERR_BUSY, "request queue is full");
  }
  r->scene = scene_id;
  r->ticket = S->next_ticket++;
  S->reqs[r->ticket] = r;
  S->queue.push_back(r);
  *ticket = r->ticket;
  S->cv.notify_all();
  return GES_OK;
}

ges_status ges_serve_poll(ges_server* S, uint64_t ticket, int64_t timeout_us, float* latency_ms) {
  if (!S) return fail(GES_ERR_INVALID_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return fail(GES_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
  Request* r = it->second;
  auto finished = [&] { return r->state == kDone || r->state == kFailed; };
  if (!finished()) {
    if (timeout_us <= 0) return GES_ERR_NOT_READY;
    if (!S->cv.wait_for(lk, std::chrono::microseconds(timeout_us), finished)) return GES_ERR_TIMEOUT;
  }
  ges_status st = r->status;
  std::string msg = r->err;
  if (latency_ms) *latency_ms = r->latency_ms;
  S->reqs.erase(it);
  delete r;
  if (st != GES_OK) return fail(st, "%s", msg.c_str());
  return GES_OK;
}

ges_status ges_serve_destroy(ges_server* S) {
  if (!S) return GES_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  use_device(S->ctx->device);
  for (auto& w : S->ws) ws_free(S, w);
  for (auto& sc : S->scenes) {
    const int64_t n = sc.dev.n;
    const int nb = (sc.dev.sh_degree + 1) * (sc.dev.sh_degree + 1);
    ctx_free(S->ctx, (void*)sc.dev.means, 12 * (size_t)n);
    ctx_free(S->ctx, (void*)sc.dev.scales, 12 * (size_t)n);
    ctx_free(S->ctx, (void*)sc.dev.quats, 16 * (size_t)n);
    ctx_free(S->ctx, (void*)sc.dev.betas, 4 * (size_t)n);
    ctx_free(S->ctx, (void*)sc.dev.opacities, 4 * (size_t)n);
    ctx_free(S->ctx, (void*)sc.dev.shs, 12 * (size_t)nb * n);
  }
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
  return GES_OK;
}

}  // extern "C"
