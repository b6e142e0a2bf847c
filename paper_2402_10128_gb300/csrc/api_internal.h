// Host-side structures behind the opaque handles of ges.h (shared by api.cu and serve.cu).
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "ges.h"
#include "common.cuh"
#include "kernels.cuh"

struct ges_trace_rec {
  const char* name;  // static string
  cudaEvent_t a, b;
};

constexpr int kScratchSlots = 3;  // 0 mask, 1 image loss, 2 density control

struct ges_ctx {
  int device = 0;
  size_t budget = 0;   // bytes this context may allocate (0 = unbounded)
  size_t used = 0;
  int num_sms = 0;
  std::mutex mu;
  // grow-only scratch of the calls that keep state in the context (ctx_scratch)
  std::mutex scratch_mu;
  void* scratch[kScratchSlots] = {};
  size_t scratch_bytes[kScratchSlots] = {};
  // kernel tracing (ges_trace_enable / ges_trace_read)
  bool trace_on = false;
  std::vector<ges_trace_rec> trace;
  std::vector<cudaEvent_t> event_pool;
};

struct ges_frame {
  ges_ctx* ctx = nullptr;
  int64_t n_cap = 0;
  int32_t W = 0, H = 0, tiles_x = 0, tiles_y = 0;
  int64_t n_tiles = 0;
  int64_t n_segs = 0;              // list segments of the current parameters (<= n_tiles)
  int64_t key_cap = 0;
  bool auto_cap = false;
  // per primitive
  uint32_t* depth_key = nullptr;  // float bits of the camera depth, kCulledKey if culled
  uint32_t* dk[2] = {nullptr, nullptr};
  uint32_t* pv[2] = {nullptr, nullptr};
  ushort4* rect = nullptr;
  ges::Rec* rec = nullptr;
  ges::KeyShape* ks = nullptr;     // what the key generation reads: extent shape, 2D mean, box
  uint32_t* tprim = nullptr;       // tiles met per primitive
  uint32_t* touched = nullptr;     // the same, in depth order
  unsigned long long* offsets = nullptr;
  float4* g2d = nullptr;
  // per duplicate
  uint32_t* tk[2] = {nullptr, nullptr};
  uint32_t* tv[2] = {nullptr, nullptr};
  uint32_t* hist = nullptr;
  int64_t hist_cap = 0;
  ges::ScanScratch scan;
  // per tile
  uint2* ranges = nullptr;
  uint32_t* tile_bucket = nullptr;   // the backward's cost class per tile
  uint32_t* tile_order = nullptr;    // the backward's launch order: heavy tiles first
  uint32_t* order_count = nullptr;   // [2 * kOrderBuckets]: tiles per class, then cursors
  // counters
  unsigned long long* d_K = nullptr;
  uint32_t* d_flags = nullptr;
  unsigned long long* h_K = nullptr;  // pinned
  // state of the current frame
  ges::FrameViews vt;
  ges::Params P;
  int64_t n = 0;
  int32_t sh_degree = 0;
  uint32_t* sorted_prims = nullptr;
  uint32_t* tile_keys = nullptr;
  uint32_t* tile_vals = nullptr;
  bool have_pre = false, have_sort = false, have_bwd = false;
  // scratch for ges_frame_count_work
  float* work_img = nullptr;
  unsigned long long* work_stats = nullptr;
};

namespace ges {
ges_status fail(ges_status st, const char* fmt, ...);
ges_status cuda_fail(cudaError_t e, const char* what);
ges_status ctx_alloc(ges_ctx* ctx, void** p, size_t bytes);
void ctx_free(ges_ctx* ctx, void* p, size_t bytes);
ges_status use_device(int device);
Params to_params(const ges_params& p);
ges_status check_params(const ges_params* p);
ges_status check_camera(const ges_camera* c);
ges_status check_scene(const ges_scene* s);
void fill_view(ViewDesc& v, const ges_camera& c, const ges_scene& s, int64_t prim_base, int32_t tile_base,
               int32_t seg_base, int seg_log2);
ges_status set_segment_bits(Params& P, int64_t total_segs);
void set_pack_bits(Params& P, int64_t n, int64_t segs_per_view);
int bits_for(int64_t count);
// grow-only device scratch of the context, one buffer per slot; replacing a buffer synchronises the device
ges_status ctx_scratch(ges_ctx* ctx, int slot, size_t bytes, void** out);
// brackets the launches made in its lifetime with an NVTX range (for profilers) and, when tracing
// is on, with two events on stream s
struct TraceScope {
  ges_ctx* c;
  const char* name;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  TraceScope(ges_ctx* c_, const char* name_, cudaStream_t s_);
  ~TraceScope();
  TraceScope(const TraceScope&) = delete;
  TraceScope& operator=(const TraceScope&) = delete;
};
}  // namespace ges
