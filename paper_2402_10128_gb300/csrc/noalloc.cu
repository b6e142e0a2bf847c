// ges_render_fwd_noalloc: the forward render (preprocess, binning sort, composite) for callers
// that cannot allocate device memory.
//
// Such callers exist: code that runs under another runtime's memory manager which has already
// reserved the device's memory for its own pool, or latency-critical loops where cudaMalloc /
// cudaFree are not acceptable because they can synchronise the whole device and stall unrelated
// streams.  This entry point therefore allocates nothing.  Every intermediate buffer of the
// pipeline lives in one fixed-size array in device global memory, declared below at file scope;
// the caller passes only its inputs (the scene) and its outputs (image, final transmittance,
// contributor count).
//
// The array costs kScratchBytes (about 24 MB) on every GPU that loads this library, for as long
// as the process lives.  All calls share it and it keeps the last call's contents, so calls whose
// work overlaps on the GPU (different streams, or different host threads on the same device)
// race on it and must be serialised by the caller.
#include <mutex>

#include "api_internal.h"

namespace ges {
namespace {

// Limits of one call.
constexpr int64_t kNaMaxPrims = 65536;     // primitives
constexpr int64_t kNaMaxKeys = 1 << 20;    // (tile, primitive) duplicates
constexpr int64_t kNaMaxTiles = 16384;     // 16x16 tiles (e.g. 2048 x 2048 pixels)
// radix-sort scratch of the one-sweep form: counters and digit counts (8 + 4 x 256), two status
// regions of 256 per 4096-key chunk
constexpr int64_t kNaHistEntries = 8 + 4 * 256 + 2 * 256 * ((kNaMaxKeys + 4095) / 4096);
constexpr int64_t kNaScanBytes = 4096;     // multi-level scan scratch for <= 2^20 elements

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Layout {
  size_t depth_key, dk0, dk1, pv0, pv1, rect, rec, ks, tprim, touched, offsets;
  size_t tk0, tk1, tv0, tv1, hist, scan, ranges, K, flags, total;
};

constexpr Layout make_layout() {
  Layout L{};
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.depth_key = take(4 * kNaMaxPrims);
  L.dk0 = take(4 * kNaMaxPrims);
  L.dk1 = take(4 * kNaMaxPrims);
  L.pv0 = take(4 * kNaMaxPrims);
  L.pv1 = take(4 * kNaMaxPrims);
  L.rect = take(8 * kNaMaxPrims);
  L.rec = take(sizeof(Rec) * kNaMaxPrims);
  L.ks = take(sizeof(KeyShape) * kNaMaxPrims);
  L.tprim = take(4 * kNaMaxPrims);
  L.touched = take(4 * kNaMaxPrims);
  L.offsets = take(8 * kNaMaxPrims);
  L.tk0 = take(4 * kNaMaxKeys);
  L.tk1 = take(4 * kNaMaxKeys);
  L.tv0 = take(4 * kNaMaxKeys);
  L.tv1 = take(4 * kNaMaxKeys);
  L.hist = take(4 * kNaHistEntries);
  L.scan = take(kNaScanBytes);
  L.ranges = take(8 * kNaMaxTiles);
  L.K = take(8);
  L.flags = take(4);
  L.total = o;
  return L;
}

constexpr Layout kL = make_layout();
constexpr size_t kScratchBytes = kL.total;

// The scratch array.  In host code this name is only a handle for cudaGetSymbolAddress, never a
// device address: kernels receive the address obtained below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceState {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch on this device
  int num_sms = 0;
};

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
DeviceState g_na_state[kMaxDevices];

// Once per device, with that device current: resolve the array's device address and upload the
// key-path constants.  Runs inside the first call on each device, so that first call should not be
// made while a stream is being captured.
ges_status setup_device(int device, DeviceState** out) {
  if (device < 0 || device >= kMaxDevices) return fail(GES_ERR_INVALID_ARG, "device %d out of range", device);
  std::lock_guard<std::mutex> lk(g_na_mu);
  DeviceState& st = g_na_state[device];
  if (!st.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    e = cudaDeviceGetAttribute(&st.num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    set_key_constants(0);
    e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return cuda_fail(e, "uploading key constants");
    st.base = static_cast<unsigned char*>(p);
    st.ready = true;
  }
  *out = &st;
  return GES_OK;
}

template <typename T>
T* at(unsigned char* base, size_t off) {
  return reinterpret_cast<T*>(base + off);
}

}  // namespace
}  // namespace ges

using namespace ges;

extern "C" ges_status ges_render_fwd_noalloc(const ges_scene* scene, const ges_camera* cam, const ges_params* params,
                                             float* img, float* final_T, uint32_t* n_contrib, void* stream) {
  ges_status st;
  if ((st = check_scene(scene)) != GES_OK || (st = check_camera(cam)) != GES_OK || (st = check_params(params)) != GES_OK)
    return st;
  if (!img || !final_T || !n_contrib) return fail(GES_ERR_INVALID_ARG, "output pointer is NULL");
  const int64_t tiles = (int64_t)((cam->width + kTile - 1) / kTile) * ((cam->height + kTile - 1) / kTile);
  if (scene->n > kNaMaxPrims)
    return fail(GES_ERR_INVALID_ARG, "no-alloc render: %lld primitives exceed the limit of %lld", (long long)scene->n,
                (long long)kNaMaxPrims);
  if (tiles > kNaMaxTiles)
    return fail(GES_ERR_INVALID_ARG, "no-alloc render: %dx%d image has %lld tiles, above the limit of %lld", cam->width,
                cam->height, (long long)tiles, (long long)kNaMaxTiles);
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  DeviceState* ds = nullptr;
  if ((st = setup_device(device, &ds)) != GES_OK) return st;

  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* b = ds->base;
  const int64_t n = scene->n;
  Params P = to_params(*params);
  FrameViews vt;
  vt.t.n = 1;
  fill_view(vt.t.v[0], *cam, *scene, 0, 0, 0, P.seg_log2);
  vt.t.total_prims = (unsigned long long)scene->n;
  vt.t.total_tiles = tiles;
  const int64_t segs = (int64_t)vt.t.v[0].segs_x * vt.t.v[0].tiles_y;
  vt.t.total_segs = segs;
  if ((st = set_segment_bits(P, segs)) != GES_OK) return st;
  set_pack_bits(P, n, segs);
  uint32_t* dk[2] = {at<uint32_t>(b, kL.dk0), at<uint32_t>(b, kL.dk1)};
  uint32_t* pv[2] = {at<uint32_t>(b, kL.pv0), at<uint32_t>(b, kL.pv1)};
  uint32_t* tk[2] = {at<uint32_t>(b, kL.tk0), at<uint32_t>(b, kL.tk1)};
  uint32_t* tv[2] = {at<uint32_t>(b, kL.tv0), at<uint32_t>(b, kL.tv1)};
  uint32_t* depth_key = at<uint32_t>(b, kL.depth_key);
  ushort4* rect = at<ushort4>(b, kL.rect);
  Rec* rec = at<Rec>(b, kL.rec);
  uint32_t* touched = at<uint32_t>(b, kL.touched);
  unsigned long long* offsets = at<unsigned long long>(b, kL.offsets);
  uint32_t* hist = at<uint32_t>(b, kL.hist);
  uint2* ranges = at<uint2>(b, kL.ranges);
  unsigned long long* dK = at<unsigned long long>(b, kL.K);
  uint32_t* flags = at<uint32_t>(b, kL.flags);
  ScanScratch scan;
  scan.buf = b + kL.scan;
  scan.bytes = kNaScanBytes;

  // what must start at zero on every call: the overflow flag and the segment ranges (empty
  // segments are never written by the ranges kernel)
  if ((e = cudaMemsetAsync(flags, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "clear flags");
  if ((e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * segs, s)) != cudaSuccess) return cuda_fail(e, "clear ranges");
  KeyShape* ks = at<KeyShape>(b, kL.ks);
  uint32_t* tprim = at<uint32_t>(b, kL.tprim);
  launch_preprocess<FrameViews>(vt, n, P, depth_key, dk[0], pv[0], rect, rec, ks, tprim, ds->num_sms, s);
  int cur = 0;
  if (!radix_sort_pairs(dk, pv, cur, n, nullptr, n, 32, hist, kNaHistEntries, scan, s, flags))
    return fail(GES_ERR_CUDA, "internal: depth-sort histogram exceeds its buffer");
  if (P.id_bits)
    scan_unpack_onepass(pv[cur], P.id_bits, offsets, n, dK, scan, flags, s);
  else
    scan_gather_onepass(tprim, pv[cur], touched, offsets, n, dK, scan, flags, s);
  launch_keygen<FrameViews>(vt, offsets, touched, dK, n, pv[cur], ks, P, kNaMaxKeys,
                            tk[0], tv[0], flags, s);
  int tcur = 0;
  if (!radix_sort_pairs(tk, tv, tcur, 0, dK, kNaMaxKeys, P.seg_bits, hist, kNaHistEntries, scan, s, flags))
    return fail(GES_ERR_CUDA, "internal: list-sort histogram exceeds its buffer");
  launch_ranges(tk[tcur], dK, kNaMaxKeys, (uint32_t)((1ull << P.seg_bits) - 1), ranges, ds->num_sms, s);
  vt.t.v[0].img = img;
  vt.t.v[0].final_T = final_T;
  vt.t.v[0].n_contrib = n_contrib;
  launch_render_fwd<FrameViews>(vt, tiles, ranges, tk[tcur], tv[tcur], rec, P, s);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "no-alloc render launch");
  // the duplicate count is known only on the device: wait for it to report an overflow
  uint32_t h_flags = 0;
  unsigned long long h_K = 0;
  if ((e = cudaMemcpyAsync(&h_flags, flags, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(e, "read flags");
  if ((e = cudaMemcpyAsync(&h_K, dK, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return cuda_fail(e, "read K");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "stream sync");
  if (h_flags & kFlagOverflow)
    return fail(GES_ERR_CAPACITY, "no-alloc render: %llu duplicates exceed the limit of %lld (outputs hold the background only)", h_K,
                (long long)kNaMaxKeys);
  if (h_flags & kFlagSortWait) return fail(GES_ERR_DEVICE_WAIT, "no-alloc render: a radix sort's bounded look-back gave up");
  return GES_OK;
}
