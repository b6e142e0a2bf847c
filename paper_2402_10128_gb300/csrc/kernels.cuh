// Kernel entry points of libges and their launch helpers (host side).
#pragma once

#include "common.cuh"

namespace ges {

// kernels launched through the library by this process (all threads)
void count_launches(int n);

// ---- per-primitive kernels (preprocess.cu)
// VS is FrameViews (table by value) or BatchViews (table in device memory).  grid_total sizes the
// grid; the kernels loop over the table's total_prims.
// outputs per primitive: depth key (twice: kept and sort copy), sort value, bounding box of the
// extent in tiles, record, extent shape (2D covariance and q limit), tiles met (row spans)
template <class VS>
void launch_preprocess(const VS& vs, int64_t grid_total, const Params& P, uint32_t* depth_key, uint32_t* sort_keys,
                       uint32_t* sort_vals, ushort4* rect, Rec* rec, KeyShape* ks, uint32_t* tprim, int num_sms,
                       cudaStream_t s);
template <class VS>
void launch_preprocess_bwd(const VS& vs, int64_t grid_total, const Params& P, const uint32_t* depth_key,
                           const float4* g2d, int num_sms, cudaStream_t s);
void set_key_constants(cudaStream_t s);

// ---- binning (sort.cu)
struct ScanScratch {
  void* buf = nullptr;   // device scratch for multi-level scans; the first kReserved bytes hold counters
  size_t bytes = 0;
  static constexpr size_t kReserved = 256;
  static size_t required(int64_t max_n);
};
// exclusive prefix sum of n elements (in may equal out); *total (device, optional) gets the sum.
// With n_dev, the element count is min(*n_dev, n) (n is then the capacity).
template <typename TIn, typename TOut>
void scan_exclusive(const TIn* in, TOut* out, int64_t n, TOut* total, ScanScratch& sc, cudaStream_t s,
                    const unsigned long long* n_dev = nullptr);

// the same for uint32 counts into 64-bit offsets, in one launch (decoupled look-back); a bounded
// wait that gives up sets kFlagSortWait in *flags (when given).  Uses the scratch that
// scan_exclusive would, so the two must not run at the same time on one ScanScratch.
void scan_exclusive_onepass(const uint32_t* in, unsigned long long* out, int64_t n, unsigned long long* total,
                            ScanScratch& sc, uint32_t* flags, cudaStream_t s, const unsigned long long* n_dev = nullptr);
void scan_exclusive_onepass(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, ScanScratch& sc,
                            uint32_t* flags, cudaStream_t s, const unsigned long long* n_dev = nullptr);

// the same over packed[j] >> shift (the list entries that the depth sort's values carry above the
// primitive id)
void scan_unpack_onepass(const uint32_t* packed, int shift, unsigned long long* out, int64_t n,
                         unsigned long long* total, ScanScratch& sc, uint32_t* flags, cudaStream_t s,
                         const unsigned long long* n_dev = nullptr);
// the same over counts[ids[j]]: gathered[j] = counts[ids[j]] and out[j] = the sum of gathered[0..j)
// for j < count (min(*n_dev, n) with n_dev, else n); *total gets the sum.  The list entries of the
// primitives in depth order and their offsets, in one launch.
void scan_gather_onepass(const uint32_t* counts, const uint32_t* ids, uint32_t* gathered, unsigned long long* out,
                         int64_t n, unsigned long long* total, ScanScratch& sc, uint32_t* flags, cudaStream_t s,
                         const unsigned long long* n_dev = nullptr);

// stable LSD radix sort of (u32 key, u32 value) on the low `total_bits` bits.  The element count is
// n_dev (device) if non-null, else n_host; buffers hold n_cap elements.  keys[cur]/vals[cur] hold the
// input; on return `cur` indexes the sorted output.  hist holds hist_cap entries; returns false,
// launching nothing, if a pass's histogram would not fit (radix_hist_entries gives the need).
// With hist_cap >= radix_hist_entries(n_cap, .), a sort of three or four passes runs in one sweep
// (digit counts in one read, one kernel per pass with a bounded decoupled look-back; a look-back
// that gives up sets kFlagSortWait in *flags when flags is given), else as hist / scan / scatter
// per pass.
// bin_ranges (optional, n_ranges entries): when the sort takes a single pass over all total_bits, the
// [start, end) range of every key value in the sorted output is written there from the pass's
// scanned histogram, and *ranges_done is set (else it is cleared and bin_ranges left alone)
bool radix_sort_pairs(uint32_t* keys[2], uint32_t* vals[2], int& cur, int64_t n_host, const unsigned long long* n_dev,
                      int64_t n_cap, int total_bits, uint32_t* hist, int64_t hist_cap, ScanScratch& sc, cudaStream_t s,
                      uint32_t* flags = nullptr, uint2* bin_ranges = nullptr, int64_t n_ranges = 0,
                      bool* ranges_done = nullptr);
int64_t radix_hist_entries(int64_t n_cap, int max_bits);

// n: primitives (the capacity when n_dev gives the count on the device); touched: list entries per
// primitive in depth order (the scan's input), not read when P.id_bits > 0 (sorted_vals then
// carries them above the id)
template <class VS>
void launch_keygen(const VS& vs, const unsigned long long* offsets, const uint32_t* touched,
                   const unsigned long long* K_dev, int64_t n, const uint32_t* sorted_vals, const KeyShape* ks,
                   const Params& P, int64_t cap,
                   uint32_t* tile_keys, uint32_t* tile_vals, uint32_t* flags, cudaStream_t s,
                   const unsigned long long* n_dev = nullptr);
// [start, end) per segment of the sorted list (segment id = key & seg_mask); ranges of empty
// segments are left as they are (the caller zeroes them)
void launch_ranges(const uint32_t* tile_keys, const unsigned long long* K_dev, int64_t cap, uint32_t seg_mask,
                   uint2* ranges, int num_sms, cudaStream_t s);

constexpr uint32_t kFlagOverflow = 1u;
constexpr uint32_t kFlagSortWait = 2u;  // a radix sort's bounded look-back gave up (results invalid)

// ---- compositing (raster.cu)
// ranges: per segment; keys, vals: the sorted list (segment key, primitive id).
// stats (optional, device u64[3]): numbers of (fragment, pixel) pairs evaluated before the stop, of
// those within the primitive's extent, and of those composited.
// One CTA per tile (grid = total_tiles), or, with tile_counter, a persistent grid whose CTAs take
// tiles from *tile_counter (zeroed by the caller) until the table's total_tiles are done.
template <class VS>
void launch_render_fwd(const VS& vs, int64_t total_tiles, const uint2* ranges, const uint32_t* keys,
                       const uint32_t* vals, const Rec* rec, const Params& P, cudaStream_t s,
                       unsigned long long* stats = nullptr, unsigned int* tile_counter = nullptr, int num_sms = 0);
template <class VS>
void launch_render_bwd(const VS& vs, int64_t total_tiles, const uint2* ranges, const uint32_t* keys,
                       const uint32_t* vals, const Rec* rec, const Params& P, float4* g2d, cudaStream_t s,
                       const uint32_t* order = nullptr);

// Launch order of the backward's tiles, heaviest first: a tile's cost is the sum over its four 8x8
// warp blocks of the largest n_contrib, binned on a log scale (kOrderBuckets classes, 8 per
// octave); counts (2 * kOrderBuckets uint32, zeroed here) give each class its range of order[].
constexpr int kOrderBuckets = 256;
template <class VS>
void launch_tile_order(const VS& vs, int64_t total_tiles, uint32_t* bucket, uint32_t* counts, uint32_t* order,
                       cudaStream_t s);

}  // namespace ges
