// Binning: duplicate (tile, primitive) keys and sort them by tile, then depth.
//
// The result is a stable sort of the 64-bit keys (tile << 32 | depth bits) with values =
// primitive index, computed as an LSD radix sort whose low 32-bit passes run on the N
// primitives instead of the K duplicates: every duplicate of a primitive shares its depth
// bits, so sorting primitives by depth first and duplicating them in that order gives the
// same list as sorting the duplicates on the depth digits.  The remaining passes are a
// stable radix sort of the duplicates on their segment id alone (ceil(log2 segments) bits).
//   K2  list entries per primitive in depth order (unpacked from the sorted values, or gathered
//       through the sorted ids) and their exclusive scan (u64 offsets, K on the device), one launch
//   K3  keygen: load-balanced walk of (primitive, row) slots, one lane per slot
//   K4  stable LSD radix passes (<= 8-bit digits): per-chunk histogram, scan, stable scatter
//   K5  per-tile [start, end) from the sorted tile ids
#include <atomic>

#include "common.cuh"
#include "kernels.cuh"

namespace ges {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kChunk = kThreads * kItems;  // elements per CTA in scans and radix passes

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, v, o);
    if ((int)lane_id() >= o) v += y;
  }
  return v;
}

// ---------------------------------------------------------------- scan kernels
// element count of a scan: min(*n_dev, cap) when a device count is given, else cap
__device__ __forceinline__ int64_t scan_count(int64_t cap, const unsigned long long* n_dev) {
  if (!n_dev) return cap;
  const unsigned long long n = *n_dev;
  return n < (unsigned long long)cap ? (int64_t)n : cap;
}

template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kThreads) k_scan_reduce(const TIn* __restrict__ in, int64_t cap,
                                                          const unsigned long long* __restrict__ n_dev,
                                                          TOut* __restrict__ sums) {
  const int64_t n = scan_count(cap, n_dev);
  const int64_t base = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kItems;
  TOut acc = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k)
    if (base + k < n) acc += (TOut)in[base + k];
  __shared__ TOut red[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane_id() == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    TOut t = 0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    sums[blockIdx.x] = t;
  }
}

// exclusive scan of one chunk per CTA plus a per-CTA offset (block_off may be null)
template <typename TIn, typename TOut>
__global__ void __launch_bounds__(kThreads) k_scan_down(const TIn* __restrict__ in, TOut* __restrict__ out, int64_t cap,
                                                        const unsigned long long* __restrict__ n_dev,
                                                        const TOut* __restrict__ block_off, TOut* __restrict__ total) {
  const int64_t n = scan_count(cap, n_dev);
  if ((int64_t)blockIdx.x * kChunk >= n && !(total && gridDim.x == 1)) return;  // idle CTA past the count
  const int64_t base = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kItems;
  TOut v[kItems];
  TOut acc = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    v[k] = (base + k < n) ? (TOut)in[base + k] : TOut(0);
    acc += v[k];
  }
  __shared__ TOut ws[kThreads / 32 + 1];
  TOut inc = warp_inclusive_scan(acc);
  const int w = threadIdx.x >> 5;
  if (lane_id() == 31) ws[w] = inc;
  __syncthreads();
  if (w == 0) {
    TOut x = (lane_id() < kThreads / 32) ? ws[lane_id()] : TOut(0);
    TOut xi = warp_inclusive_scan(x);
    if (lane_id() < kThreads / 32) ws[lane_id()] = xi - x;
    if (lane_id() == 31) ws[kThreads / 32] = xi;
  }
  __syncthreads();
  TOut run = inc - acc + ws[w] + (block_off ? block_off[blockIdx.x] : TOut(0));
  // in may alias out: all loads of this thread happened above
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  // single-block scans report the total here; multi-level scans get it from the level above
  if (total && gridDim.x == 1 && threadIdx.x == 0) *total = ws[kThreads / 32];
}

// ---------------------------------------------------------------- radix kernels
// hist layout: [bin][chunk] so that one exclusive scan gives every (bin, chunk) output offset
// element count of a radix pass: the device count (0 if it exceeds the buffer capacity) or the host one
__device__ __forceinline__ int64_t element_count(int64_t n_host, const unsigned long long* n_dev, int64_t cap) {
  if (!n_dev) return n_host;
  const unsigned long long n = *n_dev;
  return n > (unsigned long long)cap ? 0 : (int64_t)n;
}

// hist layout: [bin][chunk] over the active chunks (ceil(count / kChunk)); the matrix size goes to
// *entries (device) for the scan that follows
template <int NB>
__global__ void __launch_bounds__(kThreads) k_radix_hist(const uint32_t* __restrict__ keys, int64_t n_host,
                                                         const unsigned long long* __restrict__ n_dev, int64_t cap,
                                                         int shift, int bits, uint32_t* __restrict__ hist,
                                                         unsigned long long* __restrict__ entries) {
  constexpr int kWarps = kThreads / 32;
  __shared__ uint32_t cnt[kWarps][NB];  // one private histogram per warp: less atomic contention
  const int nbins = 1 << bits;
  const int64_t n = element_count(n_host, n_dev, cap);
  const uint32_t mask = (uint32_t)nbins - 1u;
  const int w = threadIdx.x >> 5;
  const int64_t nchunks = (n + kChunk - 1) / kChunk;
  if (blockIdx.x == 0 && threadIdx.x == 0) *entries = (unsigned long long)nbins * (unsigned long long)nchunks;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t base = c * kChunk;
    __syncthreads();
    for (int i = threadIdx.x; i < kWarps * NB; i += kThreads) (&cnt[0][0])[i] = 0;
    __syncthreads();
    if (base + kChunk <= n) {
      const uint4* k4 = reinterpret_cast<const uint4*>(keys + base);
#pragma unroll
      for (int k = 0; k < kItems / 4; ++k) {
        const uint4 v = k4[k * kThreads + threadIdx.x];
        atomicAdd(&cnt[w][(v.x >> shift) & mask], 1u);
        atomicAdd(&cnt[w][(v.y >> shift) & mask], 1u);
        atomicAdd(&cnt[w][(v.z >> shift) & mask], 1u);
        atomicAdd(&cnt[w][(v.w >> shift) & mask], 1u);
      }
    } else {
      for (int k = 0; k < kItems; ++k) {
        int64_t idx = base + (int64_t)k * kThreads + threadIdx.x;
        if (idx < n) atomicAdd(&cnt[w][(keys[idx] >> shift) & mask], 1u);
      }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += kThreads) {
      uint32_t t = 0;
#pragma unroll
      for (int ww = 0; ww < kWarps; ++ww) t += cnt[ww][b];
      hist[(int64_t)b * nchunks + c] = t;
    }
  }
}

// Stable scatter.  Warp w of the CTA owns chunk elements [w*256, (w+1)*256) and walks them in
// order, 32 at a time.  Lanes with equal digits (found with one ballot per digit bit) are ranked
// by lane order; the group's first lane adds the group size to the warp's running count of that
// digit with a shared-memory atomic and hands the old count to the group with a shuffle, so ranks
// preserve input order within each digit.  The chunk is then reordered by digit in shared memory
// and written out so that consecutive threads store consecutive positions of one digit's run.
constexpr int kScThreads = 512;                 // scatter CTA: twice the warps of the other kernels
constexpr int kScItems = kChunk / kScThreads;   // 8 items per thread, same chunk

// shared memory of k_radix_scatter<NB> (dynamic: above 48 KB for NB = 512)
template <int NB>
struct ScatterSmem {
  uint32_t wcnt[kScThreads / 32][NB];  // per warp and digit: running count, then prefix
  uint32_t goff[NB];
  uint32_t bstart[NB + 1];
  uint32_t wsum[kScThreads / 32];
  uint32_t skeys[kChunk];
  uint32_t svals[kChunk];
};

template <int NB>
__global__ void __launch_bounds__(kScThreads) k_radix_scatter(const uint32_t* __restrict__ keys_in,
                                                            const uint32_t* __restrict__ vals_in,
                                                            uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                                            int64_t n_host, const unsigned long long* __restrict__ n_dev,
                                                            int64_t cap, int shift, int bits,
                                                            const uint32_t* __restrict__ hist_scanned,
                                                            uint2* __restrict__ ranges, int64_t n_ranges) {
  constexpr int kWarps = kScThreads / 32;
  extern __shared__ __align__(16) unsigned char sc_smem[];
  ScatterSmem<NB>& sm = *reinterpret_cast<ScatterSmem<NB>*>(sc_smem);
  auto& wcnt = sm.wcnt;
  auto& goff = sm.goff;
  auto& bstart = sm.bstart;
  auto& wsum = sm.wsum;
  auto& skeys = sm.skeys;
  auto& svals = sm.svals;
  const int nbins = 1 << bits;
  const uint32_t mask = (uint32_t)nbins - 1u;
  const int64_t n = element_count(n_host, n_dev, cap);
  const int64_t nchunks = (n + kChunk - 1) / kChunk;
  const int w = threadIdx.x >> 5;
  const unsigned lane = lane_id();
  // a single pass over all the key bits: the [start, end) range of every bin in the output comes
  // from the scanned histogram ([bin][chunk], exclusive over the whole matrix): bin b starts where
  // its first chunk's entries go and ends where bin b + 1's start (the last bin at the count)
  if (ranges) {
    for (int64_t b = (int64_t)blockIdx.x * kScThreads + threadIdx.x; b < n_ranges; b += (int64_t)gridDim.x * kScThreads) {
      uint2 r = make_uint2(0u, 0u);
      if (nchunks > 0 && b < nbins) {
        r.x = hist_scanned[b * nchunks];
        r.y = b + 1 < nbins ? hist_scanned[(b + 1) * nchunks] : (uint32_t)n;
      }
      ranges[b] = r;
    }
  }
  for (int64_t c = blockIdx.x; c * kChunk < n; c += gridDim.x) {
  const int64_t base = c * kChunk;
  const int count = (int)min((int64_t)kChunk, n - base);
  __syncthreads();  // the previous chunk's readers of the shared arrays are done
  {
    uint4* z = reinterpret_cast<uint4*>(&wcnt[0][0]);
    for (int i = threadIdx.x; i < kWarps * NB / 4; i += kScThreads) z[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int b = threadIdx.x; b < nbins; b += kScThreads) goff[b] = hist_scanned[(int64_t)b * nchunks + c];
  __syncthreads();
  const unsigned lt_mask = (1u << lane) - 1u;
  uint32_t key[kScItems], val[kScItems], rank[kScItems];
#pragma unroll
  for (int r = 0; r < kScItems; ++r) {
    const int li = w * (kScItems * 32) + r * 32 + (int)lane;
    const bool ok = li < count;
    key[r] = ok ? keys_in[base + li] : 0u;
    val[r] = ok ? vals_in[base + li] : 0u;
  }
#pragma unroll
  for (int r = 0; r < kScItems; ++r) {
    const int li = w * (kScItems * 32) + r * 32 + (int)lane;
    const bool ok = li < count;
    const uint32_t d = (key[r] >> shift) & mask;
    unsigned peers = __ballot_sync(0xffffffffu, ok);
    for (int b = 0; b < bits; ++b) {
      const bool bit = (d >> b) & 1u;
      const unsigned bal = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? bal : ~bal;
    }
    const int leader = peers ? __ffs(peers) - 1 : 0;
    uint32_t prev = 0;
    if (ok && (int)lane == leader) prev = atomicAdd(&wcnt[w][d], (uint32_t)__popc(peers));
    prev = __shfl_sync(0xffffffffu, prev, leader);
    rank[r] = prev + (uint32_t)__popc(peers & lt_mask);
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, and the digit's total in the chunk
  uint32_t total = 0;
  if ((int)threadIdx.x < nbins) {
    const int b = threadIdx.x;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
      uint32_t cw = wcnt[ww][b];
      wcnt[ww][b] = total;
      total += cw;
    }
  }
  // exclusive scan of the digit totals over the CTA (thread b holds digit b)
  uint32_t inc = total;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if ((int)lane >= o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int ww = 0; ww < kWarps; ++ww) {
      uint32_t c = wsum[ww];
      wsum[ww] = run;
      run += c;
    }
  }
  __syncthreads();
  if ((int)threadIdx.x < nbins) bstart[threadIdx.x] = wsum[w] + inc - total;
  __syncthreads();
  // reorder the chunk by digit in shared memory
#pragma unroll
  for (int r = 0; r < kScItems; ++r) {
    const int li = w * (kScItems * 32) + r * 32 + (int)lane;
    if (li < count) {
      const int d = (int)((key[r] >> shift) & mask);
      const uint32_t pos = bstart[d] + wcnt[w][d] + rank[r];
      skeys[pos] = key[r];
      svals[pos] = val[r];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += kScThreads) {
    const uint32_t k = skeys[i];
    const int d = (int)((k >> shift) & mask);
    const uint32_t gpos = goff[d] + ((uint32_t)i - bstart[d]);
    keys_out[gpos] = k;
    vals_out[gpos] = svals[i];
  }
  }  // chunk loop
}

// ---------------------------------------------------------------- one-sweep radix sort
// The same stable LSD sort with one read of the keys for every pass's digit counts and one kernel
// per pass: a CTA takes the next chunk from a counter (so a chunk's predecessors are always
// running or done), ranks its elements as k_radix_scatter does, publishes its per-digit counts,
// and finds the counts of all earlier chunks by a decoupled look-back (Merrill & Garland): a chunk
// publishes its digit count as an aggregate (flag 1) at once and, when its own prefix is known,
// the inclusive prefix (flag 2); a successor adds aggregates walking back until it meets a prefix.
// Status words: flag in bits 30-31, count in bits 0-29 (so at most 2^30 elements).  Two status
// regions alternate between passes; each pass's CTAs zero their chunk's entries of the other one.
// Every wait is bounded: a CTA that gives up publishes a prefix of 0, writes nothing, and sets
// kFlagSortWait in the caller's flags (its successors then finish with wrong offsets but every
// store is bounds-checked).
constexpr int kOsMaxPasses = 4;
// keys per thread and per chunk of a one-sweep pass: 1.5M keys make 293 chunks, one wave of two
// CTAs per SM (4,096-key chunks took two rounds and measured 3% slower)
constexpr int kOsItems = 10;
constexpr int kOsChunk = kScThreads * kOsItems;
constexpr int64_t kOsHeader = 8 + kOsMaxPasses * 256;  // chunk counters per pass, digit counts per pass
constexpr uint32_t kOsAgg = 1u << 30, kOsPre = 2u << 30, kOsValue = (1u << 30) - 1u;
constexpr int kOsSpinLimit = 1 << 22;

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}
__device__ __forceinline__ void st_volatile_u32(uint32_t* p, uint32_t v) { *reinterpret_cast<volatile uint32_t*>(p) = v; }

__global__ void __launch_bounds__(kThreads) k_os_counts(const uint32_t* __restrict__ keys, int64_t n_host,
                                                        const unsigned long long* __restrict__ n_dev, int64_t cap,
                                                        int passes, int bits_per, int total_bits,
                                                        uint32_t* __restrict__ counts) {
  constexpr int kWarps = kThreads / 32;
  __shared__ uint32_t cnt[kWarps / 2][kOsMaxPasses][256];  // one histogram per warp pair
  for (int i = threadIdx.x; i < (kWarps / 2) * kOsMaxPasses * 256; i += kThreads) (&cnt[0][0][0])[i] = 0;
  __syncthreads();
  const int64_t n = element_count(n_host, n_dev, cap);
  const int h = (threadIdx.x >> 5) >> 1;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    const uint32_t k = keys[i];
    for (int p = 0; p < passes; ++p) {
      const int shift = p * bits_per;
      const int bits = (total_bits - shift) < bits_per ? (total_bits - shift) : bits_per;
      atomicAdd(&cnt[h][p][(k >> shift) & ((1u << bits) - 1u)], 1u);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < passes * 256; j += kThreads) {
    uint32_t t = 0;
#pragma unroll
    for (int hh = 0; hh < kWarps / 2; ++hh) t += (&cnt[hh][0][0])[j];
    if (t) atomicAdd(&counts[j], t);
  }
}

__global__ void __launch_bounds__(kScThreads) k_os_scatter(const uint32_t* __restrict__ keys_in,
                                                         const uint32_t* __restrict__ vals_in,
                                                         uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                                                         int64_t n_host, const unsigned long long* __restrict__ n_dev,
                                                         int64_t cap, int shift, int bits, int pass, int zero_next,
                                                         uint32_t* __restrict__ os, int64_t nchunks_cap,
                                                         uint32_t* __restrict__ flags) {
  constexpr int kWarps = kScThreads / 32;
  __shared__ __align__(16) uint32_t wcnt[kWarps][256];
  __shared__ uint32_t goff[256];
  __shared__ uint32_t dbase[256];
  __shared__ uint32_t bstart[257];
  __shared__ uint32_t wsum[kWarps];
  __shared__ uint32_t skeys[kOsChunk];
  __shared__ uint32_t svals[kOsChunk];
  __shared__ int64_t s_chunk;
  __shared__ int s_fail;
  const int nbins = 1 << bits;
  const uint32_t mask = (uint32_t)nbins - 1u;
  const int64_t n = element_count(n_host, n_dev, cap);
  const int64_t nchunks = (n + kOsChunk - 1) / kOsChunk;
  const int w = threadIdx.x >> 5;
  const unsigned lane = lane_id();
  uint32_t* counter = os + pass;
  const uint32_t* counts = os + 8 + pass * 256;
  uint32_t* st_cur = os + kOsHeader + (int64_t)(pass & 1) * 256 * nchunks_cap;  // [chunk][digit]
  uint32_t* st_next = os + kOsHeader + (int64_t)((pass + 1) & 1) * 256 * nchunks_cap;
  // exclusive digit offsets of this pass (the same in every CTA)
  if (threadIdx.x < 32) {
    uint32_t run = 0;
    for (int b0 = 0; b0 < nbins; b0 += 32) {
      const int b = b0 + (int)lane;
      const uint32_t c = b < nbins ? counts[b] : 0u;
      uint32_t inc = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if ((int)lane >= o) inc += y;
      }
      if (b < nbins) dbase[b] = run + inc - c;
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
  for (;;) {
    __syncthreads();  // the previous chunk's readers of the shared arrays (and of s_chunk) are done
    if (threadIdx.x == 0) {
      s_chunk = (int64_t)atomicAdd(counter, 1u);
      s_fail = 0;
    }
    {
      uint4* z = reinterpret_cast<uint4*>(&wcnt[0][0]);
      for (int i = threadIdx.x; i < kWarps * 256 / 4; i += kScThreads) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    const int64_t c = s_chunk;
    if (c >= nchunks) break;
    const int64_t base = c * kOsChunk;
    const int count = (int)min((int64_t)kOsChunk, n - base);
    const unsigned lt_mask = (1u << lane) - 1u;
    uint32_t key[kOsItems], val[kOsItems], rank[kOsItems];
#pragma unroll
    for (int r = 0; r < kOsItems; ++r) {
      const int li = w * (kOsItems * 32) + r * 32 + (int)lane;
      const bool ok = li < count;
      key[r] = ok ? keys_in[base + li] : 0u;
      val[r] = ok ? vals_in[base + li] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kOsItems; ++r) {
      const int li = w * (kOsItems * 32) + r * 32 + (int)lane;
      const bool ok = li < count;
      const uint32_t d = (key[r] >> shift) & mask;
      unsigned peers = __ballot_sync(0xffffffffu, ok);
      for (int b = 0; b < bits; ++b) {
        const bool bit = (d >> b) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
      }
      const int leader = peers ? __ffs(peers) - 1 : 0;
      uint32_t prev = 0;
      if (ok && (int)lane == leader) prev = atomicAdd(&wcnt[w][d], (uint32_t)__popc(peers));
      prev = __shfl_sync(0xffffffffu, prev, leader);
      rank[r] = prev + (uint32_t)__popc(peers & lt_mask);
    }
    __syncthreads();
    uint32_t total = 0;
    if ((int)threadIdx.x < nbins) {
      const int b = threadIdx.x;
#pragma unroll
      for (int ww = 0; ww < kWarps; ++ww) {
        const uint32_t cw = wcnt[ww][b];
        wcnt[ww][b] = total;
        total += cw;
      }
      // decoupled look-back for digit b
      uint32_t* my = st_cur + c * 256 + b;
      if (zero_next) st_next[c * 256 + b] = 0u;
      uint32_t prefix = 0;
      if (c == 0) {
        st_volatile_u32(my, kOsPre | total);
      } else {
        st_volatile_u32(my, kOsAgg | total);
        int64_t look = c - 1;
        int spins = 0;
        for (;;) {
          const uint32_t v = ld_volatile_u32(st_cur + look * 256 + b);
          const uint32_t flag = v & ~kOsValue;
          if (flag == 0u) {
            if (++spins > kOsSpinLimit) {
              s_fail = 1;
              prefix = 0;
              break;
            }
            __nanosleep(32);
            continue;
          }
          prefix += v & kOsValue;
          if (flag == kOsPre || look == 0) break;
          --look;
        }
        st_volatile_u32(my, kOsPre | ((prefix + total) & kOsValue));
      }
      goff[b] = dbase[b] + prefix;
    }
    // exclusive scan of the digit totals over the CTA (thread b holds digit b)
    uint32_t inc = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if ((int)lane >= o) inc += y;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t run = 0;
      for (int ww = 0; ww < kWarps; ++ww) {
        const uint32_t cc = wsum[ww];
        wsum[ww] = run;
        run += cc;
      }
      if (s_fail && flags) atomicOr(flags, kFlagSortWait);
    }
    __syncthreads();
    if ((int)threadIdx.x < nbins) bstart[threadIdx.x] = wsum[w] + inc - total;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kOsItems; ++r) {
      const int li = w * (kOsItems * 32) + r * 32 + (int)lane;
      if (li < count) {
        const int d = (int)((key[r] >> shift) & mask);
        const uint32_t pos = bstart[d] + wcnt[w][d] + rank[r];
        skeys[pos] = key[r];
        svals[pos] = val[r];
      }
    }
    __syncthreads();
    if (!s_fail) {
      for (int i = threadIdx.x; i < count; i += kScThreads) {
        const uint32_t k = skeys[i];
        const int d = (int)((k >> shift) & mask);
        const int64_t gpos = (int64_t)goff[d] + ((uint32_t)i - bstart[d]);
        if (gpos < n) {
          keys_out[gpos] = k;
          vals_out[gpos] = svals[i];
        } else if (flags) {
          atomicOr(flags, kFlagSortWait);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- K3 keygen
// Primitive j (depth order) owns entries [offsets[j], offsets[j] + t_j), t_j its list entries (packed
// above the id in the sorted value when P.id_bits > 0, else touched[j]): per tile row of
// its bounding box, one entry per segment that the row's span meets, keyed seg_key(segment,
// span columns inside the segment).  A warp takes 32 consecutive primitives, whose entries are
// one contiguous range: it walks their (primitive, row) slots 32 at a time (one row span per
// lane), prefix-sums the slots' entry counts, and each lane writes its slot's entries (at most the
// segments of one tile row) at its offset.  Writes stay below K whatever the inputs.
constexpr int kKeygenThreads = 256;

template <class VS>
__global__ void __launch_bounds__(kKeygenThreads, 4) k_keygen(const __grid_constant__ VS vs,
                                                           const unsigned long long* __restrict__ offsets,
                                                           const unsigned long long* __restrict__ K_dev, int64_t n_cap,
                                                           const unsigned long long* __restrict__ n_dev,
                                                           const uint32_t* __restrict__ sorted_vals,
                                                           const uint32_t* __restrict__ touched,
                                                           const KeyShape* __restrict__ ks, const Params P, int64_t cap,
                                                           uint32_t* __restrict__ tile_keys,
                                                           uint32_t* __restrict__ tile_vals, uint32_t* __restrict__ flags) {
  const auto& vt = vs.get();
  const unsigned long long K = *K_dev;
  if ((int64_t)K > cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(flags, kFlagOverflow);
    return;
  }
  const int64_t n = scan_count(n_cap, n_dev);
  const unsigned lane = lane_id();
  const int L = P.seg_log2;
  const int64_t wpb = kKeygenThreads / 32;
  const int64_t stride = (int64_t)gridDim.x * wpb * 32;
  for (int64_t base = ((int64_t)blockIdx.x * wpb + (threadIdx.x >> 5)) * 32; base < n; base += stride) {
    const int64_t j = base + lane;
    uint32_t t = 0;
    unsigned g = 0;
    if (j < n) {
      if (P.id_bits) {  // the sorted value carries the entry count above the id
        const uint32_t pv = sorted_vals[j];
        t = pv >> P.id_bits;
        g = pv & ((1u << P.id_bits) - 1u);
      } else {
        t = touched[j];
        if (t) g = sorted_vals[j];
      }
    }
    RowSpan rs{};
    unsigned h = 0, y0 = 0, sb = 0, sx = 0;
    if (t) {
      const KeyShape k = ks[g];  // one 32-byte sector
      const ushort4 r = k.box;
      rs = make_row_span(k.ext, k.mean.x, k.mean.y, P.margin_abs, r);
      const ViewDesc& vd = vt.v[view_of_prim(vt, (int64_t)g)];
      h = (unsigned)(r.w - r.y);
      y0 = r.y;
      sb = (unsigned)vd.seg_base;
      sx = (unsigned)vd.segs_x;
    }
    unsigned R;
    const unsigned hex = warp_excl_scan(h, R);
    unsigned long long eb = 0;
    if (lane == 0) eb = offsets[base];
    eb = __shfl_sync(0xffffffffu, eb, 0);
    for (unsigned cb = 0; cb < R; cb += 32) {
      const unsigned s = cb + lane;
      const int ow = warp_last_le(hex, s);
      RowSpan q;
      q.u = __shfl_sync(0xffffffffu, rs.u, ow);
      q.v = __shfl_sync(0xffffffffu, rs.v, ow);
      q.ql = __shfl_sync(0xffffffffu, rs.ql, ow);
      q.mabs = P.margin_abs;  // the same for every primitive
      q.Y = __shfl_sync(0xffffffffu, rs.Y, ow);
      q.sl = __shfl_sync(0xffffffffu, rs.sl, ow);
      q.g = __shfl_sync(0xffffffffu, rs.g, ow);
      q.ic = __shfl_sync(0xffffffffu, rs.ic, ow);
      q.dys = __shfl_sync(0xffffffffu, rs.dys, ow);
      q.r0 = __shfl_sync(0xffffffffu, rs.r0, ow);
      q.r1 = __shfl_sync(0xffffffffu, rs.r1, ow);
      const unsigned qy0 = __shfl_sync(0xffffffffu, y0, ow);
      const unsigned qhex = __shfl_sync(0xffffffffu, hex, ow);
      const unsigned qg = __shfl_sync(0xffffffffu, g, ow);
      // one view: its segment base and row width are the same for every lane
      const unsigned qsb = VS::kMax == 1 ? (unsigned)vt.v[0].seg_base : __shfl_sync(0xffffffffu, sb, ow);
      const unsigned qsx = VS::kMax == 1 ? (unsigned)vt.v[0].segs_x : __shfl_sync(0xffffffffu, sx, ow);
      unsigned w = 0, kb = 0, tt = 0;
      if (s < R) {
        const int ty = (int)(qy0 + (s - qhex));
        int t0, t1;
        if (tile_row_span(q, ty, t0, t1)) {
          w = (unsigned)((t1 >> L) - (t0 >> L) + 1);
          kb = qsb + (unsigned)ty * qsx + (unsigned)(t0 >> L);  // the span's first segment
          tt = (unsigned)t0 | ((unsigned)t1 << 16);
        }
      }
      unsigned W;
      const unsigned wex = warp_excl_scan(w, W);
      // the lane writes its span's w entries itself (w is at most the segments of a tile row)
      const unsigned t0 = tt & 0xffffu, t1 = tt >> 16;
      unsigned long long e = eb + wex;
      for (unsigned i = 0; i < w; ++i, ++e) {
        if (e >= K) break;
        const unsigned lo = ((t0 >> L) + i) << L;          // first tile of the span's i-th segment
        const unsigned off0 = (t0 > lo ? t0 : lo) - lo;
        const unsigned hi = lo + (1u << L) - 1u;
        const unsigned off1 = (t1 < hi ? t1 : hi) - lo;
        tile_keys[e] = seg_key(kb + i, off0, off1, P);
        tile_vals[e] = qg;
      }
      eb += W;
    }
  }
}

// ---------------------------------------------------------------- K5 ranges
// Four entries per thread (one 16-byte load); a segment starts where an entry's segment id (the
// key's low bits, seg_mask) differs from its predecessor's and ends where it differs from its
// successor's.  Neighbours across threads come from the adjacent lanes; the warp's end lanes load
// theirs.
__global__ void k_ranges(const uint32_t* __restrict__ tile_keys, const unsigned long long* __restrict__ K_dev, int64_t cap,
                         uint32_t seg_mask, uint2* __restrict__ ranges) {
  const int64_t K = (int64_t)*K_dev;
  if (K > cap) return;
  const unsigned lane = lane_id();
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  constexpr uint32_t kNone = 0xffffffffu;  // never a segment id
  const int64_t nq = (K + 3) / 4;
  for (int64_t base = wid * 32; base < nq; base += nwarps * 32) {
    const int64_t e = 4 * (base + lane);
    uint32_t t[4];
    if (e + 3 < K) {
      const uint4 v = *reinterpret_cast<const uint4*>(tile_keys + e);
      t[0] = v.x & seg_mask; t[1] = v.y & seg_mask; t[2] = v.z & seg_mask; t[3] = v.w & seg_mask;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) t[i] = e + i < K ? (tile_keys[e + i] & seg_mask) : kNone;
    }
    uint32_t prev = __shfl_up_sync(0xffffffffu, t[3], 1);
    uint32_t next = __shfl_down_sync(0xffffffffu, t[0], 1);
    if (lane == 0) prev = e > 0 && e - 1 < K ? (tile_keys[e - 1] & seg_mask) : kNone;
    if (lane == 31) next = e + 4 < K ? (tile_keys[e + 4] & seg_mask) : kNone;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (e + i >= K) break;
      const uint32_t p = i == 0 ? prev : t[i - 1];
      const uint32_t q = i == 3 ? next : t[i + 1];
      if (p != t[i]) ranges[t[i]].x = (uint32_t)(e + i);
      if (q != t[i]) ranges[t[i]].y = (uint32_t)(e + i + 1);
    }
  }
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// streaming multiprocessors of the current device (cached per device)
int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 152;
  if (!cache[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 152;
  }
  return cache[dev];
}

// grid for a grid-stride loop over `items` units: at most `per_sm` CTAs per SM
unsigned grid_cap(int64_t items, int per_sm) {
  const int64_t cap = (int64_t)sm_count() * per_sm;
  return (unsigned)(items < cap ? (items > 0 ? items : 1) : cap);
}

}  // namespace

// ---------------------------------------------------------------- host drivers
size_t ScanScratch::required(int64_t max_n) {
  size_t total = kReserved;
  int64_t n = max_n;
  while (n > kChunk) {
    n = cdiv(n, kChunk);
    total += (size_t)(n + 1) * sizeof(unsigned long long);
  }
  return total + 256;
}

// n is the capacity; with n_dev the element count is min(*n_dev, n) and CTAs past it do nothing
template <typename TIn, typename TOut>
static void scan_level(const TIn* in, TOut* out, int64_t n, const unsigned long long* n_dev, TOut* total, char* scratch,
                       cudaStream_t s) {
  const int64_t nb = cdiv(n, kChunk);
  if (nb <= 1) {
    k_scan_down<TIn, TOut><<<1, kThreads, 0, s>>>(in, out, n, n_dev, nullptr, total);
    count_launches(1);
    return;
  }
  TOut* sums = reinterpret_cast<TOut*>(scratch);
  char* next = scratch + (size_t)(nb + 1) * sizeof(unsigned long long);
  k_scan_reduce<TIn, TOut><<<(unsigned)nb, kThreads, 0, s>>>(in, n, n_dev, sums);
  scan_level<TOut, TOut>(sums, sums, nb, nullptr, total, next, s);
  k_scan_down<TIn, TOut><<<(unsigned)nb, kThreads, 0, s>>>(in, out, n, n_dev, sums, nullptr);
  count_launches(2);
}

template <typename TIn, typename TOut>
void scan_exclusive(const TIn* in, TOut* out, int64_t n, TOut* total, ScanScratch& sc, cudaStream_t s,
                    const unsigned long long* n_dev) {
  if (n <= 0) {
    if (total) cudaMemsetAsync(total, 0, sizeof(TOut), s);
    return;
  }
  scan_level<TIn, TOut>(in, out, n, n_dev, total, reinterpret_cast<char*>(sc.buf) + ScanScratch::kReserved, s);
}

// ---------------------------------------------------------------- single-pass scan
// Exclusive scan of uint32 counts into 64-bit offsets in one launch, by the decoupled look-back of
// the one-sweep sort: a CTA takes the next chunk from a counter (so a chunk's predecessors are
// always running or done), publishes its chunk sum as an aggregate at once and its inclusive
// prefix when its own is known; warp 0 looks back over 32 predecessors at a time.  Status words
// are 64-bit: flag in bits 62-63 (1 aggregate, 2 inclusive prefix), value in bits 0-61.  The wait
// is bounded: a CTA that gives up takes 0 for what it did not see, publishes its prefix, and sets
// kFlagSortWait in *flags (the offsets are then wrong, the run ends).
constexpr unsigned long long kScAgg = 1ull << 62, kScPre = 2ull << 62, kScValue = (1ull << 62) - 1ull;

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ void st_volatile_u64(unsigned long long* p, unsigned long long v) {
  *reinterpret_cast<volatile unsigned long long*>(p) = v;
}

// status: [0] the chunk counter (low 32 bits), [1 + c] chunk c's word; all zero at launch.  in may
// equal out: a CTA writes its chunk only after reading it.  With idx (GATHER), element j is
// in[idx[j]] and is also written to gathered[j]; otherwise it is in[j] >> shift.  Three CTAs per SM hold every chunk of the
// depth-ordered entry counts of 1.5M primitives (367) at once.
template <typename TOut, bool GATHER>
__global__ void __launch_bounds__(kThreads, 3) k_scan_onepass(const uint32_t* in, const uint32_t* __restrict__ idx,
                                                              uint32_t* __restrict__ gathered, int shift, TOut* out,
                                                              int64_t cap,
                                                              const unsigned long long* __restrict__ n_dev,
                                                              unsigned long long* __restrict__ status,
                                                              TOut* __restrict__ total, uint32_t* __restrict__ flags) {
  const int64_t n = scan_count(cap, n_dev);
  const int64_t nchunks = (n + kChunk - 1) / kChunk;
  __shared__ unsigned long long ws[kThreads / 32 + 1];
  __shared__ unsigned long long s_prefix;
  __shared__ int64_t s_chunk;
  if (threadIdx.x == 0) s_chunk = (int64_t)atomicAdd(reinterpret_cast<unsigned int*>(status), 1u);
  __syncthreads();
  const int64_t c = s_chunk;
  if (c >= nchunks) {
    if (c == 0 && total && threadIdx.x == 0) *total = TOut(0);  // nothing to scan
    return;
  }
  // coalesced loads (element i of the chunk by thread i mod 256), transposed through shared memory
  // (one padding word per 16) so that each thread then holds 16 consecutive elements
  __shared__ TOut sbuf[kChunk + kChunk / 16];
  const int64_t cb = c * kChunk;
  const int cnt = (int)min((int64_t)kChunk, n - cb);
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int i = k * kThreads + (int)threadIdx.x;
    uint32_t x = 0u;
    if (i < cnt) {
      if (GATHER) {
        x = in[idx[cb + i]];
        gathered[cb + i] = x;
      } else {
        x = in[cb + i] >> shift;
      }
    }
    sbuf[i + (i >> 4)] = (TOut)x;
  }
  __syncthreads();
  uint32_t v[kItems];
  unsigned long long acc = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int i = (int)threadIdx.x * kItems + k;
    v[k] = (uint32_t)sbuf[i + (i >> 4)];
    acc += v[k];
  }
  const unsigned long long inc = warp_inclusive_scan(acc);
  const int w = threadIdx.x >> 5;
  const unsigned lane = threadIdx.x & 31u;
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  if (w == 0) {
    const unsigned long long x = (lane < kThreads / 32) ? ws[lane] : 0ull;
    const unsigned long long xi = warp_inclusive_scan(x);
    if (lane < kThreads / 32) ws[lane] = xi - x;
    const unsigned long long agg = __shfl_sync(0xffffffffu, xi, 31);  // the chunk's sum
    unsigned long long* my = status + 1 + c;
    unsigned long long prefix = 0;
    if (c == 0) {
      if (lane == 0) st_volatile_u64(my, kScPre | (agg & kScValue));
    } else {
      if (lane == 0) st_volatile_u64(my, kScAgg | (agg & kScValue));
      int64_t end = c;  // the window is chunks [end - 32, end), lane l reading end - 1 - l
      int spins = 0;
      bool fail = false;
      for (;;) {
        const int64_t idx = end - 1 - (int64_t)lane;
        const unsigned long long sw = idx >= 0 ? ld_volatile_u64(status + 1 + idx) : kScPre;
        const unsigned long long flag = sw & ~kScValue;
        const unsigned pre = __ballot_sync(0xffffffffu, flag == kScPre);
        const unsigned unset = __ballot_sync(0xffffffffu, flag == 0ull);
        const int first = pre ? __ffs(pre) - 1 : 32;  // nearest predecessor with a prefix
        const unsigned need = first >= 31 ? 0xffffffffu : ((2u << first) - 1u);
        if (unset & need) {
          if (++spins > kOsSpinLimit) {
            fail = true;
            break;
          }
          __nanosleep(32);
          continue;
        }
        unsigned long long part = ((int)lane <= first) ? (sw & kScValue) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        prefix += part;
        if (first < 32) break;
        end -= 32;
      }
      if (lane == 0) {
        st_volatile_u64(my, kScPre | ((prefix + agg) & kScValue));
        if (fail && flags) atomicOr(flags, kFlagSortWait);
      }
    }
    if (lane == 0) {
      s_prefix = prefix;
      if (c == nchunks - 1 && total) *total = (TOut)(prefix + agg);
    }
  }
  __syncthreads();  // every thread's reads of sbuf happened before the block scan's barrier
  unsigned long long run = inc - acc + ws[w] + s_prefix;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int i = (int)threadIdx.x * kItems + k;
    sbuf[i + (i >> 4)] = (TOut)run;
    run += v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int i = k * kThreads + (int)threadIdx.x;
    if (i < cnt) out[cb + i] = sbuf[i + (i >> 4)];
  }
}

template <typename TOut, bool GATHER>
static void scan_onepass_launch(const uint32_t* in, const uint32_t* idx, uint32_t* gathered, int shift, TOut* out,
                                int64_t n, TOut* total, ScanScratch& sc, uint32_t* flags, cudaStream_t s,
                                const unsigned long long* n_dev) {
  if (n <= 0) {
    if (total) cudaMemsetAsync(total, 0, sizeof(TOut), s);
    return;
  }
  const int64_t nchunks = cdiv(n, kChunk);
  unsigned long long* status =
      reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(sc.buf) + ScanScratch::kReserved);
  cudaMemsetAsync(status, 0, (size_t)(nchunks + 1) * sizeof(unsigned long long), s);
  k_scan_onepass<TOut, GATHER><<<(unsigned)nchunks, kThreads, 0, s>>>(in, idx, gathered, shift, out, n, n_dev, status,
                                                                     total, flags);
  count_launches(1);
}

void scan_exclusive_onepass(const uint32_t* in, unsigned long long* out, int64_t n, unsigned long long* total,
                            ScanScratch& sc, uint32_t* flags, cudaStream_t s, const unsigned long long* n_dev) {
  scan_onepass_launch<unsigned long long, false>(in, nullptr, nullptr, 0, out, n, total, sc, flags, s, n_dev);
}

void scan_exclusive_onepass(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total, ScanScratch& sc,
                            uint32_t* flags, cudaStream_t s, const unsigned long long* n_dev) {
  scan_onepass_launch<uint32_t, false>(in, nullptr, nullptr, 0, out, n, total, sc, flags, s, n_dev);
}

void scan_gather_onepass(const uint32_t* counts, const uint32_t* ids, uint32_t* gathered, unsigned long long* out,
                         int64_t n, unsigned long long* total, ScanScratch& sc, uint32_t* flags, cudaStream_t s,
                         const unsigned long long* n_dev) {
  scan_onepass_launch<unsigned long long, true>(counts, ids, gathered, 0, out, n, total, sc, flags, s, n_dev);
}

void scan_unpack_onepass(const uint32_t* packed, int shift, unsigned long long* out, int64_t n,
                         unsigned long long* total, ScanScratch& sc, uint32_t* flags, cudaStream_t s,
                         const unsigned long long* n_dev) {
  scan_onepass_launch<unsigned long long, false>(packed, nullptr, nullptr, shift, out, n, total, sc, flags, s, n_dev);
}

template void scan_exclusive<uint32_t, uint32_t>(const uint32_t*, uint32_t*, int64_t, uint32_t*, ScanScratch&, cudaStream_t,
                                                 const unsigned long long*);
template void scan_exclusive<uint32_t, unsigned long long>(const uint32_t*, unsigned long long*, int64_t,
                                                           unsigned long long*, ScanScratch&, cudaStream_t,
                                                           const unsigned long long*);

// scratch entries (uint32) of a sort of n_cap keys: the one-sweep layout (counters, digit counts,
// two status regions of 256 per chunk), which also holds the per-pass histogram of the classic
// form (at most 8-bit digits: 256 per chunk)
int64_t radix_hist_entries(int64_t n_cap, int max_bits) {
  (void)max_bits;
  return kOsHeader + 2 * 256 * cdiv(n_cap > 0 ? n_cap : 1, kChunk);
}

bool radix_sort_pairs(uint32_t* keys[2], uint32_t* vals[2], int& cur, int64_t n_host, const unsigned long long* n_dev,
                      int64_t n_cap, int total_bits, uint32_t* hist, int64_t hist_cap, ScanScratch& sc, cudaStream_t s,
                      uint32_t* flags, uint2* bin_ranges, int64_t n_ranges, bool* ranges_done) {
  if (ranges_done) *ranges_done = false;
  if (n_cap <= 0 || total_bits <= 0) return true;
  const int passes = (total_bits + 7) / 8;
  const int bits_per = (total_bits + passes - 1) / passes;
  const int64_t nchunks = cdiv(n_cap, kChunk);
  const int64_t os_chunks = cdiv(n_cap, kOsChunk);
  // one sweep for sorts of three or four passes (the depth sort); shorter sorts over many chunks (the
  // list sort) measured faster in the classic form, whose passes have no look-back chain
  if (passes >= 3 && n_cap < (int64_t)kOsValue && hist_cap >= kOsHeader + 2 * 256 * nchunks) {
    // zero the counters, the digit counts and the first status region
    cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)(kOsHeader + 256 * os_chunks), s);
    // two count CTAs per SM: each flushes its four 256-bin histograms with global atomics
    k_os_counts<<<grid_cap(cdiv(n_cap, kThreads * 4), 2), kThreads, 0, s>>>(keys[cur], n_host, n_dev, n_cap, passes,
                                                                           bits_per, total_bits, hist + 8);
    // CTAs take chunks from a counter, so the grid size does not affect the result: two per SM
    // (the register limit of 512 threads at 64 registers); no device query, as serving captures this
    const unsigned grid = grid_cap(os_chunks, 2);
    for (int p = 0; p < passes; ++p) {
      const int shift = p * bits_per;
      const int bits = (total_bits - shift) < bits_per ? (total_bits - shift) : bits_per;
      k_os_scatter<<<grid, kScThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n_host, n_dev,
                                               n_cap, shift, bits, p, p + 1 < passes ? 1 : 0, hist, os_chunks, flags);
      cur ^= 1;
    }
    count_launches(1 + passes);
    return true;
  }
  // keys of 9 bits (the list sort's segment ids at the usual sizes) in one pass of 512 bins
  const bool wide = total_bits == 9;
  const int passes_c = wide ? 1 : passes;
  const int bits_c = wide ? 9 : bits_per;
  if (((int64_t)1 << bits_c) * nchunks > hist_cap) return false;  // the histogram would not fit
  // the scatter's shared memory exceeds the 48 KB default: opt in once per device
  static std::atomic<bool> attr_set[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr_set[dev].load(std::memory_order_acquire)) {
    cudaFuncSetAttribute(k_radix_scatter<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ScatterSmem<256>));
    cudaFuncSetAttribute(k_radix_scatter<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ScatterSmem<512>));
    if (dev >= 0 && dev < 64) attr_set[dev].store(true, std::memory_order_release);
  }
  for (int p = 0; p < passes_c; ++p) {
    const int shift = p * bits_c;
    const int bits = (total_bits - shift) < bits_c ? (total_bits - shift) : bits_c;
    const int64_t entries = ((int64_t)1 << bits) * nchunks;  // capacity of the matrix
    unsigned long long* n_entries = reinterpret_cast<unsigned long long*>(sc.buf);
    if (wide) {
      k_radix_hist<512><<<grid_cap(nchunks, 8), kThreads, 0, s>>>(keys[cur], n_host, n_dev, n_cap, shift, bits, hist,
                                                                  n_entries);
    } else {
      k_radix_hist<256><<<grid_cap(nchunks, 8), kThreads, 0, s>>>(keys[cur], n_host, n_dev, n_cap, shift, bits, hist,
                                                                  n_entries);
    }
    scan_exclusive_onepass(hist, hist, entries, (uint32_t*)nullptr, sc, flags, s, n_entries);
    // a single pass over all the key bits also gives every bin's range (written by the scatter)
    const bool with_ranges = bin_ranges && passes_c == 1 && bits == total_bits && n_ranges > 0;
    uint2* rg_out = with_ranges ? bin_ranges : nullptr;
    if (with_ranges && ranges_done) *ranges_done = true;
    if (wide) {
      k_radix_scatter<512><<<grid_cap(nchunks, 2), kScThreads, sizeof(ScatterSmem<512>), s>>>(
          keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n_host, n_dev, n_cap, shift, bits, hist, rg_out,
          n_ranges);
    } else {
      k_radix_scatter<256><<<grid_cap(nchunks, 4), kScThreads, sizeof(ScatterSmem<256>), s>>>(
          keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n_host, n_dev, n_cap, shift, bits, hist, rg_out,
          n_ranges);
    }
    count_launches(2);
    cur ^= 1;
  }
  return true;
}

template <class VS>
void launch_keygen(const VS& vs, const unsigned long long* offsets, const uint32_t* touched,
                   const unsigned long long* K_dev, int64_t n, const uint32_t* sorted_vals, const KeyShape* ks,
                   const Params& P, int64_t cap, uint32_t* tile_keys, uint32_t* tile_vals, uint32_t* flags,
                   cudaStream_t s, const unsigned long long* n_dev) {
  if (n <= 0 || cap <= 0) return;
  k_keygen<VS><<<grid_cap(cdiv(n, kKeygenThreads), 8), kKeygenThreads, 0, s>>>(
      vs, offsets, K_dev, n, n_dev, sorted_vals, touched, ks, P, cap, tile_keys, tile_vals, flags);
  count_launches(1);
}

void launch_ranges(const uint32_t* tile_keys, const unsigned long long* K_dev, int64_t cap, uint32_t seg_mask,
                   uint2* ranges, int num_sms, cudaStream_t s) {
  if (cap <= 0) return;
  int64_t blocks = cdiv(cdiv(cap, 4), 256);
  if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
  k_ranges<<<(unsigned)blocks, 256, 0, s>>>(tile_keys, K_dev, cap, seg_mask, ranges);
  count_launches(1);
}

template void launch_keygen<FrameViews>(const FrameViews&, const unsigned long long*, const uint32_t*,
                                        const unsigned long long*, int64_t, const uint32_t*, const KeyShape*,
                                        const Params&, int64_t, uint32_t*, uint32_t*, uint32_t*, cudaStream_t,
                                        const unsigned long long*);
template void launch_keygen<BatchViews>(const BatchViews&, const unsigned long long*, const uint32_t*,
                                        const unsigned long long*, int64_t, const uint32_t*, const KeyShape*,
                                        const Params&, int64_t, uint32_t*, uint32_t*, uint32_t*, cudaStream_t,
                                        const unsigned long long*);

}  // namespace ges
