// soma_scan.cu -- prefix sums and the stable radix sort of the chain reorder.
//
// Scan (reduce, then scan): one CTA per tile of kScanTile values sums its
// tile; one CTA scans the tile sums; every tile then scans its own values
// from its offset.  Integers only, so the order of additions does not
// matter.  Used for the placement's running weight sums (64-bit) and the
// sort's digit offsets (32-bit).
//
// Sort (least significant digit first, 8-bit digits): per pass every tile of
// kSortTile items counts its digits; one exclusive scan over the counts laid
// out digit-major ([digit][tile]) gives every (digit, tile) its first output
// position, so that equal digits keep the order of their tiles; inside a
// tile each warp owns kSortTile / 8 consecutive items, counts its digits per
// warp, turns the counts into positions (warps in order) and scatters its
// items 32 at a time in order, ranking equal digits among the lanes with
// __match_any_sync.  Every pass is therefore stable, and so is the sort.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "soma_launch.h"

namespace soma {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kTopThreads = 1024;

template <class T>
__device__ __forceinline__ T warp_inclusive(T v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// Exclusive scan of one value per thread over the CTA (blockDim.x a multiple
// of 32, at most 1024); *total receives the CTA's sum.
template <class T>
__device__ __forceinline__ T block_exclusive(T v, T* warp_sums, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  const T inc = warp_inclusive(v, lane);
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const T w = lane < n_warps ? warp_sums[lane] : T(0);
    const T wi = warp_inclusive(w, lane);
    if (lane < n_warps) warp_sums[lane] = wi - w;
    if (lane == n_warps - 1) *total = wi;
  }
  __syncthreads();
  const T out = warp_sums[warp] + inc - v;
  __syncthreads();  // warp_sums may be reused by the caller
  return out;
}

template <class T>
__global__ void k_scan_reduce(const T* __restrict__ in, int64_t n, T* __restrict__ tile_sums) {
  __shared__ T warp_sums[kScanThreads / 32];
  __shared__ T total;
  const int64_t t0 = (int64_t)blockIdx.x * kScanTile;
  T s = 0;
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t i = t0 + (int64_t)threadIdx.x * kScanItems + j;
    if (i < n) s += in[i];
  }
  block_exclusive<T>(s, warp_sums, &total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// One CTA: exclusive scan of the tile sums in place.
template <class T>
__global__ void k_scan_top(T* __restrict__ sums, int64_t n) {
  __shared__ T warp_sums[kTopThreads / 32];
  __shared__ T total;
  const int64_t per = (n + kTopThreads - 1) / kTopThreads;
  const int64_t lo = min((int64_t)threadIdx.x * per, n), hi = min(lo + per, n);
  T s = 0;
  for (int64_t i = lo; i < hi; ++i) s += sums[i];
  T run = block_exclusive<T>(s, warp_sums, &total);
  for (int64_t i = lo; i < hi; ++i) {
    const T v = sums[i];
    sums[i] = run;
    run += v;
  }
}

// out may be in: each value is read and written by the same thread.
template <class T>
__global__ void k_scan_down(const T* in, T* out, int64_t n, const T* __restrict__ tile_offsets, int inclusive) {
  __shared__ T warp_sums[kScanThreads / 32];
  __shared__ T total;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = base + j < n ? in[base + j] : T(0);
    s += v[j];
  }
  T run = tile_offsets[blockIdx.x] + block_exclusive<T>(s, warp_sums, &total);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < n) out[base + j] = inclusive ? run + v[j] : run;
    run += v[j];
  }
}

static int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

template <class T>
static size_t scan_temp_bytes_t(int64_t n) {
  return sizeof(T) * (size_t)std::max<int64_t>(1, scan_tiles(n));
}

template <class T>
static cudaError_t launch_scan_t(const T* in, T* out, int64_t n, bool inclusive, void* temp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t tiles = scan_tiles(n);
  T* sums = static_cast<T*>(temp);
  k_scan_reduce<T><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
  k_scan_top<T><<<1, kTopThreads, 0, s>>>(sums, tiles);
  k_scan_down<T><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums, inclusive ? 1 : 0);
  return cudaGetLastError();
}

size_t scan_temp_bytes_u64(int64_t n) { return scan_temp_bytes_t<unsigned long long>(n); }

cudaError_t launch_scan_u64(const unsigned long long* in, unsigned long long* out, int64_t n, bool inclusive,
                            void* temp, cudaStream_t s) {
  return launch_scan_t<unsigned long long>(in, out, n, inclusive, temp, s);
}

// ---------------------------------------------------------------------------
// Radix sort of (64-bit key, 32-bit value) pairs.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortTile = 1024;  // small tiles: many CTAs even for 10^5 chains
constexpr int kWarpItems = kSortTile / kSortWarps;  // 128 consecutive items per warp
constexpr int kDigits = 256;

static int64_t sort_tiles(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

// digit of a key: bits [shift, shift + 8) masked to the bits below end_bit
__device__ __forceinline__ int radix_digit(unsigned long long key, int shift, unsigned mask) {
  return (int)((key >> shift) & mask);
}

__global__ void k_radix_count(const unsigned long long* __restrict__ keys, int64_t n, int shift, unsigned mask,
                              uint32_t* __restrict__ counts, int64_t n_tiles) {
  __shared__ uint32_t hist[kDigits];
  for (int d = threadIdx.x; d < kDigits; d += blockDim.x) hist[d] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * kSortTile, t1 = min(n, t0 + kSortTile);
  for (int64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x) atomicAdd(&hist[radix_digit(keys[i], shift, mask)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kDigits; d += blockDim.x) counts[(int64_t)d * n_tiles + blockIdx.x] = hist[d];
}

__global__ void k_radix_scatter(const unsigned long long* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                                unsigned long long* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int64_t n,
                                int shift, unsigned mask, const uint32_t* __restrict__ offsets, int64_t n_tiles) {
  __shared__ uint32_t wpos[kSortWarps][kDigits];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  for (int d = lane; d < kDigits; d += 32) wpos[warp][d] = 0;
  __syncwarp();
  const int64_t w0 = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * kWarpItems;
  // this warp's digit counts (items in order, 32 at a time)
  for (int r = 0; r < kWarpItems / 32; ++r) {
    const int64_t i = w0 + r * 32 + lane;
    const int d = i < n ? radix_digit(keys_in[i], shift, mask) : kDigits;  // kDigits: no item
    const unsigned m = __match_any_sync(0xffffffffu, d);
    if (d < kDigits && (m & lt) == 0) wpos[warp][d] += __popc(m);
    __syncwarp();
  }
  __syncthreads();
  // counts -> first output position of each (warp, digit), warps in order
  for (int d = threadIdx.x; d < kDigits; d += blockDim.x) {
    uint32_t run = offsets[(int64_t)d * n_tiles + blockIdx.x];
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = wpos[w][d];
      wpos[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  // scatter in order: equal digits ranked by lane within each group of 32
  for (int r = 0; r < kWarpItems / 32; ++r) {
    const int64_t i = w0 + r * 32 + lane;
    const bool ok = i < n;
    const unsigned long long key = ok ? keys_in[i] : 0ull;
    const int d = ok ? radix_digit(key, shift, mask) : kDigits;
    const unsigned m = __match_any_sync(0xffffffffu, d);
    if (ok) {
      const uint32_t pos = wpos[warp][d] + (uint32_t)__popc(m & lt);
      keys_out[pos] = key;
      vals_out[pos] = vals_in[i];
    }
    __syncwarp();
    if (ok && (m & lt) == 0) wpos[warp][d] += __popc(m);
    __syncwarp();
  }
}

size_t radix_sort_temp_bytes(int64_t n) {
  const int64_t words = (int64_t)kDigits * std::max<int64_t>(1, sort_tiles(n));
  const size_t counts = ((sizeof(uint32_t) * (size_t)words + 255) / 256) * 256;
  return counts + scan_temp_bytes_t<uint32_t>(words);
}

cudaError_t launch_radix_sort_pairs(unsigned long long* keys_a, unsigned long long* keys_b, uint32_t* vals_a,
                                    uint32_t* vals_b, int64_t n, int end_bit, void* temp, bool* in_b,
                                    cudaStream_t s) {
  *in_b = false;
  if (n <= 1) return cudaSuccess;
  const int64_t tiles = sort_tiles(n);
  const int64_t words = (int64_t)kDigits * tiles;
  uint32_t* counts = static_cast<uint32_t*>(temp);
  void* scan_temp = static_cast<char*>(temp) + ((sizeof(uint32_t) * (size_t)words + 255) / 256) * 256;
  unsigned long long *ki = keys_a, *ko = keys_b;
  uint32_t *vi = vals_a, *vo = vals_b;
  for (int shift = 0; shift < end_bit; shift += 8) {
    const int bits = std::min(8, end_bit - shift);
    const unsigned mask = (1u << bits) - 1u;
    k_radix_count<<<(unsigned)tiles, kSortThreads, 0, s>>>(ki, n, shift, mask, counts, tiles);
    cudaError_t e = launch_scan_t<uint32_t>(counts, counts, words, false, scan_temp, s);
    if (e != cudaSuccess) return e;
    k_radix_scatter<<<(unsigned)tiles, kSortThreads, 0, s>>>(ki, vi, ko, vo, n, shift, mask, counts, tiles);
    std::swap(ki, ko);
    std::swap(vi, vo);
    *in_b = !*in_b;
  }
  return cudaGetLastError();
}

}  // namespace soma
