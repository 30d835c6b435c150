// fcs_scan.cu - device-wide exclusive scan of int64 counts (reduce, scan of
// block sums, downsweep).  Used for particle -> task / hit offsets, the
// compaction offsets and the deterministic mode's cell offsets.  The element count may
// live in device memory, so the launches need no host synchronisation.
#include "fcs_internal.cuh"

namespace fcs {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t load_n(const int64_t* n_dev, int64_t n_host) {
  return n_dev ? *n_dev : n_host;
}

// Exclusive block scan of one int64 per thread; returns the block total in *total.
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* s_warp, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = (lane < (kScanThreads >> 5)) ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < (kScanThreads >> 5)) s_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const int64_t warp_excl = warp ? s_warp[warp - 1] : 0;
  *total = s_warp[(kScanThreads >> 5) - 1];
  __syncthreads();
  return warp_excl + x - v;
}

template <typename In>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const In* __restrict__ in,
                                                            const int64_t* n_dev, int64_t n_host,
                                                            int64_t* __restrict__ block_sums) {
  const int64_t n = load_n(n_dev, n_host);
  const int64_t chunk = (n + kScanBlocks - 1) / kScanBlocks;
  const int64_t b = (int64_t)blockIdx.x * chunk, e = min(b + chunk, n);
  int64_t acc = 0;
  for (int64_t i = b + threadIdx.x; i < e; i += kScanThreads) acc += (int64_t)in[i];
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ int64_t s[kScanThreads / 32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int i = 0; i < kScanThreads / 32; ++i) t += s[i];
    block_sums[blockIdx.x] = t;
  }
}

// One block of kScanBlocks threads: exclusive scan of the block sums plus the
// optional base; writes the grand total.
__global__ void __launch_bounds__(kScanBlocks) k_scan_blocks(int64_t* block_sums, const int64_t* base_dev,
                                                             int64_t* total_dst) {
  __shared__ int64_t s_warp[kScanBlocks / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t v = block_sums[threadIdx.x];
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = (lane < kScanBlocks / 32) ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanBlocks / 32) s_warp[lane] = w;
  }
  __syncthreads();
  const int64_t base = base_dev ? *base_dev : 0;
  const int64_t excl = (warp ? s_warp[warp - 1] : 0) + x - v;
  const int64_t total = s_warp[kScanBlocks / 32 - 1];
  __syncthreads();  // every thread has read *base_dev before it may be overwritten
  block_sums[threadIdx.x] = base + excl;
  if (threadIdx.x == 0) {
    block_sums[kScanBlocks] = base + total;
    if (total_dst) *total_dst = base + total;
  }
}

// Tiles of kScanTile elements move through shared memory: coalesced loads
// and stores of the tile, while each thread scans kScanItems consecutive
// elements of it.  Element j sits at j + j / kScanItems (one pad word per
// thread's run keeps the per-thread accesses off a single bank).
template <typename In>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const In* __restrict__ in,
                                                          int64_t* __restrict__ out,
                                                          const int64_t* n_dev, int64_t n_host,
                                                          const int64_t* __restrict__ block_sums) {
  __shared__ int64_t s_warp[kScanThreads / 32];
  __shared__ int64_t s_tile[kScanTile + kScanTile / kScanItems];
  const int64_t n = load_n(n_dev, n_host);
  const int64_t chunk = (n + kScanBlocks - 1) / kScanBlocks;
  const int64_t b = (int64_t)blockIdx.x * chunk, e = min(b + chunk, n);
  int64_t carry = block_sums[blockIdx.x];
  for (int64_t t0 = b; t0 < e; t0 += kScanTile) {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const int j = k * kScanThreads + threadIdx.x;
      const int64_t i = t0 + j;
      s_tile[j + j / kScanItems] = i < e ? (int64_t)in[i] : 0;
    }
    __syncthreads();
    int64_t v[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = s_tile[threadIdx.x * (kScanItems + 1) + k];
      sum += v[k];
    }
    int64_t tile_total;
    int64_t run = carry + block_excl_scan(sum, s_warp, &tile_total);  // synchronises the block
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      s_tile[threadIdx.x * (kScanItems + 1) + k] = run;
      run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const int j = k * kScanThreads + threadIdx.x;
      const int64_t i = t0 + j;
      if (i < e) out[i] = s_tile[j + j / kScanItems];
    }
    carry += tile_total;
    __syncthreads();  // the tile buffer is reused
  }
}

}  // namespace

// out[i] = base + sum_{j<i} in[j]; base = *total_dst if base_from_dst != 0
// (a running total in device memory) else 0.  Writes base + sum to
// *total_dst when total_dst is non-NULL.  in and out may alias.
template <typename In>
static cudaError_t launch_scan(const In* in, int64_t* out, const int64_t* n_dev, int64_t n_host,
                               int64_t* total_dst, int64_t base_from_dst, ScanTmp tmp, cudaStream_t s) {
  k_scan_reduce<In><<<kScanBlocks, kScanThreads, 0, s>>>(in, n_dev, n_host, tmp.block_sums);
  k_scan_blocks<<<1, kScanBlocks, 0, s>>>(tmp.block_sums, base_from_dst ? total_dst : nullptr,
                                          total_dst);
  k_scan_down<In><<<kScanBlocks, kScanThreads, 0, s>>>(in, out, n_dev, n_host, tmp.block_sums);
  return cudaGetLastError();
}

cudaError_t launch_scan_i64(const int64_t* in, int64_t* out, const int64_t* n_dev, int64_t n_host,
                            int64_t* total_dst, int64_t base_from_dst, ScanTmp tmp, cudaStream_t s) {
  return launch_scan(in, out, n_dev, n_host, total_dst, base_from_dst, tmp, s);
}

cudaError_t launch_scan_u32(const uint32_t* in, int64_t* out, int64_t n, ScanTmp tmp, cudaStream_t s) {
  return launch_scan(in, out, nullptr, n, nullptr, 0, tmp, s);
}

}  // namespace fcs
