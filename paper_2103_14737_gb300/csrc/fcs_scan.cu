// fcs_scan.cu - device-wide exclusive scan of counts in one pass (decoupled
// look-back, Merrill & Garland 2016).  Used for particle -> task / hit
// offsets, the compaction offsets and the deterministic mode's cell offsets.
// The element count may live in device memory, so the launch needs no host
// synchronisation.
//
// Persistent CTAs take tiles of 256 threads x 16 elements (32 for the hit
// offsets, whose tile map work makes fewer, larger tiles pay) in increasing order from
// an atomic ticket.  A tile publishes its aggregate, then (after looking back
// over its predecessors) its inclusive prefix, each as one 64-bit status word
// [flag:2 | value:62].  A tile waits only on tiles with smaller tickets, which
// CTAs that are already running hold, so the waits end; each wait is bounded
// all the same and sets FCS_FLAG_WAIT_TIMEOUT when it gives up.  Input and
// output move through shared memory (coalesced), each thread scanning
// its consecutive elements.  The last CTA to finish resets the ticket
// and the status words it used, so the state is zero again for the next scan.
//
// The scan of the tasks' hit counts also writes the tile map: granule g (hits
// [g kGranule, (g + 1) kGranule)) -> the task holding hit g kGranule, from
// each task's first hit and count while the tile is at hand (granules below
// the map's capacity; the hit kernel reports a map too small for the hits).
#include <atomic>

#include "fcs_internal.cuh"
#include "fcs_lookback.cuh"

namespace fcs {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;  // elements per thread: 16, or 32 for the hit offsets
constexpr int kScanTile = kScanThreads * kScanItems;  // the smallest tile (sizes the status words)
constexpr int kHitScanItems = 32;

// Dynamic shared memory of a scan with `items` elements per thread: its tile,
// element j at j + j / items.
constexpr size_t scan_smem_bytes(int items) { return (size_t)kScanThreads * (items + 1) * sizeof(int64_t); }

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

// Out: the offsets' type (int64, or int32 for the deterministic mode's cell
// offsets, which also zero their uint32 inputs as they read them: ZERO_IN).
template <typename In, bool GMAP, int ITEMS, typename Out = int64_t, bool ZERO_IN = false>
__global__ void __launch_bounds__(kScanThreads) k_scan(const In* in, Out* out, const int64_t* n_dev, int64_t n_host,
                                                     int64_t* total_dst, int base_from_dst, uint64_t* state,
                                                     int64_t cap_tiles, uint32_t* flags, int32_t* gmap,
                                                     int64_t gmap_cap, int64_t mute_tile) {
  constexpr int TILE = kScanThreads * ITEMS;
  extern __shared__ int64_t s_tile[];  // scan_smem_bytes(ITEMS): element j at j + j / ITEMS
  __shared__ int64_t s_warp[kScanThreads / 32];
  __shared__ int64_t s_excl;
  __shared__ unsigned long long s_ticket;
  __shared__ int s_last;
  unsigned long long* ticket = reinterpret_cast<unsigned long long*>(state);
  unsigned long long* done = ticket + 1;
  uint64_t* status = state + 2;
  const int64_t n = load_n(n_dev, n_host);
  int64_t n_tiles = (n + TILE - 1) / TILE;
  if (n_tiles > cap_tiles) {  // the workspace sizes the state for its arrays: never
    if (threadIdx.x == 0) atomicOr(flags, (uint32_t)FCS_FLAG_WAIT_TIMEOUT);
    n_tiles = 0;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  while (true) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(ticket, 1ull);
    __syncthreads();
    const int64_t t = (int64_t)s_ticket;
    if (t >= n_tiles) break;
    const int64_t t0 = t * TILE;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const int j = k * kScanThreads + threadIdx.x;
      const int64_t i = t0 + j;
      s_tile[j + j / ITEMS] = i < n ? (int64_t)in[i] : 0;
    }
    __syncthreads();
    int64_t sum = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) sum += s_tile[threadIdx.x * (ITEMS + 1) + k];
    int64_t tile_total;
    const int64_t thread_excl = block_excl_scan(sum, s_warp, &tile_total);  // synchronises the block
    if (warp == 0) {
      int64_t excl;
      if (t == 0) {
        excl = base_from_dst ? *total_dst : 0;
      } else {
        if (lane == 0 && t != mute_tile)
          atomicExch(reinterpret_cast<unsigned long long*>(status + t), kFlagAgg | (uint64_t)tile_total);
        excl = look_back(status, t, flags);
      }
      if (lane == 0 && t != mute_tile) {
        atomicExch(reinterpret_cast<unsigned long long*>(status + t), kFlagPrefix | (uint64_t)(excl + tile_total));
      }
      if (lane == 0) {
        s_excl = excl;
        if (t == n_tiles - 1 && total_dst) *total_dst = excl + tile_total;
      }
    }
    __syncthreads();
    int64_t run = s_excl + thread_excl;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {  // the thread's inputs, still in the tile buffer
      const int64_t x = s_tile[threadIdx.x * (ITEMS + 1) + k];
      s_tile[threadIdx.x * (ITEMS + 1) + k] = run;
      run += x;
    }
    __syncthreads();
    if constexpr (GMAP) {
#pragma unroll 1
      for (int k = 0; k < ITEMS; ++k) {
        const int j = k * kScanThreads + threadIdx.x;
        const int64_t i = t0 + j;
        if (i < n) {
          const int64_t b = s_tile[j + j / ITEMS];
          out[i] = b;
          // task i holds hits [b, e): e is the next task's first hit (the
          // tile's end for its last task)
          const int jn = j + 1;
          const int64_t e = (jn < TILE && i + 1 < n) ? s_tile[jn + jn / ITEMS] : s_excl + tile_total;
          for (int64_t g = (b + kGranule - 1) / kGranule; g * kGranule < e && g < gmap_cap; ++g) gmap[g] = (int32_t)i;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const int j = k * kScanThreads + threadIdx.x;
        const int64_t i = t0 + j;
        if (i < n) {
          out[i] = (Out)s_tile[j + j / ITEMS];
          if constexpr (ZERO_IN) const_cast<In*>(in)[i] = 0;  // read whole before the scan
        }
      }
    }
    __syncthreads();  // the tile buffer and s_ticket are reused
  }
  // every CTA has left its loop (and its look-backs) before it counts itself
  // done; the last one resets the state
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(done, 1ull) == (unsigned long long)gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (int64_t i = threadIdx.x; i < n_tiles; i += kScanThreads) status[i] = 0;
    if (threadIdx.x == 0) {
      if (n_tiles == 0 && total_dst && !base_from_dst) *total_dst = 0;
      *ticket = 0;
      *done = 0;
    }
  }
}

}  // namespace

int64_t scan_state_words(int64_t max_elements) {
  return 2 + (std::max<int64_t>(max_elements, 1) + kScanTile - 1) / kScanTile;
}

// out[i] = base + sum_{j<i} in[j]; base = *total_dst if base_from_dst != 0
// (a running total in device memory) else 0.  Writes base + sum to
// *total_dst when total_dst is non-NULL.  in and out may alias (a tile is
// read whole before it is written).
template <typename In, bool GMAP = false, int ITEMS = kScanItems, typename Out = int64_t, bool ZERO_IN = false>
static cudaError_t launch_scan(const In* in, Out* out, const int64_t* n_dev, int64_t n_host,
                               int64_t* total_dst, int64_t base_from_dst, ScanTmp tmp, cudaStream_t s,
                               int32_t* gmap = nullptr, int64_t gmap_cap = 0) {
  constexpr size_t smem = scan_smem_bytes(ITEMS);
  if constexpr (smem > 48 * 1024) {  // above the default limit: opt in, once per device
    constexpr int kMaxDevices = 64;
    static std::atomic<bool> opted[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = -1;
    if (dev < 0 || !opted[dev].load(std::memory_order_acquire)) {
      const cudaError_t e = cudaFuncSetAttribute(k_scan<In, GMAP, ITEMS, Out, ZERO_IN>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      if (dev >= 0) opted[dev].store(true, std::memory_order_release);
    }
  }
  // the status words are sized for kScanTile-element tiles; larger tiles need fewer
  k_scan<In, GMAP, ITEMS, Out, ZERO_IN><<<tmp.grid, kScanThreads, smem, s>>>(in, out, n_dev, n_host, total_dst,
                                                                            base_from_dst ? 1 : 0, tmp.state,
                                                                            tmp.cap_tiles, tmp.flags, gmap, gmap_cap,
                                                                            -1);
  return cudaGetLastError();
}

cudaError_t launch_scan_i64(const int64_t* in, int64_t* out, const int64_t* n_dev, int64_t n_host,
                            int64_t* total_dst, int64_t base_from_dst, ScanTmp tmp, cudaStream_t s) {
  return launch_scan(in, out, n_dev, n_host, total_dst, base_from_dst, tmp, s);
}

cudaError_t launch_scan_u32_zero(uint32_t* in, int32_t* out, int64_t n, ScanTmp tmp, cudaStream_t s) {
  return launch_scan<uint32_t, false, kScanItems, int32_t, true>(in, out, nullptr, n, nullptr, 0, tmp, s);
}

// Self-test of the bounded wait: a scan of three tiles on four CTAs, in its
// own zeroed buffers, in which tile 1 never publishes its status, so that the
// look-back of tile 2 gives up after kSpinLimit polls and sets
// FCS_FLAG_WAIT_TIMEOUT.  Writes the device flag word and the kernel's time.
cudaError_t scan_wait_selftest(uint32_t* flags_out, float* ms, cudaStream_t s) {
  constexpr int64_t n_tiles = 3, n = n_tiles * kScanTile;
  const size_t bytes = (size_t)(2 * n + 2 + n_tiles + 1) * 8;
  unsigned char* buf = nullptr;
  cudaError_t e = cudaMalloc((void**)&buf, bytes);
  if (e != cudaSuccess) return e;
  int64_t* in = reinterpret_cast<int64_t*>(buf);
  int64_t* out = in + n;
  uint64_t* state = reinterpret_cast<uint64_t*>(out + n);
  uint32_t* flags = reinterpret_cast<uint32_t*>(state + 2 + n_tiles);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess &&
      (e = cudaMemsetAsync(buf, 0, bytes, s)) == cudaSuccess && (e = cudaEventRecord(e0, s)) == cudaSuccess) {
    k_scan<int64_t, false, kScanItems><<<4, kScanThreads, scan_smem_bytes(kScanItems), s>>>(
        in, out, nullptr, n, nullptr, 0, state, n_tiles, flags, nullptr, 0, 1);
    if ((e = cudaGetLastError()) == cudaSuccess && (e = cudaEventRecord(e1, s)) == cudaSuccess &&
        (e = cudaMemcpyAsync(flags_out, flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) == cudaSuccess &&
        (e = cudaStreamSynchronize(s)) == cudaSuccess)
      e = cudaEventElapsedTime(ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  return e;
}

cudaError_t launch_scan_hits(const int32_t* tn, int64_t* th, const int64_t* n_tasks, int64_t* n_hits, int32_t* gmap,
                             int64_t gmap_cap, ScanTmp tmp, cudaStream_t s) {
  return launch_scan<int32_t, true, kHitScanItems>(tn, th, n_tasks, 0, n_hits, 0, tmp, s, gmap, gmap_cap);
}

}  // namespace fcs
