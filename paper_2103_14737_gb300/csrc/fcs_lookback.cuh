// fcs_lookback.cuh - the status words and the look-back of a single-pass
// device-wide scan with decoupled look-back (Merrill & Garland 2016), shared by
// the scans (fcs_scan.cu) and the one-pass compaction (fcs_compact.cu).  A tile
// publishes its aggregate, then its inclusive prefix, each as one 64-bit status
// word [flag:2 | value:62]; a tile waits only on tiles with smaller tickets,
// which CTAs that are already running hold, and each wait is bounded.
#pragma once
#include "fcs_internal.cuh"

namespace fcs {

inline constexpr uint64_t kFlagAgg = 1ull << 62;
inline constexpr uint64_t kFlagPrefix = 2ull << 62;
inline constexpr uint64_t kValueMask = (1ull << 62) - 1;
inline constexpr uint32_t kSpinLimit = 1u << 20;  // status polls before a wait gives up (about 0.2 s on GB300)

__device__ __forceinline__ int64_t warp_sum(int64_t x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Sum of the tiles before tile t, by warp 0: lane l reads the status of tile
// j - l, 32 tiles per step from the nearest predecessor back, until a tile
// with its inclusive prefix is found (position -1 counts as a prefix of 0).
__device__ __forceinline__ int64_t look_back(const uint64_t* status, int64_t t, uint32_t* flags) {
  const int lane = threadIdx.x & 31;
  int64_t excl = 0;
  for (int64_t j = t - 1;; j -= 32) {
    const int64_t idx = j - lane;
    uint64_t st = kFlagPrefix;
    if (idx >= 0) {
      const volatile uint64_t* p = status + idx;
      uint32_t spins = 0;
      st = *p;
      while ((st >> 62) == 0 && ++spins < kSpinLimit) st = *p;
      if ((st >> 62) == 0) {  // gave up: the result is invalid, the flag says so
        atomicOr(flags, (uint32_t)FCS_FLAG_WAIT_TIMEOUT);
        st = kFlagPrefix;
      }
    }
    const unsigned pm = __ballot_sync(0xffffffffu, (st >> 62) == 2);
    const int64_t v = (int64_t)(st & kValueMask);
    if (pm) {
      const int first = __ffs(pm) - 1;  // the nearest tile with a prefix
      return excl + warp_sum(lane <= first ? v : 0);
    }
    excl += warp_sum(v);
  }
}

}  // namespace fcs
