// fcs_params.cu - builds the inverse-CDF thresholds and guide tables of the
// shape histograms on the device (one thread per parametrisation entry).
//
// Thresholds: with C_k the FP64 left-to-right prefix sum of the first k
// weights and K the last bin of non-zero weight, T[k] = min(2^32 - 1,
// floor(2^32 C_{k+1} / C_128)) for k < K and 2^32 - 1 for k >= K.  The bin of
// a 32-bit random word x is the first k < K with x < T[k], else K.
//
// Guide table (Chen and Asau's indexed search): for guide cell j (the words
// with x >> 25 == j) lo_j is the bin of x = j << 25 and hi_j the bin of
// x = (j + 1) << 25 (K for the last cell); the bin of every x in the cell lies
// in [lo_j, hi_j] and equals lo_j plus the number of thresholds T[k],
// lo_j <= k < hi_j, with T[k] <= x (T does not decrease).  Within the cell
// such a threshold satisfies j 2^25 < T[k] <= (j + 1) 2^25, so it is stored
// exactly as the 25-bit offset t_k = T[k] - j 2^25 - 1, and x >= T[k] reads
// (x mod 2^25) > t_k.  A cell packs, in 64 bits, t_lo and t_lo+1 (the value
// 2^25 - 1, which no offset exceeds, where the cell spans fewer bins), lo_j
// and the span hi_j - lo_j:
//   x: t_lo | (t_lo+1 & 0x7F) << 25;  y: t_lo+1 >> 7 | lo_j << 18 | span << 25.
// So the bin of a word is decided by one 8-byte load and two comparisons
// unless the cell spans three or more bins and x lies past T[lo_j + 1]; then
// a binary search over T[lo_j + 2 .. hi_j] finishes it.
#include "fcs_internal.cuh"

namespace fcs {
namespace {

constexpr uint32_t kGuideNever = 0x1FFFFFFu;  // an offset no word of the cell exceeds

__device__ __forceinline__ uint2 guide_cell(uint32_t t0, uint32_t t1, int lo, int span) {
  return make_uint2(t0 | (t1 << 25), (t1 >> 7) | ((uint32_t)lo << 18) | ((uint32_t)span << 25));
}

__global__ void k_build_tables(const float* __restrict__ shape_w, int n_entries,
                               uint32_t* __restrict__ thr, uint2* __restrict__ guide,
                               int32_t* __restrict__ bad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_entries) return;
  const float* w = shape_w + (int64_t)e * kNBins;
  uint32_t* T = thr + (int64_t)e * kNBins;
  uint2* G = guide + (int64_t)e * kGuideCells;
  double C = 0.0;
  int K = -1;
  for (int k = 0; k < kNBins; ++k) {
    const float wk = w[k];
    C = __dadd_rn(C, (double)wk);
    if (wk > 0.0f) K = k;
  }
  if (!(C > 0.0) || K < 0) {
    for (int k = 0; k < kNBins; ++k) T[k] = 0xFFFFFFFFu;
    for (int j = 0; j < kGuideCells; ++j) G[j] = guide_cell(kGuideNever, kGuideNever, 0, 0);
    bad[e] = 1;
    return;
  }
  bad[e] = 0;
  double c = 0.0;
  for (int k = 0; k < kNBins; ++k) {
    c = __dadd_rn(c, (double)w[k]);
    if (k < K) {
      double t = floor(__ddiv_rn(__dmul_rn(4294967296.0, c), C));
      if (t > 4294967295.0) t = 4294967295.0;
      T[k] = (uint32_t)t;
    } else {
      T[k] = 0xFFFFFFFFu;
    }
  }
  // lo_j = first k < K with (j << 25) < T[k], else K (monotone sweep)
  int k = 0;
  int lo_prev = 0;
  for (int j = 0; j <= kGuideCells; ++j) {
    int lo;
    if (j < kGuideCells) {
      const uint32_t x = (uint32_t)j << 25;
      while (k < K && x >= T[k]) ++k;
      lo = k;
    } else {
      lo = K;
    }
    if (j > 0) {
      const uint32_t base = (uint32_t)(j - 1) << 25;
      const int span = lo - lo_prev;
      const uint32_t t0 = span >= 1 ? T[lo_prev] - base - 1u : kGuideNever;
      const uint32_t t1 = span >= 2 ? T[lo_prev + 1] - base - 1u : kGuideNever;
      G[j - 1] = guide_cell(t0, t1, lo_prev, span);
    }
    lo_prev = lo;
  }
}

}  // namespace

cudaError_t launch_build_tables(const float* shape_w, int n_entries, uint32_t* thr, uint2* guide,
                                int32_t* bad, cudaStream_t s) {
  if (n_entries <= 0) return cudaSuccess;
  const int threads = 128;
  k_build_tables<<<(n_entries + threads - 1) / threads, threads, 0, s>>>(shape_w, n_entries, thr,
                                                                         guide, bad);
  return cudaGetLastError();
}

}  // namespace fcs
