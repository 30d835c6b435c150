// fcs_sort.cu - deterministic mode: sort the (cell, task, count) records of
// the hit kernel by (cell, task) with an LSD radix sort, then fold each cell
// in ascending task order:
//   E_cell = fold_{tasks ascending} fl32( fl32(n_cell,task) * Ehit_task )
// starting from 0.0f.  Every hit of a task carries the same energy (Listing 1:
// one Ehit per layer loop), so the per-task integer count n and one FP32
// product per task give a result that does not depend on the order in which
// hits were processed: the run-to-run reproducible counterpart of the
// paper's atomicAdd accumulation (Sec. 4, Listing 2).
//
// Record layout (uint64): [ cell_global | task | count - 1 (5 bits) ], with
// cell_global = row * n_cells + cell.  Records of the same (cell, task) from
// different warps are merged by the fold (their counts add exactly).
//
// The hit kernel writes each record to the slot of a hit of its group, so
// the slot array (one per hit of the range, empty slots all ones) is in hit
// order, which is task order.  A stable LSD radix sort on the cell bits alone
// therefore yields (cell, task) order: 8-bit digits over bits
// [cell_shift, total_bits); the first pass drops the empty slots.  Each warp of the grid is a
// sorting unit owning a contiguous slice of the slots; per pass a per-unit
// digit histogram, a digit-major exclusive scan over (digit, unit), and a
// stable scatter in which each warp ranks 32 records at a time with
// __match_any_sync.  No inter-CTA waits.
#include "fcs_internal.cuh"

namespace fcs {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsBlocksPerSm = 4;
constexpr int kRsBatch = 4;  // 32-key groups a warp loads before ranking them (loads in flight)
constexpr uint64_t kEmpty = ~0ull;

__device__ __forceinline__ void unit_range(int64_t n, int64_t U, int64_t u, int64_t* b, int64_t* e) {
  int64_t chunk = (n + U - 1) / U;
  chunk = (chunk + 31) & ~(int64_t)31;
  *b = min(u * chunk, n);
  *e = min(*b + chunk, n);
}

// Keys a pass reads: the hit-slot array (empty slots skipped) in the first
// pass, the non-empty records after it.
__device__ __forceinline__ int64_t pass_count(const Sizes* sz, int64_t cap, bool slots) {
  return min(slots ? sz->n_hits : sz->n_records, cap);
}

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t* __restrict__ keys, const Sizes* sz,
                                                      int64_t cap, int shift, int64_t* __restrict__ hist,
                                                      int64_t U, int slots) {
  __shared__ uint32_t s_h[kRsWarps][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = lane; d < 256; d += 32) s_h[warp][d] = 0;
  __syncwarp();
  const int64_t n = pass_count(sz, cap, slots);
  const int64_t u = (int64_t)blockIdx.x * kRsWarps + warp;
  int64_t b, e;
  unit_range(n, U, u, &b, &e);
  for (int64_t i0 = b; i0 < e; i0 += 32 * kRsBatch) {
    uint64_t k[kRsBatch];
#pragma unroll
    for (int j = 0; j < kRsBatch; ++j) {
      const int64_t i = i0 + 32 * j + lane;
      k[j] = i < e ? keys[i] : kEmpty;
    }
#pragma unroll
    for (int j = 0; j < kRsBatch; ++j) {
      const bool act = k[j] != kEmpty;
      const unsigned m = __ballot_sync(0xffffffffu, act);
      if (act) {
        const uint32_t d = (uint32_t)(k[j] >> shift) & 255u;
        const unsigned peers = __match_any_sync(m, d);
        if (lane == __ffs(peers) - 1) s_h[warp][d] += __popc(peers);
      }
      __syncwarp();
    }
  }
  for (int d = lane; d < 256; d += 32) hist[(int64_t)d * U + u] = s_h[warp][d];
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t* __restrict__ in,
                                                         uint64_t* __restrict__ out, const Sizes* sz,
                                                         int64_t cap, int shift,
                                                         const int64_t* __restrict__ offs, int64_t U, int slots) {
  __shared__ int64_t s_off[kRsWarps][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t u = (int64_t)blockIdx.x * kRsWarps + warp;
  for (int d = lane; d < 256; d += 32) s_off[warp][d] = offs[(int64_t)d * U + u];
  __syncwarp();
  const int64_t n = pass_count(sz, cap, slots);
  int64_t b, e;
  unit_range(n, U, u, &b, &e);
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t i0 = b; i0 < e; i0 += 32 * kRsBatch) {
    uint64_t k[kRsBatch];
#pragma unroll
    for (int j = 0; j < kRsBatch; ++j) {
      const int64_t i = i0 + 32 * j + lane;
      k[j] = i < e ? in[i] : kEmpty;
    }
    // rank the groups in slice order: the scatter is stable
#pragma unroll
    for (int j = 0; j < kRsBatch; ++j) {
      const bool act = k[j] != kEmpty;
      const unsigned m = __ballot_sync(0xffffffffu, act);
      uint32_t d = 0;
      unsigned peers = 0;
      if (act) {
        d = (uint32_t)(k[j] >> shift) & 255u;
        peers = __match_any_sync(m, d);
        out[s_off[warp][d] + __popc(peers & lt)] = k[j];
      }
      __syncwarp();
      if (act && lane == __ffs(peers) - 1) s_off[warp][d] += __popc(peers);
      __syncwarp();
    }
  }
}

__global__ void k_det_heads(const uint64_t* __restrict__ keys, Sizes* sz, int64_t cap, int cell_shift,
                            int64_t* __restrict__ flags) {
  const int64_t n = min(sz->n_records, cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) sz->n_rec_used = n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = (i == 0 || (keys[i - 1] >> cell_shift) != (keys[i] >> cell_shift)) ? 1 : 0;
}

// Index of each cell's first record: idx[h] = i for the h-th head record i
// (head_off holds the call's running output positions; record 0 is a head).
__global__ void k_det_index(const Sizes* sz, int64_t cap, const int64_t* __restrict__ flags,
                            const int64_t* __restrict__ head_off, int64_t* __restrict__ idx) {
  const int64_t n = min(sz->n_records, cap);
  if (n == 0) return;
  const int64_t base = head_off[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (flags[i]) idx[head_off[i] - base] = i;
}

// One thread per non-zero cell: the records [idx[h], idx[h + 1]) in
// ascending task order; the counts of one task add exactly before its single
// FP32 product.
__global__ void k_det_fold(const uint64_t* __restrict__ keys, const Sizes* sz, int64_t cap, int cell_shift,
                           uint64_t task_mask, const int64_t* __restrict__ idx,
                           const int64_t* __restrict__ head_off, const float* __restrict__ task_ehit,
                           int32_t n_cells, int32_t ev_lo, float* __restrict__ cells_out,
                           int32_t* __restrict__ cell_ids, float* __restrict__ cell_E,
                           int64_t* __restrict__ event_offsets_out, int64_t capacity) {
  const int64_t n = min(sz->n_records, cap);
  if (n == 0) return;
  const int64_t base = head_off[0];
  const int64_t n_heads = sz->nnz_total - base;  // the scan has added this range's heads
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n_heads;
       h += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = idx[h], i1 = (h + 1 < n_heads) ? idx[h + 1] : n;
    const uint64_t cg = keys[i0] >> cell_shift;
    float E = 0.0f;
    int64_t prev_task = -1;
    int64_t cnt = 0;
    for (int64_t j = i0; j < i1; ++j) {
      const uint64_t k = keys[j];
      const int64_t task = (int64_t)((k >> kRecordCountBits) & task_mask);
      const int64_t c = (int64_t)(k & ((1u << kRecordCountBits) - 1u)) + 1;
      if (task != prev_task) {
        if (prev_task >= 0) E = __fadd_rn(E, __fmul_rn((float)cnt, task_ehit[prev_task]));
        prev_task = task;
        cnt = 0;
      }
      cnt += c;
    }
    E = __fadd_rn(E, __fmul_rn((float)cnt, task_ehit[prev_task]));
    const int64_t row = (int64_t)(cg / (uint64_t)n_cells);
    const int32_t cell = (int32_t)(cg % (uint64_t)n_cells);
    const int64_t o = base + h;
    if (o < capacity) {
      if (cell_ids) cell_ids[o] = cell;
      if (cell_E) cell_E[o] = E;
    }
    if (cells_out) cells_out[(ev_lo + row) * (int64_t)n_cells + cell] = E;
    if (event_offsets_out) {
      const int64_t prev_row = (h == 0) ? -1 : (int64_t)((keys[idx[h - 1]] >> cell_shift) / (uint64_t)n_cells);
      for (int64_t r = prev_row + 1; r <= row; ++r) event_offsets_out[ev_lo + r] = o;
    }
  }
}

// Rows after the last non-empty one start at the running total.
__global__ void k_det_tail(const uint64_t* __restrict__ keys, const Sizes* sz, int64_t cap, int cell_shift,
                           int32_t n_cells, int32_t rows, int32_t ev_lo, int64_t* __restrict__ event_offsets_out) {
  const int64_t n = min(sz->n_records, cap);
  const int64_t last = n > 0 ? (int64_t)((keys[n - 1] >> cell_shift) / (uint64_t)n_cells) : -1;
  for (int64_t r = last + 1 + threadIdx.x; r < rows; r += blockDim.x) event_offsets_out[ev_lo + r] = sz->nnz_total;
}

}  // namespace

int64_t det_hist_entries(int num_sms) { return (int64_t)256 * num_sms * kRsBlocksPerSm * kRsWarps; }

cudaError_t launch_det_reduce(const GeoDev& g, WsDev w, int32_t rows, int32_t ev_lo, int key_task_bits,
                              int key_total_bits, uint32_t* /*unused*/, int64_t hist_cap, int64_t* head_flags,
                              int64_t* head_offsets, ScanTmp tmp, float* cells_out, int32_t* cell_ids,
                              float* cell_E, int64_t* event_offsets_out, int32_t n_events_total,
                              int64_t capacity, const Launch& L) {
  (void)n_events_total;
  const int nb = L.num_sms * kRsBlocksPerSm;
  const int64_t U = (int64_t)nb * kRsWarps;
  if (256 * U > hist_cap) return cudaErrorInvalidValue;
  // the histogram buffer doubles as the digit-offset buffer (scanned in place)
  int64_t* hist = head_flags;  // reuse: sized >= max(records, 256 * U) by the workspace
  uint64_t* a = w.keys;
  uint64_t* b = w.keys_alt;
  const int cell_shift = kRecordCountBits + key_task_bits;
  for (int shift = cell_shift; shift < key_total_bits; shift += 8) {
    const int slots = shift == cell_shift;
    k_rs_hist<<<nb, kRsThreads, 0, L.s>>>(a, w.sizes, w.rec_cap, shift, hist, U, slots);
    cudaError_t e = launch_scan_i64(hist, hist, nullptr, 256 * U, nullptr, 0, tmp, L.s);
    if (e != cudaSuccess) return e;
    k_rs_scatter<<<nb, kRsThreads, 0, L.s>>>(a, b, w.sizes, w.rec_cap, shift, hist, U, slots);
    uint64_t* t = a;
    a = b;
    b = t;
  }
  const uint64_t task_mask = (key_task_bits >= 64) ? ~0ull : ((1ull << key_task_bits) - 1ull);
  k_det_heads<<<L.num_sms * 4, 256, 0, L.s>>>(a, w.sizes, w.rec_cap, cell_shift, head_flags);
  cudaError_t e = launch_scan_i64(head_flags, head_offsets, &w.sizes->n_rec_used, 0, &w.sizes->nnz_total, 1,
                                  tmp, L.s);
  if (e != cudaSuccess) return e;
  // the first record of each cell, in the sort's free ping-pong buffer
  int64_t* idx = reinterpret_cast<int64_t*>(b);
  k_det_index<<<L.num_sms * 4, 256, 0, L.s>>>(w.sizes, w.rec_cap, head_flags, head_offsets, idx);
  k_det_fold<<<L.num_sms * 4, 256, 0, L.s>>>(a, w.sizes, w.rec_cap, cell_shift, task_mask, idx,
                                             head_offsets, w.tmu, g.n_cells, ev_lo, cells_out, cell_ids,
                                             cell_E, event_offsets_out, capacity);
  if (event_offsets_out)
    k_det_tail<<<1, 256, 0, L.s>>>(a, w.sizes, w.rec_cap, cell_shift, g.n_cells, rows, ev_lo, event_offsets_out);
  return cudaGetLastError();
}

}  // namespace fcs
