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
// Radix sort: 8-bit digits over bits [5, total_bits).  Each warp of the grid
// is a sorting unit owning a contiguous slice of the records; per pass a
// per-unit digit histogram, a digit-major exclusive scan over (digit, unit),
// and a stable scatter in which each warp ranks 32 records at a time with
// __match_any_sync.  No inter-CTA waits.
#include "fcs_internal.cuh"

namespace fcs {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsBlocksPerSm = 2;

__device__ __forceinline__ void unit_range(int64_t n, int64_t U, int64_t u, int64_t* b, int64_t* e) {
  int64_t chunk = (n + U - 1) / U;
  chunk = (chunk + 31) & ~(int64_t)31;
  *b = min(u * chunk, n);
  *e = min(*b + chunk, n);
}

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t* __restrict__ keys, const Sizes* sz,
                                                      int64_t cap, int shift, int64_t* __restrict__ hist,
                                                      int64_t U) {
  __shared__ uint32_t s_h[kRsWarps][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = lane; d < 256; d += 32) s_h[warp][d] = 0;
  __syncwarp();
  const int64_t n = min(sz->n_records, cap);
  const int64_t u = (int64_t)blockIdx.x * kRsWarps + warp;
  int64_t b, e;
  unit_range(n, U, u, &b, &e);
  for (int64_t i0 = b; i0 < e; i0 += 32) {
    const int64_t i = i0 + lane;
    const bool act = i < e;
    const unsigned m = __ballot_sync(0xffffffffu, act);
    if (act) {
      const uint32_t d = (uint32_t)(keys[i] >> shift) & 255u;
      const unsigned peers = __match_any_sync(m, d);
      if (lane == __ffs(peers) - 1) s_h[warp][d] += __popc(peers);
    }
    __syncwarp();
  }
  for (int d = lane; d < 256; d += 32) hist[(int64_t)d * U + u] = s_h[warp][d];
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t* __restrict__ in,
                                                         uint64_t* __restrict__ out, const Sizes* sz,
                                                         int64_t cap, int shift,
                                                         const int64_t* __restrict__ offs, int64_t U) {
  __shared__ int64_t s_off[kRsWarps][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t u = (int64_t)blockIdx.x * kRsWarps + warp;
  for (int d = lane; d < 256; d += 32) s_off[warp][d] = offs[(int64_t)d * U + u];
  __syncwarp();
  const int64_t n = min(sz->n_records, cap);
  int64_t b, e;
  unit_range(n, U, u, &b, &e);
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t i0 = b; i0 < e; i0 += 32) {
    const int64_t i = i0 + lane;
    const bool act = i < e;
    const unsigned m = __ballot_sync(0xffffffffu, act);
    uint64_t key = 0;
    uint32_t d = 0;
    unsigned peers = 0;
    if (act) {
      key = in[i];
      d = (uint32_t)(key >> shift) & 255u;
      peers = __match_any_sync(m, d);
      out[s_off[warp][d] + __popc(peers & lt)] = key;
    }
    __syncwarp();
    if (act && lane == __ffs(peers) - 1) s_off[warp][d] += __popc(peers);
    __syncwarp();
  }
}

__global__ void k_det_heads(const uint64_t* __restrict__ keys, Sizes* sz, int64_t cap, int cell_shift,
                            int64_t* __restrict__ flags) {
  const int64_t n = min(sz->n_records, cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) sz->n_rec_used = n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = (i == 0 || (keys[i - 1] >> cell_shift) != (keys[i] >> cell_shift)) ? 1 : 0;
}

__global__ void k_det_fold(const uint64_t* __restrict__ keys, const Sizes* sz, int64_t cap, int cell_shift,
                           uint64_t task_mask, const int64_t* __restrict__ flags,
                           const int64_t* __restrict__ head_off, const TaskRec* __restrict__ tasks,
                           int32_t n_cells, int32_t ev_lo, float* __restrict__ cells_out,
                           int32_t* __restrict__ cell_ids, float* __restrict__ cell_E,
                           int64_t* __restrict__ event_offsets_out, int64_t capacity) {
  const int64_t n = min(sz->n_records, cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!flags[i]) continue;
    const uint64_t cg = keys[i] >> cell_shift;
    float E = 0.0f;
    int64_t prev_task = -1;
    int64_t cnt = 0;
    for (int64_t j = i; j < n && (keys[j] >> cell_shift) == cg; ++j) {
      const int64_t task = (int64_t)((keys[j] >> kRecordCountBits) & task_mask);
      const int64_t c = (int64_t)(keys[j] & ((1u << kRecordCountBits) - 1u)) + 1;
      if (task != prev_task) {
        if (prev_task >= 0) E = __fadd_rn(E, __fmul_rn((float)cnt, tasks[prev_task].Ehit));
        prev_task = task;
        cnt = 0;
      }
      cnt += c;
    }
    E = __fadd_rn(E, __fmul_rn((float)cnt, tasks[prev_task].Ehit));
    const int64_t row = (int64_t)(cg / (uint64_t)n_cells);
    const int32_t cell = (int32_t)(cg % (uint64_t)n_cells);
    const int64_t o = head_off[i];
    if (o < capacity) {
      if (cell_ids) cell_ids[o] = cell;
      if (cell_E) cell_E[o] = E;
    }
    if (cells_out) cells_out[(ev_lo + row) * (int64_t)n_cells + cell] = E;
    if (event_offsets_out) {
      const int64_t prev_row = (i == 0) ? -1 : (int64_t)((keys[i - 1] >> cell_shift) / (uint64_t)n_cells);
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
  for (int shift = kRecordCountBits; shift < key_total_bits; shift += 8) {
    k_rs_hist<<<nb, kRsThreads, 0, L.s>>>(a, w.sizes, w.rec_cap, shift, hist, U);
    cudaError_t e = launch_scan_i64(hist, hist, nullptr, 256 * U, nullptr, 0, tmp, L.s);
    if (e != cudaSuccess) return e;
    k_rs_scatter<<<nb, kRsThreads, 0, L.s>>>(a, b, w.sizes, w.rec_cap, shift, hist, U);
    uint64_t* t = a;
    a = b;
    b = t;
  }
  const int cell_shift = kRecordCountBits + key_task_bits;
  const uint64_t task_mask = (key_task_bits >= 64) ? ~0ull : ((1ull << key_task_bits) - 1ull);
  k_det_heads<<<L.num_sms * 4, 256, 0, L.s>>>(a, w.sizes, w.rec_cap, cell_shift, head_flags);
  cudaError_t e = launch_scan_i64(head_flags, head_offsets, &w.sizes->n_rec_used, 0, &w.sizes->nnz_total, 1,
                                  tmp, L.s);
  if (e != cudaSuccess) return e;
  k_det_fold<<<L.num_sms * 4, 256, 0, L.s>>>(a, w.sizes, w.rec_cap, cell_shift, task_mask, head_flags,
                                             head_offsets, w.tasks, g.n_cells, ev_lo, cells_out, cell_ids,
                                             cell_E, event_offsets_out, capacity);
  if (event_offsets_out)
    k_det_tail<<<1, 256, 0, L.s>>>(a, w.sizes, w.rec_cap, cell_shift, g.n_cells, rows, ev_lo, event_offsets_out);
  return cudaGetLastError();
}

}  // namespace fcs
