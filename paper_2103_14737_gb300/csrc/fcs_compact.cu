// fcs_compact.cu - gathers the hit cells of each event as (cell id, E) pairs
// for the transfer of results (the paper's sim_ct kernel, Sec. 4) and resets
// the accumulation rows to zero in the same pass (the paper's separate
// clean kernel, Sec. 4, is folded in).  The rows are FP64 (fcs_internal.cuh:
// acc_add); each hit cell is rounded once to the float of the output.
// Output order: event-major, ascending
// cell id; offsets come from an exclusive scan of per-chunk counts, so the
// result is deterministic.  Rows that stay in L2 take two passes (count, scan,
// write); rows that do not take one pass, each chunk's offset from a
// decoupled look-back over the chunks before it, so that the rows are read
// from DRAM once.
#include "fcs_internal.cuh"
#include "fcs_lookback.cuh"

namespace fcs {
namespace {

constexpr int kCThreads = 256;
constexpr int kCItems = 16;  // eight 16-byte loads of FP64 cells per thread (rows are padded to 64 cells)
constexpr int kCVec = kCItems / 2;
constexpr int kChunk = kCThreads * kCItems;
// rows above this size (more than the L2 holds beside the other traffic) take
// the one-pass compaction
constexpr int64_t kOnePassRowBytes = 128ll << 20;
constexpr int kOnePassCtasPerSm = 4;  // resident: 54 registers x 256 threads each

// A row value is a hit cell when it is not +-0 (an integer test, off the FP64 pipe).
__device__ __forceinline__ bool acc_nonzero(double d) {
  return ((unsigned long long)__double_as_longlong(d) << 1) != 0ull;
}

// Both kernels take the chunks (kChunk cells of one row) t = row * cpr + chunk
// grid-stride, so a capped grid leaves SMs to concurrent work.
__global__ void __launch_bounds__(kCThreads) k_compact_count(const double* __restrict__ acc, int32_t n_cells,
                                                           int32_t stride, int32_t cpr, int64_t n_chunks,
                                                           int64_t* __restrict__ counts) {
  __shared__ int s[kCThreads / 32];
  for (int64_t t = blockIdx.x; t < n_chunks; t += gridDim.x) {
    const int chunk = (int)(t % cpr), row = (int)(t / cpr);
    const int64_t c0 = (int64_t)chunk * kChunk + threadIdx.x * kCItems;
    const double2* src = reinterpret_cast<const double2*>(acc + (int64_t)row * stride + c0);
    int cnt = 0;
    if (c0 < n_cells) {
      double2 a[kCVec];
#pragma unroll
      for (int q = 0; q < kCVec; ++q) a[q] = src[q];
#pragma unroll
      for (int q = 0; q < kCVec; ++q) {
        cnt += (c0 + 2 * q < n_cells) && acc_nonzero(a[q].x);
        cnt += (c0 + 2 * q + 1 < n_cells) && acc_nonzero(a[q].y);
      }
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      int sum = 0;
      for (int i = 0; i < kCThreads / 32; ++i) sum += s[i];
      counts[t] = sum;
    }
    __syncthreads();  // s is reused
  }
}

__global__ void __launch_bounds__(kCThreads) k_compact_write(
    double* __restrict__ acc, int32_t n_cells, int32_t stride, int32_t cpr, int64_t n_chunks, int32_t ev_lo,
    const int64_t* __restrict__ offsets, float* __restrict__ cells_out, int32_t* __restrict__ cell_ids,
    float* __restrict__ cell_E, int64_t* __restrict__ event_offsets_out, int64_t capacity) {
  __shared__ int s_w[kCThreads / 32];
  __shared__ int32_t s_id[kChunk];
  __shared__ float s_E[kChunk];
  __shared__ int s_total;
  for (int64_t t = blockIdx.x; t < n_chunks; t += gridDim.x) {
    const int chunk = (int)(t % cpr), row = (int)(t / cpr);
    const int64_t c0 = (int64_t)chunk * kChunk + threadIdx.x * kCItems;
    double2* src = reinterpret_cast<double2*>(acc + (int64_t)row * stride + c0);
    float v[kCItems];
    unsigned mask = 0;
#pragma unroll
    for (int k = 0; k < kCItems; ++k) v[k] = 0.0f;
    if (c0 < n_cells) {
      double2 a[kCVec];
#pragma unroll
      for (int q = 0; q < kCVec; ++q) a[q] = src[q];
      const double2 z = make_double2(0.0, 0.0);
#pragma unroll
      for (int q = 0; q < kCVec; ++q) {
        if (c0 + 2 * q < n_cells && acc_nonzero(a[q].x)) {
          mask |= 1u << (2 * q);
          v[2 * q] = acc_to_f32(a[q].x);
        }
        if (c0 + 2 * q + 1 < n_cells && acc_nonzero(a[q].y)) {
          mask |= 1u << (2 * q + 1);
          v[2 * q + 1] = acc_to_f32(a[q].y);
        }
        // re-zero only what is not zero (the padding past n_cells stays zero):
        // many row cells are never hit, and a store of zeros would still dirty
        // the line
        if (acc_nonzero(a[q].x) || acc_nonzero(a[q].y)) src[q] = z;
      }
    }
    const int cnt = __popc(mask);
    // block exclusive scan of cnt
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    int pre = 0;
    for (int w = 0; w < warp; ++w) pre += s_w[w];
    // the block's pairs go through shared memory so that the output is written
    // with consecutive threads on consecutive positions
    int lpos = pre + x - cnt;
#pragma unroll
    for (int k = 0; k < kCItems; ++k) {
      if (mask & (1u << k)) {
        s_id[lpos] = (int32_t)(c0 + k);
        s_E[lpos] = v[k];
        ++lpos;
      }
    }
    if (threadIdx.x == kCThreads - 1) s_total = lpos;  // the last thread ends the block's run
    __syncthreads();
    const int total = s_total;
    const int64_t base = offsets[t];
    for (int j = threadIdx.x; j < total; j += kCThreads) {
      const int64_t pos = base + j;
      if (pos < capacity) {
        if (cell_ids) cell_ids[pos] = s_id[j];
        if (cell_E) cell_E[pos] = s_E[j];
      }
    }
    if (cells_out && c0 < n_cells) {
      float* dst = cells_out + (int64_t)(ev_lo + row) * n_cells + c0;
      if (c0 + kCItems <= n_cells && (n_cells & 3) == 0) {
#pragma unroll
        for (int q = 0; q < kCItems / 4; ++q)
          reinterpret_cast<float4*>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else {
#pragma unroll
        for (int k = 0; k < kCItems; ++k)
          if (c0 + k < n_cells) dst[k] = v[k];
      }
    }
    if (chunk == 0 && threadIdx.x == 0 && event_offsets_out) event_offsets_out[ev_lo + row] = base;
    __syncthreads();  // the staging arrays are reused
  }
}


// One pass: CTAs take chunks in ticket order; a chunk counts its hit cells,
// publishes the count, looks back for the count of the chunks before it (the
// first chunk starts at *total_dst, the call's running output size) and
// writes its pairs; the last chunk leaves the new total in *total_dst.  The
// last CTA to finish resets the ticket and the status words.
__global__ void __launch_bounds__(kCThreads) k_compact_one(
    double* __restrict__ acc, int32_t n_cells, int32_t stride, int32_t cpr, int64_t n_chunks, int32_t ev_lo,
    uint64_t* __restrict__ state, int64_t cap_tiles, uint32_t* flags, int64_t* total_dst, float* __restrict__ cells_out,
    int32_t* __restrict__ cell_ids, float* __restrict__ cell_E, int64_t* __restrict__ event_offsets_out,
    int64_t capacity) {
  __shared__ int s_w[kCThreads / 32];
  __shared__ int32_t s_id[kChunk];
  __shared__ float s_E[kChunk];
  __shared__ int s_total;
  __shared__ int64_t s_base;
  __shared__ unsigned long long s_ticket;
  __shared__ int s_last;
  unsigned long long* ticket = reinterpret_cast<unsigned long long*>(state);
  unsigned long long* done = ticket + 1;
  uint64_t* status = state + 2;
  int64_t n_t = n_chunks;
  if (n_t > cap_tiles) {  // the workspace sizes the state for its chunks: never
    if (threadIdx.x == 0) atomicOr(flags, (uint32_t)FCS_FLAG_WAIT_TIMEOUT);
    n_t = 0;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  while (true) {
    if (threadIdx.x == 0) s_ticket = atomicAdd(ticket, 1ull);
    __syncthreads();
    const int64_t t = (int64_t)s_ticket;
    if (t >= n_t) break;
    const int chunk = (int)(t % cpr), row = (int)(t / cpr);
    const int64_t c0 = (int64_t)chunk * kChunk + threadIdx.x * kCItems;
    double2* src = reinterpret_cast<double2*>(acc + (int64_t)row * stride + c0);
    float v[kCItems];
    unsigned mask = 0;
#pragma unroll
    for (int k = 0; k < kCItems; ++k) v[k] = 0.0f;
    if (c0 < n_cells) {
      double2 a[kCVec];
#pragma unroll
      for (int q = 0; q < kCVec; ++q) a[q] = src[q];
      const double2 z = make_double2(0.0, 0.0);
#pragma unroll
      for (int q = 0; q < kCVec; ++q) {
        if (c0 + 2 * q < n_cells && acc_nonzero(a[q].x)) {
          mask |= 1u << (2 * q);
          v[2 * q] = acc_to_f32(a[q].x);
        }
        if (c0 + 2 * q + 1 < n_cells && acc_nonzero(a[q].y)) {
          mask |= 1u << (2 * q + 1);
          v[2 * q + 1] = acc_to_f32(a[q].y);
        }
        if (acc_nonzero(a[q].x) || acc_nonzero(a[q].y)) src[q] = z;  // re-zero what is not zero
      }
    }
    const int cnt = __popc(mask);
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    int pre = 0, total = 0;
    for (int w = 0; w < kCThreads / 32; ++w) {
      if (w < warp) pre += s_w[w];
      total += s_w[w];
    }
    if (warp == 0) {  // publish, look back, publish the prefix
      int64_t excl;
      if (t == 0) {
        excl = *total_dst;
      } else {
        if (lane == 0) atomicExch(reinterpret_cast<unsigned long long*>(status + t), kFlagAgg | (uint64_t)total);
        excl = look_back(status, t, flags);
      }
      if (lane == 0) {
        atomicExch(reinterpret_cast<unsigned long long*>(status + t), kFlagPrefix | (uint64_t)(excl + total));
        s_base = excl;
        if (t == n_t - 1) *total_dst = excl + total;
      }
    }
    int lpos = pre + x - cnt;
#pragma unroll
    for (int k = 0; k < kCItems; ++k) {
      if (mask & (1u << k)) {
        s_id[lpos] = (int32_t)(c0 + k);
        s_E[lpos] = v[k];
        ++lpos;
      }
    }
    __syncthreads();
    const int64_t base = s_base;
    for (int j = threadIdx.x; j < total; j += kCThreads) {
      const int64_t pos = base + j;
      if (pos < capacity) {
        if (cell_ids) cell_ids[pos] = s_id[j];
        if (cell_E) cell_E[pos] = s_E[j];
      }
    }
    if (cells_out && c0 < n_cells) {
      float* dst = cells_out + (int64_t)(ev_lo + row) * n_cells + c0;
      if (c0 + kCItems <= n_cells && (n_cells & 3) == 0) {
#pragma unroll
        for (int q = 0; q < kCItems / 4; ++q)
          reinterpret_cast<float4*>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else {
#pragma unroll
        for (int k = 0; k < kCItems; ++k)
          if (c0 + k < n_cells) dst[k] = v[k];
      }
    }
    if (chunk == 0 && threadIdx.x == 0 && event_offsets_out) event_offsets_out[ev_lo + row] = base;
    __syncthreads();  // the staging arrays, s_base and s_ticket are reused
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
    for (int64_t i = threadIdx.x; i < n_t; i += kCThreads) status[i] = 0;
    if (threadIdx.x == 0) {
      *ticket = 0;
      *done = 0;
    }
  }
}

}  // namespace

cudaError_t launch_compact(const GeoDev& g, WsDev w, int32_t rows, int32_t ev_lo, int64_t* chunk_counts,
                           int64_t* chunk_offsets, ScanTmp tmp, float* cells_out, int32_t* cell_ids,
                           float* cell_E, int64_t* event_offsets_out, int64_t capacity, int max_ctas,
                           const Launch& L) {
  if (rows <= 0) return cudaSuccess;
  const int cpr = (g.n_cells + kChunk - 1) / kChunk;
  const int64_t n_chunks = (int64_t)rows * cpr;
  if (rows * (int64_t)g.acc_stride * (int64_t)sizeof(double) > kOnePassRowBytes) {
    // one pass, persistent CTAs (the ticket order makes every look-back wait end)
    const int grid = (int)std::min<int64_t>(n_chunks, max_ctas > 0 ? max_ctas : (int64_t)L.num_sms * kOnePassCtasPerSm);
    k_compact_one<<<grid, kCThreads, 0, L.s>>>(w.acc, g.n_cells, g.acc_stride, cpr, n_chunks, ev_lo, tmp.state,
                                               tmp.cap_tiles, tmp.flags, &w.sizes->nnz_total, cells_out, cell_ids,
                                               cell_E, event_offsets_out, capacity);
    return cudaGetLastError();
  }
  const int grid = (int)std::min<int64_t>(n_chunks, max_ctas > 0 ? max_ctas : ((int64_t)1 << 30));
  k_compact_count<<<grid, kCThreads, 0, L.s>>>(w.acc, g.n_cells, g.acc_stride, cpr, n_chunks, chunk_counts);
  // offsets continue the call's running output size (per-event mode)
  cudaError_t e = launch_scan_i64(chunk_counts, chunk_offsets, nullptr, n_chunks, &w.sizes->nnz_total, 1, tmp, L.s);
  if (e != cudaSuccess) return e;
  k_compact_write<<<grid, kCThreads, 0, L.s>>>(w.acc, g.n_cells, g.acc_stride, cpr, n_chunks, ev_lo, chunk_offsets,
                                               cells_out, cell_ids, cell_E, event_offsets_out, capacity);
  return cudaGetLastError();
}

int64_t compact_chunks(int32_t n_cells, int32_t rows) {
  return (int64_t)rows * ((n_cells + kChunk - 1) / kChunk);
}

}  // namespace fcs
