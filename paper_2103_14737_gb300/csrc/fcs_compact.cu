// fcs_compact.cu - gathers the hit cells of each event as (cell id, E) pairs
// for the transfer of results (the paper's sim_ct kernel, Sec. 4) and resets
// the accumulation rows to zero in the same pass (the paper's separate
// clean kernel, Sec. 4, is folded in).  The rows are FP64 (fcs_internal.cuh:
// acc_add); each hit cell is rounded once to the float of the output.
// Output order: event-major, ascending
// cell id; each chunk's output offset is the count of the chunks before it,
// taken in one pass by a decoupled look-back, so the result is deterministic
// and the rows are read once.
#include "fcs_internal.cuh"
#include "fcs_lookback.cuh"

namespace fcs {
namespace {

constexpr int kCThreads = 256;
constexpr int kCItems = 16;  // eight 16-byte loads of FP64 cells per thread (rows are padded to 64 cells)
constexpr int kCVec = kCItems / 2;
constexpr int kChunk = kCThreads * kCItems;
constexpr int kCtasPerSm = 4;  // resident: 54 registers x 256 threads each

// A row value is a hit cell when it is not +-0 (an integer test, off the FP64 pipe).
__device__ __forceinline__ bool acc_nonzero(double d) {
  return ((unsigned long long)__double_as_longlong(d) << 1) != 0ull;
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

cudaError_t launch_compact(const GeoDev& g, WsDev w, int32_t rows, int32_t ev_lo, ScanTmp tmp, float* cells_out,
                           int32_t* cell_ids, float* cell_E, int64_t* event_offsets_out, int64_t capacity, int max_ctas,
                           const Launch& L) {
  if (rows <= 0) return cudaSuccess;
  const int cpr = (g.n_cells + kChunk - 1) / kChunk;
  const int64_t n_chunks = (int64_t)rows * cpr;
  // persistent CTAs (the ticket order makes every look-back wait end); the
  // offsets continue the call's running output size (per-event mode)
  const int grid = (int)std::min<int64_t>(n_chunks, max_ctas > 0 ? max_ctas : (int64_t)L.num_sms * kCtasPerSm);
  k_compact_one<<<grid, kCThreads, 0, L.s>>>(w.acc, g.n_cells, g.acc_stride, cpr, n_chunks, ev_lo, tmp.state,
                                             tmp.cap_tiles, tmp.flags, &w.sizes->nnz_total, cells_out, cell_ids, cell_E,
                                             event_offsets_out, capacity);
  return cudaGetLastError();
}

int64_t compact_chunks(int32_t n_cells, int32_t rows) {
  return (int64_t)rows * ((n_cells + kChunk - 1) / kChunk);
}

}  // namespace fcs
