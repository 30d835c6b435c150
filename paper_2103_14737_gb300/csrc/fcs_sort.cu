// fcs_sort.cu - deterministic mode: group the (cell, task, count) records of
// the hit kernel by cell and fold each cell in ascending task order:
//   E_cell = fold_{tasks ascending} fl32( fl32(n_cell,task) * Ehit_task )
// starting from 0.0f.  Every hit of a task carries the same energy (Listing 1:
// one Ehit per layer loop), so the per-task integer count n and one FP32
// product per task give a result that does not depend on the order in which
// hits were processed: the run-to-run reproducible counterpart of the
// paper's atomicAdd accumulation (Sec. 4, Listing 2).
//
// Record layout (uint64): [ cell | task | count - 1 (5 bits) ], with cell the
// index into the accumulation rows (row * acc_stride + cell in row).  The hit
// kernel writes the records to slots handed out in chunks (unused slots hold
// the empty record, all ones) and counts the records of every cell in the
// accumulation rows, used as uint32 counters.  Then:
//   1. an exclusive scan of the counters gives each cell the start of its
//      segment of the record array (int32) and zeroes the counters;
//   2. scatter: every record takes a place in its cell's segment from the
//      cell's offset, counted up, which ends at the segment's end (the next
//      cell's start), so that one array bounds every segment.  In the
//      segment the cell is implied and a record shrinks to 32 bits:
//      [ task - first task of the cell's event (27 bits) | count - 1 ]
//      (a row holds one event, and its tasks are consecutive), so the
//      segments take half the bytes and sort as 32-bit keys;
//   3. fold: one thread per cell sorts its segment by (task, count) - a copy
//      in registers with a sorting network of 8, 16 or 32 records, each class
//      in a kernel of its own - merges the records of a task (their counts
//      add exactly) and folds; a warp per longer segment sorts it in shared
//      memory (bitonic) before its first lane folds.  The float result goes
//      to the (FP64) accumulation row, where the compaction of the atomic
//      mode picks it up, rounds it back to the same float and re-zeroes it.
// Only the order of places inside a segment depends on scheduling, and the
// sort removes it, so the cells are bit-reproducible.
#include <algorithm>
#include <atomic>

#include "fcs_internal.cuh"

namespace fcs {
namespace {

constexpr uint64_t kEmpty = ~0ull;
constexpr int kThreadSortMax = 32;  // segments sorted by one thread (in registers) up to here
constexpr int kRelTaskBits = 32 - kRecordCountBits;  // a segment record's task, relative to its event's first
constexpr uint32_t kCountMask = (1u << kRecordCountBits) - 1u;

// The first task of each event (row) of the range, from the per-particle task
// offsets: base[r] = poff[first particle of event ev_lo + r].
__global__ void k_det_bases(const int64_t* __restrict__ event_offsets, int32_t ev_lo, int32_t rows,
                            const int64_t* __restrict__ poff, const Sizes* sz, int64_t* __restrict__ base) {
  const int64_t n_part = sz->n_part, n_tasks = sz->n_tasks;
  const int64_t p0 = event_offsets[ev_lo];
  for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    const int64_t li = event_offsets[ev_lo + r] - p0;
    base[r] = (li >= 0 && li < n_part) ? poff[li] : n_tasks;  // events without particles take no records
  }
}

// A range that outgrew the workspace (FCS_FLAG_HIT_CAPACITY) has slots the
// hit kernel did not write: the scatter and the fold then do nothing (the
// call reports the overflow; the counter scan has zeroed the rows).
// A record whose task lies 2^27 or more past its event's first sets
// FCS_FLAG_KEY_BITS and is dropped (the call then fails).
__global__ void __launch_bounds__(256) k_det_scatter(const uint64_t* __restrict__ slots, Sizes* sz, int64_t cap,
                                                     int cell_shift, uint64_t task_mask, int32_t* __restrict__ cell_off,
                                                     int64_t n_cells_all, uint32_t acc_stride,
                                                     const int64_t* __restrict__ base, uint32_t* __restrict__ out) {
  if (sz->flags & FCS_FLAG_HIT_CAPACITY) return;
  constexpr int R = 4;  // records per thread and trip: their counts-up are in flight together
  const int64_t n = min(sz->n_slots, cap);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += R * stride) {
    uint64_t k[R];
#pragma unroll
    for (int j = 0; j < R; ++j) k[j] = (i0 + j * stride < n) ? slots[i0 + j * stride] : kEmpty;
    int32_t pos[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const uint64_t c = k[j] >> cell_shift;
      // (c is always in range for records of this range)
      pos[j] = (k[j] != kEmpty && c < (uint64_t)n_cells_all) ? atomicAdd(cell_off + c, 1) : -1;
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
      if (pos[j] < 0) continue;
      const uint32_t c = (uint32_t)(k[j] >> cell_shift);
      const int64_t rel = (int64_t)((k[j] >> kRecordCountBits) & task_mask) - base[c / acc_stride];
      if (rel < 0 || rel >= ((int64_t)1 << kRelTaskBits)) {
        atomicOr(&sz->flags, (uint32_t)FCS_FLAG_KEY_BITS);
        continue;
      }
      if (pos[j] < cap) out[pos[j]] = ((uint32_t)rel << kRecordCountBits) | ((uint32_t)k[j] & kCountMask);
    }
  }
}

__device__ __forceinline__ void sift_down(uint32_t* a, int64_t root, int64_t n) {
  while (true) {
    int64_t child = 2 * root + 1;
    if (child >= n) return;
    if (child + 1 < n && a[child + 1] > a[child]) ++child;
    if (a[root] >= a[child]) return;
    const uint32_t t = a[root];
    a[root] = a[child];
    a[child] = t;
    root = child;
  }
}

// Ascending sort of a[0, n) in place (heapsort).
__device__ __noinline__ void sort_segment(uint32_t* a, int64_t n) {
  for (int64_t r = n / 2 - 1; r >= 0; --r) sift_down(a, r, n);
  for (int64_t e = n - 1; e > 0; --e) {
    const uint32_t t = a[0];
    a[0] = a[e];
    a[e] = t;
    sift_down(a, 0, e);
  }
}

// One step of the fold of a cell's records in ascending order: per task the
// summed count times the task's hit energy, added in task order.  The count
// is 32-bit (a task's hits fit in 31 bits) and converted as such: conversions
// from 64-bit integers, like float-to-double ones, run on the narrow FP64 pipe.
struct Fold {
  float E = 0.0f;
  float e = 0.0f;  // hit energy of prev_task
  int64_t prev_task = -1;  // relative to the event's first task
  uint32_t cnt = 0;
  // segment record k, whose task's hit energy is ek (loaded ahead by the caller)
  __device__ __forceinline__ void add(uint32_t k, float ek) {
    const int64_t task = (int64_t)(k >> kRecordCountBits);
    const uint32_t c = (k & kCountMask) + 1u;
    if (task != prev_task) {
      if (prev_task >= 0) E = __fadd_rn(E, __fmul_rn((float)cnt, e));
      prev_task = task;
      e = ek;
      cnt = 0;
    }
    cnt += c;
  }
  // segment record k, the task's hit energy read from the event's part of
  // the table when the task changes
  __device__ __forceinline__ void add(uint32_t k, const float* __restrict__ ev_ehit) {
    const int64_t task = (int64_t)(k >> kRecordCountBits);
    const uint32_t c = (k & kCountMask) + 1u;
    if (task != prev_task) {
      if (prev_task >= 0) E = __fadd_rn(E, __fmul_rn((float)cnt, e));
      prev_task = task;
      e = ev_ehit[task];
      cnt = 0;
    }
    cnt += c;
  }
  // the folded float, as the FP64 row value the compaction reads (an exact
  // widening done with integer operations)
  __device__ __forceinline__ double result() const { return f32_to_f64_bits(__fadd_rn(E, __fmul_rn((float)cnt, e))); }
};

// Ascending sort of N keys in registers (N a power of two): Batcher's
// odd-even merge sort (Batcher 1968; 19 compare-exchanges for 8 keys, 63 for
// 16), every index a compile-time constant; absent records are all ones and
// sort last.
__device__ __forceinline__ void cmpx(uint32_t& x, uint32_t& y) {
  const uint32_t lo = min(x, y), hi = max(x, y);
  x = lo;
  y = hi;
}

// Merge of the sorted halves of r[LO, LO + N) taken with stride R: the odd
// and even subsequences recursively, then neighbours R apart.
template <int LO, int N, int R, int M>
__device__ __forceinline__ void oe_merge(uint32_t (&r)[M]) {
  constexpr int S = 2 * R;
  if constexpr (S < N) {
    oe_merge<LO, N, S>(r);
    oe_merge<LO + R, N, S>(r);
#pragma unroll
    for (int i = LO + R; i + R < LO + N; i += S) cmpx(r[i], r[i + R]);
  } else {
    cmpx(r[LO], r[LO + R]);
  }
}
template <int LO, int N, int M>
__device__ __forceinline__ void oe_sort(uint32_t (&r)[M]) {
  if constexpr (N > 1) {
    oe_sort<LO, N / 2>(r);
    oe_sort<LO + N / 2, N / 2>(r);
    oe_merge<LO, N, 1>(r);
  }
}
template <int N>
__device__ __forceinline__ void merge_sort_net(uint32_t (&r)[N]) {
  oe_sort<0, N>(r);
}

// Sort and fold of a segment of n <= N records (a register copy).  The hit
// energies of the sorted records' tasks are loaded all at once, ahead of the
// fold, so that the cell waits for one load latency, not one per task.
template <int N>
__device__ __forceinline__ double fold_small(const uint32_t* __restrict__ recs, int64_t a, int n,
                                            const float* __restrict__ ev_ehit) {
  uint32_t r[N];
#pragma unroll
  for (int j = 0; j < N; ++j) r[j] = j < n ? recs[a + j] : ~0u;
  merge_sort_net<N>(r);
  float e[N];
#pragma unroll
  for (int j = 0; j < N; ++j) e[j] = j < n ? ev_ehit[r[j] >> kRecordCountBits] : 0.0f;
  Fold f;
#pragma unroll
  for (int j = 0; j < N; ++j)
    if (j < n) f.add(r[j], e[j]);
  return f.result();
}

// Cell c's segment [a, b) after the scatter: cell_off[c] holds its end, which
// is the next cell's start.
__device__ __forceinline__ void segment(const int32_t* __restrict__ cell_off, int64_t c, int64_t cap, int64_t& a,
                                        int64_t& b) {
  a = c > 0 ? cell_off[c - 1] : 0;
  b = min((int64_t)cell_off[c], cap);
}

// The hit energies of the tasks of cell c's event.
__device__ __forceinline__ const float* event_ehit(const float* __restrict__ task_ehit,
                                                  const int64_t* __restrict__ base, int64_t c, uint32_t acc_stride) {
  return task_ehit + base[(uint32_t)c / acc_stride];
}

// One thread per cell: segments of up to 8 records (92 % of the hit cells of
// pile-up events) are sorted as a copy in registers, with nothing written
// back, and folded; segments of 9 to 16 and of 17 to kThreadSortMax records
// are listed for the two k_det_fold_mid kernels and longer ones for
// k_det_fold_big, so that the warps of each kernel run one path.  The list
// array holds three lists, from its start, a third in and two thirds in: a
// listed cell has at least 9 records, so each list fits its third.
__global__ void __launch_bounds__(256) k_det_fold(const uint32_t* __restrict__ recs,
                                                  const int32_t* __restrict__ cell_off, int64_t n_cells_all, Sizes* sz,
                                                  int64_t cap, uint32_t acc_stride, const int64_t* __restrict__ base,
                                                  const float* __restrict__ task_ehit, double* __restrict__ acc,
                                                  int64_t* __restrict__ lists) {
  if (sz->flags & (FCS_FLAG_HIT_CAPACITY | FCS_FLAG_KEY_BITS)) return;
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  // warp-uniform trips, so that the lists take one counter update per warp
  for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); c0 < n_cells_all;
       c0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = c0 + lane;
    // the segment ends (int32, as is the record count): each lane's, and the
    // one before the warp's first cell
    const int32_t b = c < n_cells_all ? cell_off[c] : 0;
    const int32_t b0 = (lane == 0 && c0 > 0) ? cell_off[c0 - 1] : 0;
    const int32_t bp = __shfl_up_sync(0xffffffffu, b, 1);
    const int32_t a = lane ? bp : b0;
    const int32_t n = c < n_cells_all ? min((int64_t)b, cap) - a : 0;
    const unsigned mb = __ballot_sync(0xffffffffu, n > kThreadSortMax);
    const unsigned m16 = __ballot_sync(0xffffffffu, n > 8 && n <= 16);
    const unsigned m32 = __ballot_sync(0xffffffffu, n > 16 && n <= kThreadSortMax);
    if (mb | m16 | m32) {
      unsigned long long bb = 0, b16 = 0, b32 = 0;
      if (lane == 0) {
        if (mb) bb = atomicAdd((unsigned long long*)&sz->n_big, (unsigned long long)__popc(mb));
        if (m16) b16 = atomicAdd((unsigned long long*)&sz->n_mid, (unsigned long long)__popc(m16));
        if (m32) b32 = atomicAdd((unsigned long long*)&sz->n_mid32, (unsigned long long)__popc(m32));
      }
      bb = __shfl_sync(0xffffffffu, bb, 0);
      b16 = __shfl_sync(0xffffffffu, b16, 0);
      b32 = __shfl_sync(0xffffffffu, b32, 0);
      if ((mb >> lane) & 1u) lists[bb + __popc(mb & below)] = c;
      if ((m16 >> lane) & 1u) lists[cap / 3 + (int64_t)(b16 + __popc(m16 & below))] = c;
      if ((m32 >> lane) & 1u) lists[2 * (cap / 3) + (int64_t)(b32 + __popc(m32 & below))] = c;
    }
    if (n > 0 && n <= 8) acc[c] = fold_small<8>(recs, a, (int)n, event_ehit(task_ehit, base, c, acc_stride));
  }
}

// One thread per listed cell of 9 to 16 (N = 16) or 17 to 32 records
// (N = 32): sorted as a copy in registers, then folded.
template <int N>
__global__ void __launch_bounds__(256) k_det_fold_mid(const uint32_t* __restrict__ recs,
                                                      const int32_t* __restrict__ cell_off, int64_t n_cells_all,
                                                      const Sizes* sz, int64_t cap, uint32_t acc_stride,
                                                      const int64_t* __restrict__ base,
                                                      const float* __restrict__ task_ehit, double* __restrict__ acc,
                                                      const int64_t* __restrict__ lists) {
  static_assert(N == 16 || N == kThreadSortMax, "two mid classes");
  if (sz->flags & (FCS_FLAG_HIT_CAPACITY | FCS_FLAG_KEY_BITS)) return;
  const int64_t n_list = N == 16 ? sz->n_mid : sz->n_mid32;
  const int64_t* list = lists + (N == 16 ? cap / 3 : 2 * (cap / 3));
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_list; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = list[q];
    int64_t a, b;
    segment(cell_off, c, cap, a, b);
    acc[c] = fold_small<N>(recs, a, (int)(b - a), event_ehit(task_ehit, base, c, acc_stride));
  }
}

// One warp per long segment: a bitonic sort in shared memory (segments of up
// to kBigMax records; longer ones take heapsort in place), then lane 0 folds.
constexpr int kBigWarps = 4;
constexpr int kBigMax = 1024;
__global__ void __launch_bounds__(32 * kBigWarps) k_det_fold_big(uint32_t* __restrict__ recs,
                                                                 const int32_t* __restrict__ cell_off,
                                                                 int64_t n_cells_all, const Sizes* sz, int64_t cap,
                                                                 uint32_t acc_stride, const int64_t* __restrict__ base,
                                                                 const float* __restrict__ task_ehit,
                                                                 double* __restrict__ acc,
                                                                 const int64_t* __restrict__ big) {
  __shared__ uint32_t s_rec[kBigWarps][kBigMax];
  __shared__ float s_e[kBigWarps][kBigMax];  // the sorted records' hit energies
  if (sz->flags & (FCS_FLAG_HIT_CAPACITY | FCS_FLAG_KEY_BITS)) return;
  const int64_t n_big = sz->n_big;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  uint32_t* s = s_rec[wi];
  float* se = s_e[wi];
  for (int64_t q = (int64_t)blockIdx.x * kBigWarps + wi; q < n_big; q += (int64_t)gridDim.x * kBigWarps) {
    const int64_t c = big[q];
    int64_t a, b;
    segment(cell_off, c, cap, a, b);
    const int64_t n = b - a;
    uint32_t* seg = recs + a;
    const float* ev_ehit = event_ehit(task_ehit, base, c, acc_stride);
    if (n > kBigMax) {
      if (lane == 0) {
        sort_segment(seg, n);
        Fold f;
        for (int64_t j = 0; j < n; ++j) f.add(seg[j], ev_ehit);
        acc[c] = f.result();
      }
      __syncwarp();
      continue;
    }
    int m = 1;
    while (m < n) m <<= 1;
    for (int j = lane; j < m; j += 32) s[j] = j < n ? seg[j] : ~0u;
    __syncwarp();
    for (int k = 2; k <= m; k <<= 1) {
      for (int jj = k >> 1; jj > 0; jj >>= 1) {
        for (int i = lane; i < m; i += 32) {
          const int l = i ^ jj;
          if (l > i) {
            const uint32_t x = s[i], y = s[l];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              s[i] = y;
              s[l] = x;
            }
          }
        }
        __syncwarp();
      }
    }
    // the hit energies, loaded by all lanes at once; then the first lane folds
    for (int j = lane; j < n; j += 32) se[j] = ev_ehit[s[j] >> kRecordCountBits];
    __syncwarp();
    if (lane == 0) {
      Fold f;
      for (int64_t j = 0; j < n; ++j) f.add(s[j], se[j]);
      acc[c] = f.result();
    }
    __syncwarp();
  }
}

constexpr int kMaxDevices = 64;

// Blocks of 256 threads of k_det_fold that one SM holds at once (per device,
// looked up once): the kernel loops grid-stride, and a grid beyond one wave of
// resident blocks would run its surplus as a second, mostly empty wave.
int fold_resident_blocks() {
  static std::atomic<int> occ_by_device[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = kMaxDevices - 1;
  int occ = occ_by_device[dev].load(std::memory_order_relaxed);
  if (!occ) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_det_fold, 256, 0) != cudaSuccess) {
      (void)cudaGetLastError();
      occ = 1;
    }
    occ = std::max(occ, 1);
    occ_by_device[dev].store(occ, std::memory_order_relaxed);
  }
  return occ;
}

}  // namespace

cudaError_t launch_det_reduce(const GeoDev& g, WsDev w, int32_t rows, int key_task_bits, int64_t* scratch,
                              const int64_t* event_offsets, int32_t ev_lo, ScanTmp tmp, const Launch& L) {
  const int64_t n_cells_all = (int64_t)rows * g.acc_stride;
  uint32_t* counters = reinterpret_cast<uint32_t*>(w.acc);
  int64_t* base = scratch;                                       // [rows] first task of each event
  int32_t* cell_off = reinterpret_cast<int32_t*>(scratch + rows);  // [n_cells_all] segment starts, then ends
  const uint32_t stride = (uint32_t)g.acc_stride;
  k_det_bases<<<(rows + 255) / 256, 256, 0, L.s>>>(event_offsets, ev_lo, rows, w.poff, w.sizes, base);
  cudaError_t e = launch_scan_u32_zero(counters, cell_off, n_cells_all, tmp, L.s);
  if (e != cudaSuccess) return e;
  const int cell_shift = kRecordCountBits + key_task_bits;
  const uint64_t task_mask = (key_task_bits >= 64) ? ~0ull : ((1ull << key_task_bits) - 1ull);
  uint32_t* segs = reinterpret_cast<uint32_t*>(w.keys_alt);
  k_det_scatter<<<L.num_sms * 8, 256, 0, L.s>>>(w.keys, w.sizes, w.rec_cap, cell_shift, task_mask, cell_off,
                                                n_cells_all, stride, base, segs);
  // the slot array is free after the scatter: it lists the segments of more
  // than 8 records
  int64_t* lists = reinterpret_cast<int64_t*>(w.keys);
  k_det_fold<<<L.num_sms * fold_resident_blocks(), 256, 0, L.s>>>(segs, cell_off, n_cells_all, w.sizes, w.rec_cap,
                                                                  stride, base, w.tehit, w.acc, lists);
  k_det_fold_mid<16><<<L.num_sms * 4, 256, 0, L.s>>>(segs, cell_off, n_cells_all, w.sizes, w.rec_cap, stride, base,
                                                     w.tehit, w.acc, lists);
  k_det_fold_mid<kThreadSortMax><<<L.num_sms * 2, 256, 0, L.s>>>(segs, cell_off, n_cells_all, w.sizes, w.rec_cap,
                                                                stride, base, w.tehit, w.acc, lists);
  k_det_fold_big<<<L.num_sms * 4, 32 * kBigWarps, 0, L.s>>>(segs, cell_off, n_cells_all, w.sizes, w.rec_cap, stride,
                                                            base, w.tehit, w.acc, lists);
  return cudaGetLastError();
}

}  // namespace fcs
