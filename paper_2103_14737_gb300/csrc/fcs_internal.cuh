// fcs_internal.cuh - device data layout and launcher declarations shared by
// the translation units of libfcs (not part of the public ABI).
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "fcs.h"  // include/ is on the include path (build.py)

namespace fcs {

constexpr int kMaxLayers = 32;
constexpr int kMaxRegions = 256;
constexpr int kNBins = 128;      // 16 r-bins x 8 alpha-bins
constexpr int kNR = 16;
constexpr int kNA = 8;
constexpr int kGuideCells = 128; // guide cells per histogram (top 7 bits of word 0)
constexpr int kRecordChunk = 256;  // deterministic mode: record slots a warp takes at a time
constexpr int64_t kRecordSlack = 1 << 22;  // slots beyond the hits: the warps' partly filled chunks
constexpr int kGranule = 128;    // hits per granule of the tile -> task map (divides every tile)
constexpr int kRecordCountBits = 5;  // deterministic mode: count - 1 in the low 5 bits
constexpr int kLfactEntries = 8192;  // log k! table for the FP32 Poisson test (k < 8192)

// Task record: one (event, particle, layer) of the hit loop of Listing 1.
// 32 bytes (one sector); tasks are stored in (event, particle, layer) order.
// The hit count n and first hit live in the per-task arrays tn and th (the
// hits of task t are the hit numbers [th[t], th[t] + tn[t]) of its event
// range); the hit energy is fl32(El / n) (Listing 1: float Ehit = E(layer) /
// nhit), formed where a kernel needs it.
struct __align__(16) TaskRec {
  int32_t entry;       // parametrisation entry including the layer
  float El;            // layer energy fl32(E f_l), MeV
  float eta_c, phi_c;
  float s_eta, s_phi;  // FP32 scale factors of the (r, alpha) -> (eta, phi) map
  int32_t particle;    // index within the event
  uint32_t ev_layer;   // batch-local event << 8 | layer
  __device__ __forceinline__ int32_t event() const { return (int32_t)(ev_layer >> 8); }
  __device__ __forceinline__ int32_t layer() const { return (int32_t)(ev_layer & 0xFFu); }
};
static_assert(sizeof(TaskRec) == 32, "TaskRec layout");
constexpr int32_t kMaxEventsPerCall = 1 << 24;  // batch-local events fit the record's 24 bits

// FP32 view of a region for the fast path (shared-memory staged): the scaled
// indices are te = eta inv_deta + ek and tp = phi inv_dphi + pk, one FMA each,
// and the constant parts of their error bounds come with the region.
struct __align__(16) RegionF {
  float ek, inv_deta;  // -eta_lo / deta (FP32 of the FP64 quotient), 1 / deta
  float pk, inv_dphi;  // -phi_lo / dphi, 1 / dphi
  float n_eta_hf;      // n_eta - 1/2: the scaled eta index is clamped to [1/2, n_eta - 1/2]
  float ce;            // |ek| 2^-23 + 2^-22: eta-index bound beyond the position's and |te| 2^-21
  float cp;            // |pk| 2^-23 + 2^-22: phi-index bound beyond the position's and |tp| 2^-21
  int32_t n_phi, cell_off;
  int32_t pad[3];
};
static_assert(sizeof(RegionF) == 48, "RegionF layout");

// Device geometry (all pointers device memory owned by fcs_geo).
struct GeoDev {
  int32_t n_layers, n_regions, n_cells, acc_stride;
  const RegionF* regf;
  const double* eta_lo;  // FP64 copies for the recheck path
  const double* deta;
  const double* phi_lo;
  const double* dphi;
  const double* split;   // split[r] for r > layer's first region
  const float* split32;  // [n_regions] FP32 of split (the lower ownership boundary); -inf for a layer's first
  const int32_t* n_eta;
  const int32_t* n_phi;
  const int32_t* cell_off;
  const int32_t* lrb;    // [n_layers + 1]
  const double* rz;      // [n_layers]
  const float* rinv32;   // [n_layers] 1 / fl32(R), correctly rounded, for the fast path
  const int32_t* barrel; // [n_layers]
};

// Device parametrisation.
struct ParamDev {
  int32_t NT, NE, NH, NL;
  double eta_scale;
  int32_t ebin_min;
  int32_t eta_scale_int; // eta_scale when it is an integer in [1, 255] (exact integer binning), else 0
  int32_t n_entries;     // NT * NE * NH * NL
  int32_t n_lfact;       // entries of lfact
  const float* lfact;    // [n_lfact] FP32 of lgamma(k + 1) (host libm, rounded once)
  const double* lfact64; // [n_lfact] lgamma(k + 1) of the host libm, the FP64 Poisson test's value
  const float* frac;     // [n_entries]
  const float* shape_w;  // [n_entries][128] shape weights (the gradient's likelihood ratios)
  const float* mhe;      // [n_entries]
  const uint32_t* thr;   // [n_entries][128] inverse-CDF thresholds
  const uint2* guide;    // [n_entries][128] packed guide cells (fcs_params.cu: thresholds T[lo], T[lo + 1]
                         // as offsets within the cell, lo, hi - lo)
  const float* r_edges;  // [17]
  const float* a_edges;  // [9]
};

// Device-side sizes and status of one call (in the workspace).
struct Sizes {
  int64_t n_tasks;
  int64_t n_hits;
  int64_t n_recheck;    // entries appended to the recheck queue (may exceed its capacity)
  int64_t n_records;    // deterministic mode: records written
  int64_t n_slots;      // deterministic mode: record slots handed out (chunks of kRecordChunk)
  int64_t nnz;          // non-zero cells of the current event range
  int64_t nnz_total;    // running output size over the call (per-event mode)
  int64_t n_inline;     // recheck hits done inline because the queue was full
  int64_t task_base;    // tasks / hits of the earlier event ranges of the call
  int64_t hit_base;     //   (per-event mode; offsets of the debug dumps)
  int64_t recheck_total;  // recheck hits over the call
  int64_t n_part;       // particles of the current event range (checked against the capacity)
  int64_t n_big;        // deterministic mode: cells with more records than one thread sorts
  int64_t n_mid;        // deterministic mode: cells of 9 to 16 records (sorted by their own kernel)
  int64_t n_mid32;      //   and of 17 to 32 records
  int64_t n_pdefer;     // inversion draws deferred to FP64 in the current range (front of pdefer)
  int64_t n_pdefer_ptrs;  // PTRS draws deferred to FP64 in the current range (back of pdefer)
  unsigned long long queue;  // hit-kernel work-queue counter (tiles handed out)
  uint32_t flags;       // fcs_device_flag bits
  uint32_t n_poisson_fp64;  // Poisson draws that needed an FP64 decision (call total)
};
static_assert(sizeof(Sizes) % 8 == 0 && offsetof(Sizes, queue) % 8 == 0, "Sizes layout");

// Workspace views passed to kernels.
struct WsDev {
  Sizes* sizes;
  int64_t* pcount;     // [pcap] tasks per particle
  int64_t* poff;       // [pcap] exclusive offsets
  uint4* pinfo;        // [pcap] per particle: entry (without layer), event, layer mask, 0
  int64_t pcap;        // particle capacity
  TaskRec* tasks;      // [task_cap]
  float* tehit;        // [task_cap] deterministic mode: each task's hit energy, written by the
                       // hit kernel's tile that holds the task's first hit (a compact copy
                       // for the fold)
  int32_t* tn;         // [task_cap] hits of each task
  int64_t* th;         // [task_cap] first hit of each task (exclusive scan of tn)
  int32_t* pdefer;     // [pdefer_cap] tasks whose draw is redone in FP64: inversion draws from the
                       // front, PTRS draws from the back (their resume iteration waits in tn)
  int32_t* gmap;       // [gmap_cap] granule -> task
  uint2* recheck;      // [recheck_cap] (task, hit in task)
  double* acc;         // [rows][acc_stride] zero-maintained accumulation rows (FP64: see acc_add)
  int64_t task_cap, gmap_cap, recheck_cap, rows_cap, pdefer_cap;
  uint64_t* keys;      // deterministic mode record slots, one per hit [rec_cap]
  uint64_t* keys_alt;  // ping-pong buffer [rec_cap]
  int64_t rec_cap;
};

// Philox4x32-10 (Salmon et al., SC'11): published multipliers and Weyl
// constants; counter c, key (k0, k1).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The same generator with the ten round keys (k0 + i W0, k1 + i W1) given,
// e.g. from kernel parameters, so the key schedule costs no instructions.
struct PhiloxRoundKeys {
  uint32_t k[20];  // k[2 i] = k0 + i 0x9E3779B9, k[2 i + 1] = k1 + i 0xBB67AE85
};
__host__ __device__ inline PhiloxRoundKeys philox_round_keys(uint32_t k0, uint32_t k1) {
  PhiloxRoundKeys r;
  for (int i = 0; i < 10; ++i) {
    r.k[2 * i] = k0 + (uint32_t)i * 0x9E3779B9u;
    r.k[2 * i + 1] = k1 + (uint32_t)i * 0xBB67AE85u;
  }
  return r;
}
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const PhiloxRoundKeys& rk) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ rk.k[2 * i], lo1, hi0 ^ c.w ^ rk.k[2 * i + 1], lo0);
  }
  return c;
}

// Counter layout of the method's random streams:
// (index, layer | purpose << 16, particle in event, event).
constexpr uint32_t kPurposeHit = 0u;
constexpr uint32_t kPurposePoisson = 1u;
constexpr uint32_t kPurposeEnergyBin = 2u;

__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return __dmul_rn(__dadd_rn(__dmul_rn((double)(a >> 5), 67108864.0), (double)(b >> 6)),
                   1.0 / 9007199254740992.0);
}
__device__ __forceinline__ double u24d(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }
__device__ __forceinline__ float u24f(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// ---- accumulation rows ------------------------------------------------------
// Cells accumulate in FP64.  A deposit is the float count x Ehit of a group
// of hits (one rounding, relative 2^-24); FP64 sums of such terms carry no
// order-dependent error that reaches the float result, which the compaction
// rounds once.  (In FP32 a cell that collects thousands of equal group
// deposits drifts by the same rounding every time, and red.add.f32 flushes
// subnormal operands and results to zero.)  The hit kernel widens a deposit
// with the conversion instruction, exact for every float (no flush to zero
// in this build): one FP64-pipe instruction per warp step measured faster
// than the integer widening below (hit kernel 12.91 -> 12.72 ms on 1024
// pile-up events), which other kernels use where they store a float's FP64
// image: a normal float's exponent is rebiased by 1023 - 127; a subnormal
// m 2^-149 (and zero) is normalised by the position of m's leading bit.
__device__ __forceinline__ double f32_to_f64_bits(float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t a = u & 0x7FFFFFFFu;
  uint32_t hi, lo;
  if (a >= 0x00800000u) {
    hi = (a >> 3) + (896u << 20);
    lo = u << 29;
  } else {
    const int lz = __clz(a);                     // 9 .. 31 for a subnormal, 32 for zero
    const uint32_t m = (a << (lz - 8)) & 0x7FFFFFu;  // the bits below the leading one
    hi = a ? ((uint32_t)(905 - lz) << 20) | (m >> 3) : 0u;  // exponent (31 - lz) - 149 + 1023
    lo = m << 29;
  }
  return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)lo);
}
__device__ __forceinline__ void acc_add(double* cell, float v) { atomicAdd(cell, (double)v); }

// Round-to-nearest-even of an FP64 row value to float, with integer
// operations where the result is a normal float; zero, subnormal, overflowing
// and non-finite values take the conversion instruction.
__device__ __forceinline__ float acc_to_f32(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t e = (hi >> 20) & 0x7FFu;
  if (e < 897u || e > 1150u) return __double2float_rn(d);
  uint32_t r = ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const uint32_t dropped = lo & 0x1FFFFFFFu;
  r += (dropped > 0x10000000u || (dropped == 0x10000000u && (r & 1u))) ? 1u : 0u;  // a carry rounds the exponent up
  return __uint_as_float(r | (hi & 0x80000000u));
}

// ---- launchers (host) -------------------------------------------------------
struct Launch {
  cudaStream_t s;
  int num_sms;
};

// fcs_params.cu
cudaError_t launch_build_tables(const float* shape_w, int n_entries, uint32_t* thr, uint2* guide,
                                int32_t* bad, cudaStream_t s);

// fcs_scan.cu: exclusive scan of n int64 values (n on the host or device),
// one pass.  The state (ticket, done count, one status word per tile) is zero
// between scans; scan_state_words(n) words hold a scan of up to n elements.
struct ScanTmp {
  uint64_t* state;    // zeroed device words: [0] tile ticket, [1] CTAs done, [2 ..] tile status
  int64_t cap_tiles;  // tiles the status words cover
  uint32_t* flags;    // device flag word of the call (FCS_FLAG_WAIT_TIMEOUT)
  int grid;           // persistent CTAs
};
int64_t scan_state_words(int64_t max_elements);
cudaError_t launch_scan_i64(const int64_t* in, int64_t* out, const int64_t* n_dev, int64_t n_host,
                            int64_t* total_dst, int64_t total_add_base_from_dst, ScanTmp tmp,
                            cudaStream_t s);
// Self-test of the scan's bounded wait (a tile that never publishes): the
// device flag word and the kernel's time in ms.
cudaError_t scan_wait_selftest(uint32_t* flags_out, float* ms, cudaStream_t s);
// Exclusive scan of n uint32 values into int32 (no base, no total); zeroes
// the inputs as it reads them.
cudaError_t launch_scan_u32_zero(uint32_t* in, int32_t* out, int64_t n, ScanTmp tmp, cudaStream_t s);
// The hit offsets th (exclusive scan of the tasks' hit counts tn, *n_tasks of
// them; total to *n_hits) and the tile map gmap[g] = the task holding hit
// g * kGranule, for g < gmap_cap.
cudaError_t launch_scan_hits(const int32_t* tn, int64_t* th, const int64_t* n_tasks, int64_t* n_hits, int32_t* gmap,
                             int64_t gmap_cap, ScanTmp tmp, cudaStream_t s);

// fcs_tasks.cu: tasks, Poisson counts and the two scans (task and hit offsets);
// then the records' hit offsets, the tile map and the validation dumps.
// n_part_max: an upper bound of the range's particles (sizes the grids).
cudaError_t launch_task_counts(const GeoDev& g, const ParamDev& p, const fcs_particles& parts,
                               int32_t ev_lo, int32_t ev_hi, uint32_t k0, uint32_t k1,
                               int64_t first_event, WsDev w, ScanTmp tmp, int64_t n_part_max,
                               int energy_interp, const Launch& L);
cudaError_t launch_task_finish(WsDev w, const fcs_debug* dbg, int fill_map, int64_t n_task_max,
                               const Launch& L);

// Draws i = 0..n-1 with means mu (device) by the FP32 path and by the FP64
// definition (fcs_poisson_audit).
cudaError_t launch_poisson_audit(const ParamDev& p, const float* mu, int64_t n, uint32_t k0, uint32_t k1,
                                 int32_t* n32, int32_t* n64, const Launch& L);

// fcs_hits.cu: what the hit kernel does with a certified hit
enum HitMode : int {
  kModeAtomic = 0,  // float atomics into the accumulation rows
  kModeDet = 1,     // (cell, task, count) records for the sort-by-cell reduction
  kModeGrad = 2,    // gather dL/dE_cell, add E_hit dL/dE_cell to the (entry, bin) score
};
struct HitCfg {
  int block;
  int hpt;
  int det;  // deterministic (record) mode
};
cudaError_t launch_hits(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0,
                        uint32_t k1, int64_t first_event, const HitCfg& hc, int key_task_bits,
                        const fcs_debug* dbg, const Launch& L);
// One launch over the hits [h_lo, h_hi) of one task (the paper's per-task
// kernel launches, Sec. 4), a CTA per tile.
cudaError_t launch_hits_task(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0, uint32_t k1,
                             int64_t first_event, const HitCfg& hc, int key_task_bits, const fcs_debug* dbg,
                             int64_t h_lo, int64_t h_hi, int32_t task, const Launch& L);
cudaError_t launch_recheck(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0,
                           uint32_t k1, int64_t first_event, int det, int key_task_bits,
                           const fcs_debug* dbg, const Launch& L);
int hits_max_smem_tasks();

// fcs_grad.cu: the adjoint of the hit loop.  grad_in: dL/dE_cell rows of the
// range (row stride n_cells); grad_acc: FP64 [n_entries][128] scores;
// touched: [n_entries] flags of entries with scores.
cudaError_t launch_hits_grad(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0,
                             uint32_t k1, int64_t first_event, const HitCfg& hc, const float* grad_in,
                             double* grad_acc, uint8_t* touched, const Launch& L);
cudaError_t launch_recheck_grad(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0,
                                uint32_t k1, int64_t first_event, const float* grad_in, double* grad_acc,
                                uint8_t* touched, const Launch& L);
cudaError_t launch_grad_finalize(const ParamDev& p, double* grad_acc, uint8_t* touched, float* d_frac,
                                 float* d_shape_w, const Launch& L);
cudaError_t launch_check_params(const float* frac, const float* mean_hit_E, const float* shape_w,
                                int n_entries, uint32_t* bad, cudaStream_t s);

// fcs_compact.cu
// One pass over the rows with a decoupled look-back over the chunks (tmp:
// zeroed scan state with a status word per chunk, left zeroed).  max_ctas > 0
// caps the grid (its CTAs loop over the chunks), so that it leaves SMs to
// work running beside it on another stream.
cudaError_t launch_compact(const GeoDev& g, WsDev w, int32_t rows, int32_t ev_lo, ScanTmp tmp, float* cells_out,
                           int32_t* cell_ids, float* cell_E, int64_t* event_offsets_out, int64_t capacity,
                           int max_ctas, const Launch& L);

// fcs_sort.cu
int64_t compact_chunks(int32_t n_cells, int32_t rows);
// Deterministic mode: the records of the range (hit slots) grouped by cell
// and folded into the accumulation rows, whose uint32 record counters the
// hit kernel filled.  scratch: [rows * (acc_stride + 1)] int64 (each event's
// first task, then the cells' int32 segment offsets); event_offsets and
// ev_lo: the range's events.  The compaction then runs as in atomic mode.
cudaError_t launch_det_reduce(const GeoDev& g, WsDev w, int32_t rows, int key_task_bits, int64_t* scratch,
                              const int64_t* event_offsets, int32_t ev_lo, ScanTmp tmp, const Launch& L);

}  // namespace fcs
