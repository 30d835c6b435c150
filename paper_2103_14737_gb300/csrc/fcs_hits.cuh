// fcs_hits.cuh - the per-hit kernel of the hit loop (Listing 1: simulate_hit
// chain; Listing 2: HitCellMapping_d / getDDE + atomicAdd).
//
// One thread per hit as in the paper's sim_a kernel (Sec. 4), but persistent:
// CTAs take tiles of BLOCK * HPT consecutive hits from an atomic work queue
// over the whole batch (the grouped simulation of Sec. 4 at batch scale); a
// tile's task records are staged in shared memory and each hit finds its task
// through a block max-scan of task start positions.  Per hit:
//   Philox4x32-10 block (hit, layer, particle, event)        -> 4 words
//   word 0: shape bin by guide table + binary search          (integer, exact)
//   words 1, 2: uniform position in the (r, alpha) bin        (FP32)
//   (r, alpha) -> (eta, phi) linear map around the task centre (FP32, __sincosf)
//   region search + grid index                                 (FP32)
// The FP32 result is certified against a rigorous error bound; a hit whose
// eta or phi lies within the bound of a cell or region edge is queued and
// decided by the FP64 recheck kernel, which repeats the oracle's FP64 steps
// (the paper's two FP32 cell mismatches in 62M hits were removed with FP64,
// Sec. 6).  Certified hits are deposited with warp-aggregated atomics (Sec. 4
// chose atomicAdd) of the float count x Ehit into FP64 cells or, in
// deterministic mode, emitted as (cell, task, count) records for the
// sort-by-cell reduction.
#pragma once

#include <type_traits>

#include "fcs_internal.cuh"

namespace fcs {

constexpr int kSmemTasks = 128;  // staged tasks per tile (more: the hit loop reads the records)

struct HitKParams {
  GeoDev g;
  ParamDev p;
  WsDev w;
  int32_t ev_lo;
  uint32_t k0, k1;
  uint32_t first_event_lo;
  int32_t key_task_bits;
  int32_t key32;  // 32-bit (cell, task-in-tile) match keys (n_cells < 2^19)
  int32_t* dbg_hit_cell;
  int16_t* dbg_hit_bin;
  int64_t dbg_hit_cap;
  // gradient mode
  const float* grad_in;  // dL/dE_cell of the range's events, row stride n_cells
  double* grad_acc;      // [n_entries][128] sum of E_hit dL/dE_cell per (entry, shape bin)
  uint8_t* grad_touched; // [n_entries] set where grad_acc has contributions
  // one launch per task (static_tiles != 0): CTA b takes tile b of the hits
  // [h_lo, h_hi), all of task t_last
  int64_t h_lo, h_hi;
  int32_t t_last;
  int32_t static_tiles;
  PhiloxRoundKeys rk;  // the round keys of (k0, k1), read from the parameter bank
};

// ---- shape bin: inverse CDF by guide table and binary search --------------
// Binary search for the first k in [lo, hi) with x0 < T[k], else hi.
static __device__ __noinline__ int bin_search(const uint32_t* T, int lo, int hi, uint32_t x0) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (x0 < __ldg(T + mid)) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// The bin of word x0: the packed guide cell of x0's top 7 bits gives lo and
// the first two thresholds of the cell as offsets (fcs_params.cu); two
// comparisons decide unless the cell spans three or more bins and x0 lies
// past the second threshold (a few percent of the words), which finishes with
// a binary search over the thresholds.
__device__ __forceinline__ int sample_bin(const ParamDev& p, int32_t entry, uint32_t x0) {
  const uint2 gg = __ldg(p.guide + ((uint32_t)entry * kGuideCells + (x0 >> 25)));
  const uint32_t xo = x0 & 0x1FFFFFFu;
  const uint32_t t0 = gg.x & 0x1FFFFFFu;
  const uint32_t t1 = __funnelshift_r(gg.x, gg.y, 25) & 0x1FFFFFFu;
  const int lo = (int)((gg.y >> 18) & 0x7Fu);
  const int bin = lo + (xo > t0 ? 1 : 0) + (xo > t1 ? 1 : 0);
  const int span = (int)(gg.y >> 25);
  if (span > 2 && xo > t1) return bin_search(p.thr + (uint32_t)entry * kNBins, lo + 2, lo + span, x0);
  return bin;
}

// ---- FP64 path: the oracle's steps, each rounding once ----------------------
__device__ __forceinline__ void scales64(const GeoDev& g, int layer, double eta_c, double* s_eta,
                                         double* s_phi) {
  const double R = g.rz[layer];
  if (g.barrel[layer]) {
    *s_phi = __ddiv_rn(1.0, R);
    *s_eta = __ddiv_rn(1.0, __dmul_rn(R, cosh(eta_c)));
  } else {
    const double ae = fabs(eta_c);
    const double sh = sinh(ae);
    const double m = __ddiv_rn(__dmul_rn(tanh(ae), sh), R);
    *s_phi = __ddiv_rn(sh, R);
    *s_eta = (eta_c < 0.0) ? m : -m;
  }
}

__device__ __forceinline__ int32_t lookup64(const GeoDev& g, int layer, double eta, double phi) {
  const int rb = g.lrb[layer], re = g.lrb[layer + 1];
  int r = rb;
  for (int k = rb + 1; k < re; ++k)
    if (eta >= g.split[k]) r = k;
  const int ne = g.n_eta[r], np = g.n_phi[r];
  const double te = __ddiv_rn(__dsub_rn(eta, g.eta_lo[r]), g.deta[r]);
  int64_t ie;
  if (!(te >= 0.0)) ie = 0;  // also NaN
  else if (te >= (double)ne) ie = ne - 1;
  else ie = (int64_t)floor(te);
  if (ie > ne - 1) ie = ne - 1;
  double tp = __ddiv_rn(__dsub_rn(phi, g.phi_lo[r]), g.dphi[r]);
  const double lim = 4503599627370496.0;
  if (tp > lim) tp = lim;
  if (!(tp >= -lim)) tp = -lim;  // also NaN
  int64_t ip = (int64_t)floor(tp) % (int64_t)np;
  if (ip < 0) ip += np;
  return g.cell_off[r] + (int32_t)ie * np + (int32_t)ip;
}

static __device__ __noinline__ int32_t cell_fp64(const GeoDev& g, const ParamDev& p, int32_t layer,
                                                 float eta_c, float phi_c, uint4 x, int bin) {
  const int ir = bin >> 3, ia = bin & 7;
  const double r_lo = (double)p.r_edges[ir], r_hi = (double)p.r_edges[ir + 1];
  const double a_lo = (double)p.a_edges[ia], a_hi = (double)p.a_edges[ia + 1];
  const double r = __dadd_rn(r_lo, __dmul_rn(u24d(x.y), __dsub_rn(r_hi, r_lo)));
  const double alpha = __dadd_rn(a_lo, __dmul_rn(u24d(x.z), __dsub_rn(a_hi, a_lo)));
  double s_eta, s_phi;
  scales64(g, layer, (double)eta_c, &s_eta, &s_phi);
  const double deta = __dmul_rn(__dmul_rn(r, cos(alpha)), s_eta);
  const double dphi = __dmul_rn(__dmul_rn(r, sin(alpha)), s_phi);
  const double eta = __dadd_rn((double)eta_c, deta);
  const double phi = __dadd_rn((double)phi_c, dphi);
  return lookup64(g, layer, eta, phi);
}

// ---- shared tables of a CTA ---------------------------------------------------
struct HitSmemTables {
  RegionF reg[kMaxRegions];
  float split[kMaxRegions];  // lower ownership boundary of each region (FP32)
  int32_t lrb[kMaxLayers + 1];
  float4 rb[kNR];  // r bin: lo, width, hi, hi 2^-17 (the bin's term of the error bound)
  float2 ab[kNA];  // alpha bin: lo - pi, width
};

__device__ __forceinline__ void load_tables(HitSmemTables& t, const GeoDev& g, const ParamDev& p) {
  for (int i = threadIdx.x; i < g.n_regions; i += blockDim.x) {
    t.reg[i] = g.regf[i];
    t.split[i] = g.split32[i];
  }
  for (int i = threadIdx.x; i <= g.n_layers; i += blockDim.x) t.lrb[i] = g.lrb[i];
  if (threadIdx.x < kNR) {
    const float lo = p.r_edges[threadIdx.x], hi = p.r_edges[threadIdx.x + 1];
    t.rb[threadIdx.x] = make_float4(lo, hi - lo, hi, hi * 0x1p-17f);
  }
  if (threadIdx.x < kNA) {
    const double lo = p.a_edges[threadIdx.x], hi = p.a_edges[threadIdx.x + 1];
    t.ab[threadIdx.x] = make_float2((float)(lo - 3.141592653589793), (float)(hi - lo));
  }
}

// ---- FP32 fast path --------------------------------------------------------
// Error bound of the FP32 eta (and likewise phi) against the FP64 value:
//   cos/sin: |alpha32 - alpha| <= ~2^-21.4 (alpha - pi in [-pi, pi] from an
//     FMA of FP32 table values) and __sincosf's documented absolute error on
//     [-pi, pi] (2^-21.19 for cos, 2^-21.41 for sin): <= 2^-20.4 in all;
//   r32 <= r_hi * 2^-23 off; s32 (coshf, sinhf and tanhf within 2, 3 and 2
//     ulp as documented, a correctly rounded 1/R or 1/cosh and up to two
//     products: <= 8 ulp) <= 2^-20 relative; the two products 2 * 2^-24
//     relative:
//   => |deta32 - deta| <= r_hi |s_eta| 2^-19; bound used: r_hi |s| 2^-17;
//   the final add rounds by |eta| 2^-24; bound used: |eta| 2^-21.
// Scaled index te = fl(eta32 inv + ek) with inv = fl(1/deta), ek =
// fl(-eta_lo/deta): |te - te*| <= be inv + (|eta| inv) 2^-24 + |ek| 2^-24 +
// |te| 2^-24 (the reciprocal, the constant and the FMA's rounding), and
// |eta| inv <= |te| + |ek|; bound used: be inv + |ek| 2^-23 + |te| 2^-21 +
// 2^-22; |ek| 2^-23 + 2^-22 is the region's constant ce (and likewise cp for
// phi).
// A decision is certified when the FP32 value is farther than the bound
// (plus the FP32 rounding of the boundary) from the boundary it is compared
// with.
struct FastHit {
  int32_t cell;
  bool sure;
};

// The regions [a, b) of a task's layer that its hits can reach: every hit
// lies within r_max |s_eta| of eta_c in eta (r_max = the outer edge of the
// shape histogram), widened by 2^-8 relative and 2^-16 (1 + |eta_c|) for the
// FP32 scale factor and for the rounding of the FP32 and FP64 hit positions.
// Split q is left out of the search when the FP64 split lies below (above)
// every hit, judged from its FP32 copy with a 2^-22 relative margin, so the
// search over [a, b) decides exactly as the search over the whole layer and
// needs no certification at the splits it skips.
__device__ __forceinline__ uint32_t task_lay(const HitSmemTables& tb, int layer, float eta_c, float s_eta) {
  const int rb = tb.lrb[layer], re = tb.lrb[layer + 1];
  const float D = fmaf(tb.rb[kNR - 1].z * fabsf(s_eta), 1.00390625f, fmaf(fabsf(eta_c), 0x1p-16f, 0x1p-16f));
  const float L = eta_c - D, U = eta_c + D;
  int a = rb, b = re;
  for (int q = rb + 1; q < re; ++q) {
    const float sp = tb.split[q];
    if (fmaf(fabsf(sp), 0x1p-22f, sp) <= L) a = q;
    if (b == re && fmaf(-fabsf(sp), 0x1p-22f, sp) > U) b = q;
  }
  return (uint32_t)layer | ((uint32_t)a << 8) | ((uint32_t)b << 20);
}

// A task as the hit loop uses it, staged in shared memory per tile (48 B):
// 32-bit offsets and the Philox counter words are formed once per task.
struct TileTask {
  int32_t rel;      // first hit of the task - first hit of the tile (<= 0 for the tile's first task)
  int32_t entry;    // parametrisation entry (with layer)
  float Ehit, eta_c, phi_c, s_eta, s_phi;
  uint32_t ctr_y;   // layer | purpose << 16
  uint32_t ctr_z;   // particle in event
  uint32_t ctr_w;   // event number of the random stream
  uint32_t row_off; // row * acc_stride (atomic, deterministic) or row * n_cells (gradient)
  uint32_t lay;     // layer | first region << 8 | end region << 20 (the reachable regions)
};
static_assert(sizeof(TileTask) == 48, "TileTask layout");

// The tile's view of task t: hit offset relative to the tile start h0, the
// float hit energy fl32(El / n), the Philox counter words and the accumulation
// row.
__device__ __forceinline__ TileTask make_tile_task(const HitSmemTables& tb, const WsDev& w, int64_t t, int64_t h0,
                                                   uint32_t first_event_lo, int32_t ev_lo, uint32_t row_stride) {
  const TaskRec r = w.tasks[t];
  const int32_t layer = r.layer(), event = r.event();
  TileTask q;
  q.rel = (int32_t)(w.th[t] - h0);
  q.entry = r.entry;
  q.Ehit = __fdiv_rn(r.El, (float)w.tn[t]);
  q.eta_c = r.eta_c;
  q.phi_c = r.phi_c;
  q.s_eta = r.s_eta;
  q.s_phi = r.s_phi;
  q.ctr_y = (uint32_t)layer | (kPurposeHit << 16);
  q.ctr_z = (uint32_t)r.particle;
  q.ctr_w = first_event_lo + (uint32_t)event;
  q.row_off = (uint32_t)(event - ev_lo) * row_stride;
  q.lay = task_lay(tb, layer, r.eta_c, r.s_eta);
  return q;
}

template <typename TT>
__device__ __forceinline__ FastHit fast_cell(const HitSmemTables& tb, const TT& T, uint4 x, int bin) {
  const int ir = bin >> 3, ia = bin & 7;
  const float ur = u24f(x.y), ua = u24f(x.z);
  const float4 rbin = tb.rb[ir];
  const float2 abin = tb.ab[ia];
  const float r = fmaf(ur, rbin.y, rbin.x);
  const float ap = fmaf(ua, abin.y, abin.x);  // alpha - pi
  float sn, cs;
  __sincosf(ap, &sn, &cs);
  const float de = (r * -cs) * T.s_eta;
  const float dp = (r * -sn) * T.s_phi;
  const float eta = T.eta_c + de;
  const float phi = T.phi_c + dp;
  // the bounds r_hi |s| 2^-17 + |x| 2^-21 of the FP32 eta and phi
  const float be = fmaf(rbin.w, fabsf(T.s_eta), fabsf(eta) * 0x1p-21f);
  const float bp = fmaf(rbin.w, fabsf(T.s_phi), fabsf(phi) * 0x1p-21f);
  bool sure = fabsf(eta) < 1.0e30f;  // false for NaN or huge eta (a NaN phi fails its own test below)
  // region: the last of the task's reachable regions [rb, re) whose split lies
  // at or below eta.  Most tasks reach one region or two (one split, tested
  // without a branch); a loop takes the further splits.
  const int rb = (T.lay >> 8) & 0xFFF, re = T.lay >> 20;
  const bool two = re > rb + 1;
  const float sp1 = tb.split[min(rb + 1, kMaxRegions - 1)];  // read by every lane, used where two
  int rr = (two && eta >= sp1) ? rb + 1 : rb;
  sure &= !two || fabsf(eta - sp1) > fmaf(fabsf(sp1), 0x1p-23f, be);
  if (re > rb + 2) {
    for (int q = rb + 2; q < re; ++q) {
      const float sp = tb.split[q];
      if (eta >= sp) rr = q;
      sure &= fabsf(eta - sp) > fmaf(fabsf(sp), 0x1p-23f, be);
    }
  }
  const RegionF R = tb.reg[rr];
  // eta index, clamped to [1/2, n_eta - 1/2]: outside it the cell is the first
  // or the last whichever side of the region's edge the hit lies, and at the
  // clamp the distance to the nearest integer is 1/2, so only interior cell
  // edges are certified
  const float te = fminf(fmaxf(fmaf(eta, R.inv_deta, R.ek), 0.5f), R.n_eta_hf);
  const float ke = rintf(te);
  sure &= fabsf(te - ke) > fmaf(te, 0x1p-21f, fmaf(be, R.inv_deta, R.ce));
  const int ie = (int)te;  // te >= 1/2: truncation is the floor
  const float tp = fmaf(phi, R.inv_dphi, R.pk);
  const float kp = rintf(tp);
  sure &= fabsf(tp - kp) > fmaf(fabsf(tp), 0x1p-21f, fmaf(bp, R.inv_dphi, R.cp));
  int ip = (int)floorf(tp);
  if (ip < 0) ip += R.n_phi;
  else if (ip >= R.n_phi) ip -= R.n_phi;
  if ((unsigned)ip >= (unsigned)R.n_phi) {  // more than one turn in phi: rare
    ip %= R.n_phi;
    if (ip < 0) ip += R.n_phi;
  }
  FastHit f;
  f.cell = R.cell_off + ie * R.n_phi + ip;
  f.sure = sure;
  return f;
}

// ---- warp-level deposit / record emission -----------------------------------
// Deterministic mode: the first lane of each group of equal (cell, task) keys
// in the warp writes the group's record (count - 1 in the low bits) and counts
// it in the cell's uint32 counter (the accumulation row).  A warp writes its
// records contiguously into chunks of kRecordChunk slots that it takes from
// the range's slot counter (a round that does not fit continues in the next
// chunk) and fills the rest of its last chunk with the empty record (all ones)
// when it ends, so the slots handed out hold every record and a few empty
// ones.  Uncertain hits are left to the recheck kernel.  Returns the warp's
// number of records (the caller counts them per CTA: one counter hit by every
// warp would serialise).
struct RecordChunk {
  int64_t base = 0;
  int fill = kRecordChunk;  // no chunk yet
};

__device__ __forceinline__ unsigned emit_records(bool ok, unsigned long long gkey, uint32_t cell, RecordChunk& ch,
                                                 const WsDev& w) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, ok);
  unsigned peers = 0;
  if (ok) peers = __match_any_sync(m, gkey);
  const bool lead = ok && (lane == __ffs(peers) - 1);
  const unsigned lm = __ballot_sync(0xffffffffu, lead);
  const int cnt = __popc(lm);
  if (cnt == 0) return 0u;
  const bool spill = ch.fill + cnt > kRecordChunk;
  unsigned long long nbase = 0;
  if (spill) {
    if (lane == 0) nbase = atomicAdd((unsigned long long*)&w.sizes->n_slots, (unsigned long long)kRecordChunk);
    nbase = __shfl_sync(0xffffffffu, nbase, 0);
  }
  if (lead) {
    const int pos = ch.fill + __popc(lm & ((1u << lane) - 1u));
    const int64_t slot = pos < kRecordChunk ? ch.base + pos : (int64_t)nbase + (pos - kRecordChunk);
    if (slot < w.rec_cap) {
      w.keys[slot] = (gkey << kRecordCountBits) | (unsigned long long)(__popc(peers) - 1);
      atomicAdd(reinterpret_cast<uint32_t*>(w.acc) + cell, 1u);
    } else {
      atomicOr(&w.sizes->flags, (uint32_t)FCS_FLAG_HIT_CAPACITY);
    }
  }
  if (spill) {
    ch.base = (int64_t)nbase;
    ch.fill += cnt - kRecordChunk;
  } else {
    ch.fill += cnt;
  }
  return (unsigned)cnt;
}

// The empty records after a warp's last one in its chunk.
__device__ __forceinline__ void close_records(const RecordChunk& ch, const WsDev& w) {
  for (int j = ch.fill + (threadIdx.x & 31); j < kRecordChunk; j += 32)
    if (ch.base + j < w.rec_cap) w.keys[ch.base + j] = ~0ull;
}

// Sum of v over each group of lanes with equal keys, added by the group's
// first lane to grad_acc[key] in FP64 (key = entry * 128 + bin).  s_v: this
// warp's 32 floats of shared memory; groups sum in ascending lane order.
__device__ __forceinline__ void grad_warp(bool ok, uint32_t key, float v, float* s_v, const HitKParams& kp) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, ok);
  s_v[lane] = v;
  __syncwarp();
  if (ok) {
    const unsigned peers = __match_any_sync(m, key);
    if (lane == __ffs(peers) - 1) {
      float sum = 0.0f;
      for (unsigned q = peers; q; q &= q - 1) sum += s_v[__ffs(q) - 1];
      atomicAdd(kp.grad_acc + key, (double)sum);
      kp.grad_touched[key >> 7] = 1;
    }
  }
  __syncwarp();
}

__device__ __forceinline__ void deposit_single(const HitKParams& kp, int32_t event, float Ehit, int64_t task_rel,
                                               int32_t cell, int mode, int32_t entry, int bin) {
  const int64_t row = event - kp.ev_lo;
  if (mode == kModeAtomic) {
    acc_add(kp.w.acc + row * kp.g.acc_stride + cell, Ehit);
  } else if (mode == kModeGrad) {
    const float v = __fmul_rn(Ehit, __ldg(kp.grad_in + row * kp.g.n_cells + cell));
    atomicAdd(kp.grad_acc + ((int64_t)entry << 7) + bin, (double)v);
    kp.grad_touched[entry] = 1;
  } else {
    const uint32_t c = (uint32_t)(row * kp.g.acc_stride + cell);
    const unsigned long long gkey = ((unsigned long long)c << kp.key_task_bits) | (unsigned long long)task_rel;
    const int64_t slot = (int64_t)atomicAdd((unsigned long long*)&kp.w.sizes->n_slots, 1ull);  // a slot of its own
    if (slot < kp.w.rec_cap) {
      atomicAdd((unsigned long long*)&kp.w.sizes->n_records, 1ull);
      kp.w.keys[slot] = gkey << kRecordCountBits;
      atomicAdd(reinterpret_cast<uint32_t*>(kp.w.acc) + c, 1u);
    } else {
      atomicOr(&kp.w.sizes->flags, (uint32_t)FCS_FLAG_HIT_CAPACITY);
    }
  }
}

// ---- block max-scan of the tile's task-start marks ------------------------------
template <int BLOCK, int HPT>
__device__ __forceinline__ void owner_scan(int16_t* s_owner, int* s_wmax) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int v[HPT];
  int run = 0;
#pragma unroll
  for (int k = 0; k < HPT; ++k) {
    run = max(run, (int)s_owner[tid * HPT + k]);
    v[k] = run;
  }
  int x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x = max(x, y);
  }
  if (lane == 31) s_wmax[warp] = x;
  __syncthreads();
  int prefix = 0;
  for (int w = 0; w < warp; ++w) prefix = max(prefix, s_wmax[w]);
  int excl = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane == 0) excl = 0;
  excl = max(excl, prefix);
#pragma unroll
  for (int k = 0; k < HPT; ++k) s_owner[tid * HPT + k] = (int16_t)max(v[k], excl);
}

// The uncertain hits of a warp step (need set, m = their ballot, non-zero):
// queued for the FP64 recheck kernel as (task, hit in task); when the queue is
// full the hit's cell is decided here in FP64, as the recheck kernel would.
// Called by the whole warp; out of line, as it runs for well under one warp
// step in a hundred.
template <int MODE, bool DBG>
static __device__ __noinline__ void queue_uncertain(const HitKParams& kp, bool need, unsigned m, int64_t task,
                                                    uint32_t hit, int32_t layer, float eta_c, float phi_c, uint4 x,
                                                    int bin, int32_t ev, float Ehit, int32_t entry, int64_t dbg_h) {
  const WsDev& w = kp.w;
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  const int l0 = __ffs(m) - 1;
  if (lane == l0) base = atomicAdd((unsigned long long*)&w.sizes->n_recheck, (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, l0);
  if (!need) return;
  const unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
  if (pos < (unsigned long long)w.recheck_cap) {
    w.recheck[pos] = make_uint2((uint32_t)task, hit);
    return;
  }
  const int32_t c = cell_fp64(kp.g, kp.p, layer, eta_c, phi_c, x, bin);
  deposit_single(kp, ev, Ehit, task, c, MODE, entry, bin);
  atomicAdd((unsigned long long*)&w.sizes->n_inline, 1ull);
  atomicOr(&w.sizes->flags, (uint32_t)FCS_FLAG_RECHECK_SPILL);
  if (DBG && kp.dbg_hit_cell && dbg_h < kp.dbg_hit_cap) kp.dbg_hit_cell[dbg_h] = c;
}

// Atomic mode asks for 10 CTAs of 128 threads per SM (48 registers): the
// extra warps hide the guide-table loads; the other modes keep the
// compiler's choice (a minimum of 0 CTAs is no constraint).  DBG: the
// validation dumps of fcs_debug (a separate instantiation, so that the
// production kernel carries none of their code).
template <int BLOCK, int HPT, int MODE, bool DBG>
__global__ void __launch_bounds__(BLOCK, MODE == kModeAtomic ? 1280 / BLOCK : 0) k_hits(const __grid_constant__ HitKParams kp) {
  constexpr bool DET = MODE == kModeDet;
  constexpr int TILE = BLOCK * HPT;
  static_assert(TILE % kGranule == 0, "queue tiles must start on granules (the tile map's unit)");
  static_assert(TILE <= 4096, "owner index and 32-bit match keys need TILE + 1 < 2^13");
  __shared__ HitSmemTables tb;
  __shared__ __align__(16) TileTask s_task[kSmemTasks];
  __shared__ int16_t s_owner[TILE];
  __shared__ int s_wmax[BLOCK / 32];
  __shared__ uint32_t s_tile;
  __shared__ float s_gv[MODE == kModeGrad ? BLOCK : 1];
  __shared__ unsigned long long s_recs;  // deterministic mode: records of this CTA
  load_tables(tb, kp.g, kp.p);
  for (int i = threadIdx.x; i < TILE; i += BLOCK) s_owner[i] = 0;
  const WsDev& w = kp.w;
  const int64_t H = kp.static_tiles ? kp.h_hi : w.sizes->n_hits;
  const int64_t T_last = kp.static_tiles ? (int64_t)kp.t_last : w.sizes->n_tasks - 1;
  const int64_t hbase = kp.static_tiles ? kp.h_lo : 0;
  if (H > w.gmap_cap * (int64_t)kGranule) {  // the tile map is too small for the hits
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&w.sizes->flags, (uint32_t)FCS_FLAG_HIT_CAPACITY);
    return;
  }
  const uint32_t n_tiles = (uint32_t)((H - hbase + TILE - 1) / TILE);  // < 2^32: hits < 2^39
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lanes_below = (1u << lane) - 1u;
  const int64_t hit_dbg_base = DBG ? w.sizes->hit_base : 0;
  // accumulation rows (atomic, deterministic) or dL/dE_cell rows (gradient)
  const uint32_t row_stride = MODE == kModeGrad ? (uint32_t)kp.g.n_cells : (uint32_t)kp.g.acc_stride;
  if (threadIdx.x == 0) {
    s_tile = kp.static_tiles ? blockIdx.x : (uint32_t)atomicAdd(&w.sizes->queue, 1ull);
    s_recs = 0;
  }
  __syncthreads();
  uint32_t tile = s_tile;
  unsigned long long recs = 0;  // deterministic mode: this warp's records
  RecordChunk chunk;            //   and the slots it writes them to
  while (tile < n_tiles) {
    __syncthreads();  // everyone has read s_tile; s_owner is zero again
    if (threadIdx.x == 0) s_tile = kp.static_tiles ? n_tiles : (uint32_t)atomicAdd(&w.sizes->queue, 1ull);
    const int64_t h0 = hbase + (int64_t)tile * TILE;
    const int hn = (int)min((int64_t)TILE, H - h0);  // hits in this tile
    const int32_t t0 = kp.static_tiles ? kp.t_last : w.gmap[h0 / kGranule];
    const int32_t t1 = (h0 + TILE < H && !kp.static_tiles) ? w.gmap[(h0 + TILE) / kGranule] : (int32_t)T_last;
    const int nt = t1 - t0 + 1;
    // (deterministic mode: the tile that holds a task's first hit writes the
    // task's hit energy for the fold)
    if (nt <= kSmemTasks) {
      // stage the tile's tasks and mark where each starts
      for (int j = threadIdx.x; j < nt; j += BLOCK) {
        const TileTask q = make_tile_task(tb, w, t0 + j, h0, kp.first_event_lo, kp.ev_lo, row_stride);
        const int64_t s = q.rel;
        s_task[j] = q;
        if (j > 0 && s < TILE) s_owner[s] = (int16_t)j;
        if constexpr (DET) {
          if (s >= 0 && s < TILE) w.tehit[t0 + j] = q.Ehit;
        }
      }
    } else {
      for (int j = threadIdx.x; j < nt; j += BLOCK) {
        const int64_t s = w.th[t0 + j] - h0;
        if (j > 0 && s < TILE) s_owner[s] = (int16_t)j;
        if constexpr (DET) {
          if (s >= 0 && s < TILE) w.tehit[t0 + j] = __fdiv_rn(w.tasks[t0 + j].El, (float)w.tn[t0 + j]);
        }
      }
    }
    __syncthreads();
    owner_scan<BLOCK, HPT>(s_owner, s_wmax);
    __syncthreads();
    // the hit loop, compiled once for staged tiles (the common case) and once
    // for tiles with more tasks than the shared copy holds
    auto hit_loop = [&](auto staged) {
#pragma unroll 1
      for (int k = 0; k < HPT; ++k) {
        const int i = warp * 32 * HPT + k * 32 + lane;
        const bool valid = i < hn;
        const int tl = valid ? s_owner[i] : 0;
        TileTask T;
        if constexpr (decltype(staged)::value) {
          T = s_task[tl];
        } else {  // more tasks than the shared copy holds: read the record itself
          T = make_tile_task(tb, w, t0 + tl, h0, kp.first_event_lo, kp.ev_lo, row_stride);
        }
        const uint32_t hit = (uint32_t)(i - T.rel);
        // the round keys come from the kernel parameters
        const uint4 x = philox4x32_10_rk(make_uint4(hit, T.ctr_y, T.ctr_z, T.ctr_w), kp.rk);
        const int bin = sample_bin(kp.p, T.entry, x.x);
        const FastHit f = fast_cell(tb, T, x, bin);
        const bool ok = valid && f.sure;
        const bool need = valid && !f.sure;
        if constexpr (MODE == kModeGrad) {
          // dL/dE_cell of the hit's cell times its energy, summed per (entry, bin)
          const float v = ok ? __fmul_rn(T.Ehit, __ldg(kp.grad_in + T.row_off + f.cell)) : 0.0f;
          grad_warp(ok, ((uint32_t)T.entry << 7) | (uint32_t)bin, v, s_gv + warp * 32, kp);
        } else if constexpr (!DET) {
          // (cell, task-in-tile) identifies (address, hit energy): 19 + 13 bits
          const unsigned m = __ballot_sync(0xffffffffu, ok);
          if (ok) {
            const unsigned peers = kp.key32 ? __match_any_sync(m, ((uint32_t)f.cell << 13) | (uint32_t)tl)
                                            : __match_any_sync(m, ((unsigned long long)(uint32_t)tl << 32) |
                                                                      (uint32_t)f.cell);
            if ((peers & lanes_below) == 0u)  // the group's first lane deposits
              acc_add(w.acc + T.row_off + f.cell, __fmul_rn((float)__popc(peers), T.Ehit));
          }
        } else {
          const uint32_t cg = T.row_off + (uint32_t)f.cell;
          const unsigned long long gkey = ((unsigned long long)cg << kp.key_task_bits) | (unsigned long long)(t0 + tl);
          recs += emit_records(ok, gkey, cg, chunk, w);
        }
        // queue the uncertain hits for the FP64 recheck
        const unsigned m = __ballot_sync(0xffffffffu, need);
        if (m)
          queue_uncertain<MODE, DBG>(kp, need, m, t0 + tl, hit, (int32_t)(T.lay & 0xFF), T.eta_c, T.phi_c, x, bin,
                                     (int32_t)(T.ctr_w - kp.first_event_lo), T.Ehit, T.entry, hit_dbg_base + h0 + i);
        if constexpr (DBG) {
          const int64_t h = hit_dbg_base + h0 + i;
          if (valid && h < kp.dbg_hit_cap) {
            if (kp.dbg_hit_cell && f.sure) kp.dbg_hit_cell[h] = f.cell;
            if (kp.dbg_hit_bin) kp.dbg_hit_bin[h] = (int16_t)bin;
          }
        }
        s_owner[i] = 0;  // ready for the next tile (each slot is read and reset by one thread)
      }
    };
    if (nt <= kSmemTasks) hit_loop(std::true_type{});
    else hit_loop(std::false_type{});
    __syncthreads();  // the tile's shared data is dead; s_tile holds the next tile
    tile = s_tile;
  }
  if constexpr (DET) {
    close_records(chunk, w);
    if (lane == 0 && recs) atomicAdd(&s_recs, recs);
    __syncthreads();
    if (threadIdx.x == 0 && s_recs) atomicAdd((unsigned long long*)&w.sizes->n_records, s_recs);
  }
}

// FP64 recheck of the queued hits (grid-stride over the queue).
template <int MODE>
__global__ void __launch_bounds__(128) k_recheck(const __grid_constant__ HitKParams kp) {
  const WsDev& w = kp.w;
  const int64_t n = min(w.sizes->n_recheck, w.recheck_cap);
  const int64_t hit_dbg_base = kp.dbg_hit_cell ? w.sizes->hit_base : 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint2 q = w.recheck[i];
    const TaskRec T = w.tasks[q.x];
    const int32_t layer = T.layer(), event = T.event();
    const int64_t hb = w.th[q.x];
    const uint4 x = philox4x32_10(
        make_uint4(q.y, (uint32_t)layer | (kPurposeHit << 16), (uint32_t)T.particle, kp.first_event_lo + (uint32_t)event),
        kp.k0, kp.k1);
    const int bin = sample_bin(kp.p, T.entry, x.x);
    const int32_t c = cell_fp64(kp.g, kp.p, layer, T.eta_c, T.phi_c, x, bin);
    deposit_single(kp, event, __fdiv_rn(T.El, (float)w.tn[q.x]), q.x, c, MODE, T.entry, bin);
    const int64_t h = hit_dbg_base + hb + q.y;
    if (kp.dbg_hit_cell && h < kp.dbg_hit_cap) kp.dbg_hit_cell[h] = c;
  }
}

template <int MODE>
cudaError_t launch_hits_t(const HitKParams& kp, const HitCfg& hc, const Launch& L);

}  // namespace fcs
