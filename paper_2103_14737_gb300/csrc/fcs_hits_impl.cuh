// fcs_hits_impl.cuh - launch dispatch of the hit kernel over the tuned
// (threads per block, hits per thread) shapes; included by the atomic-mode,
// deterministic-mode and gradient-mode translation units.
#pragma once

#include "fcs_hits.cuh"

namespace fcs {

static inline HitKParams make_hit_params(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0,
                                         uint32_t k1, int64_t first_event, int key_task_bits,
                                         const fcs_debug* dbg) {
  HitKParams kp{};
  kp.g = g;
  kp.p = p;
  kp.w = w;
  kp.ev_lo = ev_lo;
  kp.k0 = k0;
  kp.k1 = k1;
  kp.first_event_lo = (uint32_t)first_event;
  kp.key_task_bits = key_task_bits;
  kp.key32 = g.n_cells < (1 << 19) ? 1 : 0;
  kp.dbg_hit_cell = dbg ? dbg->hit_cell : nullptr;
  kp.dbg_hit_bin = dbg ? dbg->hit_bin : nullptr;
  kp.dbg_hit_cap = dbg ? dbg->hit_capacity : 0;
  kp.rk = philox_round_keys(k0, k1);
  return kp;
}

template <int BLOCK, int HPT, int MODE, bool DBG>
static cudaError_t launch_hits_kernel(const HitKParams& kp, const Launch& L) {
  static int occ = -1;  // resident CTAs per SM of this instantiation
  if (occ < 0) {
    int o = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_hits<BLOCK, HPT, MODE, DBG>, BLOCK, 0);
    if (e != cudaSuccess) return e;
    occ = o < 1 ? 1 : o;
  }
  int64_t grid = (int64_t)L.num_sms * occ;
  if (kp.static_tiles) {
    constexpr int64_t TILE = (int64_t)BLOCK * HPT;
    grid = (kp.h_hi - kp.h_lo + TILE - 1) / TILE;
    if (grid <= 0) return cudaSuccess;
  }
  k_hits<BLOCK, HPT, MODE, DBG><<<(unsigned)grid, BLOCK, 0, L.s>>>(kp);
  return cudaGetLastError();
}

// The validation dumps run in their own instantiation (no gradient-mode dumps).
template <int BLOCK, int HPT, int MODE>
static cudaError_t launch_hits_shape(const HitKParams& kp, const Launch& L) {
  if constexpr (MODE != kModeGrad) {
    if (kp.dbg_hit_cell || kp.dbg_hit_bin) return launch_hits_kernel<BLOCK, HPT, MODE, true>(kp, L);
  }
  return launch_hits_kernel<BLOCK, HPT, MODE, false>(kp, L);
}

template <int MODE>
cudaError_t launch_hits_t(const HitKParams& kp, const HitCfg& hc, const Launch& L) {
#define FCS_HIT_CASE(B, H) \
  if (hc.block == B && hc.hpt == H) return launch_hits_shape<B, H, MODE>(kp, L);
  FCS_HIT_CASE(128, 1) FCS_HIT_CASE(128, 2) FCS_HIT_CASE(128, 4) FCS_HIT_CASE(128, 8)
  FCS_HIT_CASE(256, 1) FCS_HIT_CASE(256, 2) FCS_HIT_CASE(256, 4) FCS_HIT_CASE(256, 8)
  FCS_HIT_CASE(512, 1) FCS_HIT_CASE(512, 2) FCS_HIT_CASE(512, 4) FCS_HIT_CASE(512, 8)
#undef FCS_HIT_CASE
  return cudaErrorInvalidValue;
}

template <int MODE>
cudaError_t launch_recheck_t(const HitKParams& kp, const Launch& L) {
  // FP64 work: one warp per block spreads the queue over every SM's FP64 pipe
  k_recheck<MODE><<<L.num_sms * 8, 32, 0, L.s>>>(kp);
  return cudaGetLastError();
}

}  // namespace fcs
