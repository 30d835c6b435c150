// fcs_hits_impl.cuh - launch dispatch of the hit kernel over the tuned
// (threads per block, hits per thread) shapes; included by the atomic-mode and
// deterministic-mode translation units.
#pragma once

#include "fcs_hits.cuh"

namespace fcs {

template <int BLOCK, int HPT, bool DET>
static cudaError_t launch_hits_shape(const HitKParams& kp, const Launch& L) {
  static int occ = -1;  // resident CTAs per SM of this instantiation
  if (occ < 0) {
    int o = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_hits<BLOCK, HPT, DET>, BLOCK, 0);
    if (e != cudaSuccess) return e;
    occ = o < 1 ? 1 : o;
  }
  k_hits<BLOCK, HPT, DET><<<L.num_sms * occ, BLOCK, 0, L.s>>>(kp);
  return cudaGetLastError();
}

template <bool DET>
cudaError_t launch_hits_t(const HitKParams& kp, const HitCfg& hc, const Launch& L) {
#define FCS_HIT_CASE(B, H) \
  if (hc.block == B && hc.hpt == H) return launch_hits_shape<B, H, DET>(kp, L);
  FCS_HIT_CASE(128, 1) FCS_HIT_CASE(128, 2) FCS_HIT_CASE(128, 4) FCS_HIT_CASE(128, 8)
  FCS_HIT_CASE(256, 1) FCS_HIT_CASE(256, 2) FCS_HIT_CASE(256, 4) FCS_HIT_CASE(256, 8)
  FCS_HIT_CASE(512, 1) FCS_HIT_CASE(512, 2) FCS_HIT_CASE(512, 4) FCS_HIT_CASE(512, 8)
#undef FCS_HIT_CASE
  return cudaErrorInvalidValue;
}

template <bool DET>
cudaError_t launch_recheck_t(const HitKParams& kp, const Launch& L) {
  k_recheck<DET><<<L.num_sms * 2, 128, 0, L.s>>>(kp);
  return cudaGetLastError();
}

}  // namespace fcs
