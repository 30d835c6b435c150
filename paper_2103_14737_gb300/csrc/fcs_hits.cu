// fcs_hits.cu - atomic-mode instantiations of the hit and recheck kernels and
// the launchers used by the API layer.
#include "fcs_hits_impl.cuh"

namespace fcs {

template cudaError_t launch_hits_t<kModeAtomic>(const HitKParams&, const HitCfg&, const Launch&);
template cudaError_t launch_recheck_t<kModeAtomic>(const HitKParams&, const Launch&);
extern template cudaError_t launch_hits_t<kModeDet>(const HitKParams&, const HitCfg&, const Launch&);
extern template cudaError_t launch_recheck_t<kModeDet>(const HitKParams&, const Launch&);

cudaError_t launch_hits(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0,
                        uint32_t k1, int64_t first_event, const HitCfg& hc, int key_task_bits,
                        const fcs_debug* dbg, const Launch& L) {
  const HitKParams kp = make_hit_params(g, p, w, ev_lo, k0, k1, first_event, key_task_bits, dbg);
  return hc.det ? launch_hits_t<kModeDet>(kp, hc, L) : launch_hits_t<kModeAtomic>(kp, hc, L);
}

cudaError_t launch_hits_task(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0, uint32_t k1,
                             int64_t first_event, const HitCfg& hc, int key_task_bits, const fcs_debug* dbg,
                             int64_t h_lo, int64_t h_hi, int32_t task, const Launch& L) {
  HitKParams kp = make_hit_params(g, p, w, ev_lo, k0, k1, first_event, key_task_bits, dbg);
  kp.static_tiles = 1;
  kp.h_lo = h_lo;
  kp.h_hi = h_hi;
  kp.t_last = task;
  return hc.det ? launch_hits_t<kModeDet>(kp, hc, L) : launch_hits_t<kModeAtomic>(kp, hc, L);
}

cudaError_t launch_recheck(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0,
                           uint32_t k1, int64_t first_event, int det, int key_task_bits,
                           const fcs_debug* dbg, const Launch& L) {
  const HitKParams kp = make_hit_params(g, p, w, ev_lo, k0, k1, first_event, key_task_bits, dbg);
  return det ? launch_recheck_t<kModeDet>(kp, L) : launch_recheck_t<kModeAtomic>(kp, L);
}

int hits_max_smem_tasks() { return kSmemTasks; }

}  // namespace fcs
