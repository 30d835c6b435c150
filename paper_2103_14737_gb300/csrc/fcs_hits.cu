// fcs_hits.cu - atomic-mode instantiations of the hit and recheck kernels and
// the launchers used by the API layer.
#include "fcs_hits_impl.cuh"

namespace fcs {

template cudaError_t launch_hits_t<false>(const HitKParams&, const HitCfg&, const Launch&);
template cudaError_t launch_recheck_t<false>(const HitKParams&, const Launch&);
extern template cudaError_t launch_hits_t<true>(const HitKParams&, const HitCfg&, const Launch&);
extern template cudaError_t launch_recheck_t<true>(const HitKParams&, const Launch&);

static HitKParams make_params(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0,
                              uint32_t k1, int64_t first_event, int key_task_bits,
                              const fcs_debug* dbg) {
  HitKParams kp;
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
  return kp;
}

cudaError_t launch_hits(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0,
                        uint32_t k1, int64_t first_event, const HitCfg& hc, int key_task_bits,
                        const fcs_debug* dbg, const Launch& L) {
  const HitKParams kp = make_params(g, p, w, ev_lo, k0, k1, first_event, key_task_bits, dbg);
  return hc.det ? launch_hits_t<true>(kp, hc, L) : launch_hits_t<false>(kp, hc, L);
}

cudaError_t launch_recheck(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0,
                           uint32_t k1, int64_t first_event, int det, int key_task_bits,
                           const fcs_debug* dbg, const Launch& L) {
  const HitKParams kp = make_params(g, p, w, ev_lo, k0, k1, first_event, key_task_bits, dbg);
  return det ? launch_recheck_t<true>(kp, L) : launch_recheck_t<false>(kp, L);
}

int hits_max_smem_tasks() { return kSmemTasks; }

}  // namespace fcs
