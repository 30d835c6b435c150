// fcs_hits_det.cu - deterministic-mode (record-emitting) instantiations of
// the hit and recheck kernels.
#include "fcs_hits_impl.cuh"

namespace fcs {
template cudaError_t launch_hits_t<kModeDet>(const HitKParams&, const HitCfg&, const Launch&);
template cudaError_t launch_recheck_t<kModeDet>(const HitKParams&, const Launch&);
}  // namespace fcs
