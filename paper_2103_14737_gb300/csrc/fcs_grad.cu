// fcs_grad.cu - the adjoint of the hit loop: gradients of a loss of the cell
// energies with respect to the layer fractions and the shape weights.
//
// With the seed fixed the parametrisation's hits keep their task, count n,
// shape bin b and cell; a change of the parameters changes only the hit
// energies (the energy of a hit is E_l / n with E_l = E f_l, Sec. 4).  The
// layer fraction enters linearly, dE_hit / df = E / n; the shape weights enter
// through the likelihood ratio p_b(w) / p_b(w0) of the bin the hit was drawn
// from, p_b = w_b / W with W the sum of the entry's weights.  With
// A[e][b] = sum over entry e's hits in bin b of E_hit dL/dE_cell(hit):
//   dL/df[e]    = sum_b A[e][b] / f_e
//   dL/dw[e][b] = A[e][b] / w_b - sum_j A[e][j] / W     (A / w := 0 where w_b = 0)
// The hit kernel in gradient mode regenerates every hit (Philox, bin, cell,
// FP64 recheck of uncertain cells) exactly as the forward pass does, gathers
// dL/dE_cell, sums E_hit dL/dE_cell per (entry, bin) over each warp's hits
// and adds the sums to A in FP64; the finalize kernel turns A into the two
// gradients for the entries that received hits and clears A for the next call.
#include "fcs_hits_impl.cuh"

namespace fcs {

template cudaError_t launch_hits_t<kModeGrad>(const HitKParams&, const HitCfg&, const Launch&);
template cudaError_t launch_recheck_t<kModeGrad>(const HitKParams&, const Launch&);

namespace {

// One warp per entry; lane j holds bins j, j + 32, j + 64, j + 96.
__global__ void __launch_bounds__(256) k_grad_finalize(int32_t n_entries, double* __restrict__ acc,
                                                       uint8_t* __restrict__ touched,
                                                       const float* __restrict__ frac,
                                                       const float* __restrict__ shape_w,
                                                       float* __restrict__ d_frac, float* __restrict__ d_w) {
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= n_entries) return;
  if (!touched[e]) return;  // warp-uniform
  double a[4], w[4];
  double S = 0.0, W = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    a[j] = acc[e * kNBins + lane + 32 * j];
    w[j] = (double)shape_w[e * kNBins + lane + 32 * j];
    S += a[j];
    W += w[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    S += __shfl_xor_sync(0xffffffffu, S, o);
    W += __shfl_xor_sync(0xffffffffu, W, o);
  }
  const double SW = S / W;
  if (d_w) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const double g = (w[j] > 0.0 ? a[j] / w[j] : 0.0) - SW;
      d_w[e * kNBins + lane + 32 * j] += (float)g;
    }
  }
  if (d_frac && lane == 0) {
    const double f = (double)frac[e];
    if (f > 0.0) d_frac[e] += (float)(S / f);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) acc[e * kNBins + lane + 32 * j] = 0.0;
  __syncwarp();
  if (lane == 0) touched[e] = 0;
}

// Validation of a device-resident parametrisation (the host checks of
// fcs_load_params): bit 0 a fraction that is negative or not finite, bit 1 a
// mean hit energy that is not > 0 where the fraction is > 0, bit 2 a weight
// that is negative or not finite, bit 3 an entry with fraction > 0 whose
// weights sum to 0.  One warp per entry.
__global__ void __launch_bounds__(256) k_check_params(const float* __restrict__ frac,
                                                      const float* __restrict__ mhe,
                                                      const float* __restrict__ shape_w, int32_t n_entries,
                                                      uint32_t* __restrict__ bad) {
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= n_entries) return;
  uint32_t flags = 0;
  float any = 0.0f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float w = shape_w[e * kNBins + lane + 32 * j];
    if (!(w >= 0.0f) || !isfinite(w)) flags |= 4u;
    else any = fmaxf(any, w);
  }
  flags = __reduce_or_sync(0xffffffffu, flags);
  const bool has_weight = __any_sync(0xffffffffu, any > 0.0f);
  if (lane != 0) return;
  const float f = frac[e];
  if (!(f >= 0.0f) || !isfinite(f)) flags |= 1u;
  if (f > 0.0f) {
    const float m = mhe[e];
    if (!(m > 0.0f) || !isfinite(m)) flags |= 2u;
    if (!has_weight) flags |= 8u;
  }
  if (flags) atomicOr(bad, flags);
}

}  // namespace

cudaError_t launch_hits_grad(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0,
                             uint32_t k1, int64_t first_event, const HitCfg& hc, const float* grad_in,
                             double* grad_acc, uint8_t* touched, const Launch& L) {
  HitKParams kp = make_hit_params(g, p, w, ev_lo, k0, k1, first_event, 0, nullptr);
  kp.grad_in = grad_in;
  kp.grad_acc = grad_acc;
  kp.grad_touched = touched;
  return launch_hits_t<kModeGrad>(kp, hc, L);
}

cudaError_t launch_recheck_grad(const GeoDev& g, const ParamDev& p, WsDev w, int32_t ev_lo, uint32_t k0,
                                uint32_t k1, int64_t first_event, const float* grad_in, double* grad_acc,
                                uint8_t* touched, const Launch& L) {
  HitKParams kp = make_hit_params(g, p, w, ev_lo, k0, k1, first_event, 0, nullptr);
  kp.grad_in = grad_in;
  kp.grad_acc = grad_acc;
  kp.grad_touched = touched;
  return launch_recheck_t<kModeGrad>(kp, L);
}

cudaError_t launch_grad_finalize(const ParamDev& p, double* grad_acc, uint8_t* touched, float* d_frac,
                                 float* d_shape_w, const Launch& L) {
  const int64_t threads = (int64_t)p.n_entries * 32;
  if (threads == 0) return cudaSuccess;
  k_grad_finalize<<<(unsigned)((threads + 255) / 256), 256, 0, L.s>>>(p.n_entries, grad_acc, touched, p.frac,
                                                                       p.shape_w, d_frac, d_shape_w);
  return cudaGetLastError();
}

cudaError_t launch_check_params(const float* frac, const float* mean_hit_E, const float* shape_w,
                                int n_entries, uint32_t* bad, cudaStream_t s) {
  const int64_t threads = (int64_t)n_entries * 32;
  if (threads == 0) return cudaSuccess;
  k_check_params<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(frac, mean_hit_E, shape_w, n_entries, bad);
  return cudaGetLastError();
}

}  // namespace fcs
