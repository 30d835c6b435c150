// fcs_tasks.cu - task build of the hit loop (Listing 1): per particle the
// parametrisation entry and its layers with a non-zero float layer energy;
// per task the Poisson hit count (get_number_of_hits) and the float hit
// energy; task records in (event, particle, layer) order.  Flat per-task
// kernels keep the Poisson draws of a warp together.  (The hit-offset scan
// writes the tile -> task map; the task finish kernel here writes it again
// when a call grew the map after that scan.)
#include <algorithm>

#include <atomic>

#include "fcs_internal.cuh"

namespace fcs {
namespace {

// ---- Poisson draw (FP64; every step rounds as the oracle's C code) ----------
// mu < 10: inversion by sequential search from p0 = exp(-mu).  mu >= 10:
// PTRS, the transformed rejection with squeeze of Hoermann (1993).  Draw i of
// a task is Philox block (i, layer | 1 << 16, particle, event); its words give
// two 53-bit uniforms.  The bounds of both loops match the oracle.
constexpr int kInvMax = 200;
constexpr uint32_t kPtrsMaxIter = 64;

__device__ __forceinline__ void draw_pair(uint32_t i, uint32_t layer, uint32_t particle,
                                          uint32_t event, uint32_t k0, uint32_t k1, double* u,
                                          double* v) {
  const uint4 x = philox4x32_10(make_uint4(i, layer | (kPurposePoisson << 16), particle, event), k0, k1);
  *u = u53(x.x, x.y);
  *v = u53(x.z, x.w);
}

struct PtrsConst64 {
  double loglam, b, a, invalpha, vr;
};

__device__ __forceinline__ PtrsConst64 ptrs_const64(double mu) {
  PtrsConst64 c;
  const double slam = __dsqrt_rn(mu);
  c.loglam = log(mu);
  c.b = __dadd_rn(0.931, __dmul_rn(2.53, slam));
  c.a = __dadd_rn(-0.059, __dmul_rn(0.02483, c.b));
  c.invalpha = __dadd_rn(1.1239, __ddiv_rn(1.1328, __dsub_rn(c.b, 3.4)));
  c.vr = __dsub_rn(0.9277, __ddiv_rn(3.6224, __dsub_rn(c.b, 2.0)));
  return c;
}

// One PTRS iteration in FP64 from its two 53-bit uniforms: the accepted count,
// or -1 when the iteration rejects.  log k! = lgamma(k + 1) comes from the
// host's libm (the table), as in the C definition, for k below the table size.
__device__ __noinline__ int64_t ptrs_iter64(double mu, const PtrsConst64& c, double u, double V,
                                            const double* lfact64, int32_t n_lfact) {
  const double U = __dsub_rn(u, 0.5);
  const double us = __dsub_rn(0.5, fabs(U));
  if (us <= 0.0) return -1;
  const double t = __dadd_rn(__dadd_rn(__dmul_rn(__dadd_rn(__ddiv_rn(__dmul_rn(2.0, c.a), us), c.b), U), mu), 0.43);
  const double kd = floor(t);
  if (us >= 0.07 && V <= c.vr) return (int64_t)kd;
  if (kd < 0.0 || (us < 0.013 && V > us)) return -1;
  const double lhs = __dsub_rn(__dadd_rn(log(V), log(c.invalpha)),
                               log(__dadd_rn(__ddiv_rn(c.a, __dmul_rn(us, us)), c.b)));
  const double lg = (kd < (double)n_lfact) ? __ldg(lfact64 + (int32_t)kd) : lgamma(__dadd_rn(kd, 1.0));
  const double rhs = __dsub_rn(__dadd_rn(-mu, __dmul_rn(kd, c.loglam)), lg);
  return (lhs <= rhs) ? (int64_t)kd : -1;
}

// The whole draw in FP64 (the definition the fast path must reproduce).  A
// PTRS draw may start at iteration i0 when every earlier iteration is known
// to reject (the FP32 path certified those rejections).
__device__ __noinline__ int64_t poisson_draw(double mu, uint32_t layer, uint32_t particle, uint32_t event,
                                             uint32_t k0, uint32_t k1, const double* lfact64, int32_t n_lfact,
                                             uint32_t i0) {
  if (!(mu > 0.0)) return 0;
  if (mu < 10.0) {
    double u, v;
    draw_pair(0u, layer, particle, event, k0, k1, &u, &v);
    double p = exp(-mu);
    double F = p;
    int64_t k = 0;
    while (u >= F && k < kInvMax) {
      k += 1;
      p = __ddiv_rn(__dmul_rn(p, mu), (double)k);
      F = __dadd_rn(F, p);
    }
    return k;
  }
  const PtrsConst64 c = ptrs_const64(mu);
  for (uint32_t i = i0; i < kPtrsMaxIter; ++i) {
    double u, V;
    draw_pair(i, layer, particle, event, k0, k1, &u, &V);
    const int64_t k = ptrs_iter64(mu, c, u, V, lfact64, n_lfact);
    if (k >= 0) return k;
  }
  return (int64_t)floor(mu);
}

// ---- FP32 fast path of the same draw ------------------------------------------
// Every comparison of the FP64 definition is made in FP32 together with a
// bound on |FP32 value - exact value| (the FP64 values of the definition are
// within a few 2^-53 of exact, covered by the slack).  When the two sides are
// farther apart than the bound the FP32 decision is the FP64 one; otherwise
// the iteration (PTRS) or the whole inversion is redone in FP64.  Bounds:
//   inversion: expf <= 2 ulp, each of the k multiply/reciprocal steps adds
//     <= 3 roundings (2^-24 each) to p_k, each partial sum one more, so
//     |F32_k - F_k| <= 2^-22 + (4k + 1) 2^-24 (F <= 1); the 53-bit uniform
//     rounded to FP32 is off by <= 2^-24 and the difference u - F rounds once
//     more (<= 2^-25): (4k + 6.5) 2^-24 in all; used: 2^-21 (k + 2).
//   PTRS constants: sqrtf / logf, the FP32 images of the decimal constants
//     and __fdividef (<= 2 ulp for divisors in [2^-126, 2^126], as documented;
//     every divisor here is): a few roundings each, so b, a and 1/alpha are
//     within 2^-20 relative and v_r within 2^-21 absolute.  The quotients
//     2a/us and a/us^2 of an iteration are likewise within 2^-21 relative;
//     the bounds they feed allow 2^-18.
//   uniforms: exact integers rounded once to FP32 (relative 2^-24).
constexpr float kPtrsFastMaxMu = 4096.0f;  // larger means go to FP64 (counts of ~1e4 lose FP32 headroom)

struct PtrsConst32 {
  float loglam, b, a, invalpha, vr, two_a;
  const float* lfact;  // log k! table (|error| <= 0.5 ulp + libm's)
  int32_t n_lfact;
};

__device__ __forceinline__ PtrsConst32 ptrs_const32(float mu, const float* lfact, int32_t n_lfact) {
  PtrsConst32 c;
  c.lfact = lfact;
  c.n_lfact = n_lfact;
  const float slam = sqrtf(mu);
  c.loglam = logf(mu);
  c.b = fmaf(2.53f, slam, 0.931f);
  c.a = fmaf(0.02483f, c.b, -0.059f);
  c.invalpha = 1.1239f + __fdividef(1.1328f, c.b - 3.4f);
  c.vr = 0.9277f - __fdividef(3.6224f, c.b - 2.0f);
  c.two_a = 2.0f * c.a;
  return c;
}

// FP32 images of the 53-bit uniform u = N 2^-53, N = (a >> 5) 2^26 + (b >> 6),
// built from 32-bit integer conversions only (64-bit integer conversions run
// on the FP64 pipe).  Relative error <= 2^-23 each; where two terms of
// opposite sign could cancel, the difference is formed exactly in 32 bits.
__device__ __forceinline__ float u53f(uint32_t a, uint32_t b) {
  return fmaf((float)(b >> 6), 0x1p-53f, (float)(a >> 5) * 0x1p-27f);
}
__device__ __forceinline__ float u53f_minus_half(uint32_t a, uint32_t b) {  // u - 0.5
  const uint32_t hi = a >> 5, lo = b >> 6;
  if (hi >= (1u << 26)) return fmaf((float)lo, 0x1p-53f, (float)(hi - (1u << 26)) * 0x1p-27f);
  const uint32_t hd = (1u << 26) - hi;  // u - 0.5 = -(hd 2^26 - lo) 2^-53
  if (hd < 64u) return -(float)((hd << 26) - lo) * 0x1p-53f;
  return fmaf((float)lo, 0x1p-53f, -(float)hd * 0x1p-27f);
}
__device__ __forceinline__ float u53f_edge(uint32_t a, uint32_t b) {  // min(u, 1 - u)
  const uint32_t hi = a >> 5, lo = b >> 6;
  if (hi < (1u << 26)) return fmaf((float)lo, 0x1p-53f, (float)hi * 0x1p-27f);
  const uint32_t hp = (1u << 27) - hi;  // 1 - u = (hp 2^26 - lo) 2^-53
  if (hp < 64u) return (float)((hp << 26) - lo) * 0x1p-53f;
  return fmaf(-(float)lo, 0x1p-53f, (float)hp * 0x1p-27f);
}

// One PTRS iteration in FP32.  Returns the accepted count, -1 for a certain
// rejection, -2 when a decision is uncertain (redo the iteration in FP64).
__device__ __forceinline__ int64_t ptrs_iter32(float mu, const PtrsConst32& c, uint4 w) {
  if ((w.x >> 5) == 0 && (w.y >> 6) == 0) return -1;  // u == 0: us == 0 rejects
  const float Uf = u53f_minus_half(w.x, w.y);
  const float usf = u53f_edge(w.x, w.y);
  const float Vf = u53f(w.z, w.w);
  // k = floor((2a/us + b) U + mu + 0.43)
  const float t1 = __fdividef(c.two_a, usf);
  const float x = ((t1 + c.b) * Uf + mu) + 0.43f;
  const float bx = (fabsf(t1 * Uf) + fabsf(c.b * Uf)) * 0x1p-18f + (fabsf(x) + 1.0f) * 0x1p-22f;
  const float kf = floorf(x);
  const bool k_sure = (x - kf > bx) && (kf + 1.0f - x > bx);
  // quick accept: us >= 0.07 && V <= vr
  const float m_us = 0x1p-23f, m_v = 0x1p-19f;
  const bool us_ge_007 = usf - 0.07f > m_us, us_lt_007 = 0.07f - usf > m_us;
  const bool v_le_vr = c.vr - Vf > m_v, v_gt_vr = Vf - c.vr > m_v;
  if (us_ge_007 && v_le_vr) return k_sure ? (int64_t)(int32_t)kf : -2;
  if (!(us_lt_007 || v_gt_vr)) return -2;  // quick-accept decision uncertain
  // reject: k < 0 || (us < 0.013 && V > us)
  const bool k_neg = x + bx < 0.0f, k_nonneg = x - bx >= 0.0f;
  if (k_neg) return -1;
  if (!k_nonneg) return -2;
  const bool us_lt_0013 = 0.013f - usf > m_us, us_ge_0013 = usf - 0.013f > m_us;
  const float m_vu = (Vf + usf) * 0x1p-20f;
  const bool v_gt_us = Vf - usf > m_vu, v_le_us = usf - Vf > m_vu;
  if (us_lt_0013 && v_gt_us) return -1;
  if (!(us_ge_0013 || v_le_us)) return -2;
  // full test: log V + log invalpha - log(a / us^2 + b) <= -mu + k log mu - lgamma(k + 1)
  if (!k_sure) return -2;
  const float l1 = logf(Vf), l2 = logf(c.invalpha), l3 = logf(__fdividef(c.a, usf * usf) + c.b);
  const int32_t ki = (int32_t)kf;
  const float kl = kf * c.loglam, lg = (ki < c.n_lfact) ? __ldg(c.lfact + ki) : lgammaf(kf + 1.0f);
  const float d = (l1 + l2 - l3) - ((-mu + kl) - lg);
  const float bd = (fabsf(l1) + fabsf(l2) + fabsf(l3) + fabsf(kl) + fabsf(lg) + mu + 1.0f) * 0x1p-18f;
  if (d < -bd) return (int64_t)ki;
  if (d > bd) return -1;
  return -2;
}

// Poisson draw in FP32 where every decision is certified; where one is not,
// the caller takes poisson_draw, the FP64 definition, for the task.
//
// Inversion (mu < 10): the count, or -1 when a decision is uncertain.
// rcp[k] = __frcp_rn(k) for k <= kInvMax (a shared-memory copy: the values
// the loop would compute).
__device__ __forceinline__ int32_t poisson_inv_fp32(float mu32, uint32_t layer, uint32_t particle, uint32_t event,
                                                    const PhiloxRoundKeys& rk, const float* rcp) {
  if (!(mu32 > 0.0f)) return 0;
  const uint4 x = philox4x32_10_rk(make_uint4(0u, layer | (kPurposePoisson << 16), particle, event), rk);
  const float uf = u53f(x.x, x.y);
  float p = expf(-mu32);
  float F = p;
  float e = 0x1p-20f;  // (k + 2) 2^-21, exact in FP32 for k <= kInvMax
  float d = uf - F;
  int k = 0;
  while (d > e && k < kInvMax) {  // u > F_k for certain: the search goes on
    k += 1;
    e += 0x1p-21f;
    p = (p * mu32) * rcp[k];
    F = F + p;
    d = uf - F;
  }
  if (d < -e) return k;  // u < F_k for certain: stop at k
  if (d > e) return k;   // k == kInvMax: the definition stops here too
  return -1;             // uncertain
}

// PTRS (mu >= 10), iteration i alone: the accepted count, -1 when it rejects
// for certain (the draw continues at iteration i + 1), -2 when a decision is
// uncertain or mu is too large for FP32 headroom (the FP64 definition takes
// the draw from iteration i on).
__device__ __forceinline__ int32_t ptrs_step_fp32(float mu32, uint32_t layer, uint32_t particle, uint32_t event,
                                                  const PhiloxRoundKeys& rk, const float* lfact, int32_t n_lfact,
                                                  uint32_t i) {
  if (mu32 > kPtrsFastMaxMu) return -2;
  const PtrsConst32 c = ptrs_const32(mu32, lfact, n_lfact);
  const uint4 x = philox4x32_10_rk(make_uint4(i, layer | (kPurposePoisson << 16), particle, event), rk);
  return (int32_t)ptrs_iter32(mu32, c, x);
}

// Parametrisation entry of a particle (without the layer index).  Energy bin
// from floor(log2 E): the float's exponent field for normal E, and for a
// subnormal E = m 2^-149 the position of m's leading bit.  |eta| bin: for an
// integer scale S < 256, |eta| S =
// m S 2^(e - 150) with m the 24-bit significand, so its floor is an exact
// integer shift; other scales take the FP64 product, which is exact too.
__device__ __forceinline__ int32_t eta_bin(const ParamDev& p, float eta) {
  const uint32_t bits = __float_as_uint(eta) & 0x7FFFFFFFu;
  const int32_t ef = (int32_t)(bits >> 23);
  int32_t hb;
  if (p.eta_scale_int) {
    if (ef >= 150 + 8) {
      hb = p.NH - 1;
    } else {
      const uint32_t m = (bits & 0x7FFFFFu) | (ef ? 0x800000u : 0u);
      const uint64_t prod = (uint64_t)m * (uint32_t)p.eta_scale_int;  // < 2^32
      const int32_t sh = 150 - (ef ? ef : 1);
      const uint64_t fl = (sh >= 0) ? (sh >= 64 ? 0 : prod >> sh) : (prod << (-sh));
      hb = fl >= (uint64_t)(p.NH - 1) ? p.NH - 1 : (int32_t)fl;
    }
  } else {
    const double ae = __dmul_rn(fabs((double)eta), p.eta_scale);
    hb = (ae >= (double)(p.NH - 1)) ? (p.NH - 1) : (int32_t)floor(ae);
  }
  return hb;
}

__device__ __forceinline__ int32_t param_entry(const ParamDev& p, int32_t type, float E, float eta) {
  const uint32_t bits = __float_as_uint(E);  // E > 0
  const int32_t ef = (int32_t)((bits >> 23) & 0xFFu);
  const int32_t lg2 = ef ? ef - 127 : -118 - __clz(bits & 0x7FFFFFu);  // subnormal: -149 + (31 - clz(m))
  int32_t eb = lg2 - p.ebin_min;
  eb = max(0, min(eb, p.NE - 1));
  return (type * p.NE + eb) * p.NH + eta_bin(p, eta);
}

__device__ __forceinline__ bool particle_ok(const ParamDev& p, int32_t t, float E, float eta, float phi) {
  return t >= 0 && t < p.NT && E > 0.0f && isfinite(E) && isfinite(eta) && isfinite(phi);
}

// Event of particle i: last e in [ev_lo, ev_hi) with off[e] <= i.
__device__ __forceinline__ int32_t event_of(const int64_t* off, int32_t ev_lo, int32_t ev_hi, int64_t i) {
  int32_t lo = ev_lo, hi = ev_hi - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Layer mask of a particle: bit l set where the float layer energy
// fl32(E f_l) is > 0 (a task).  The fraction row is read with 16-byte loads,
// all issued before the tests, when the layer count is a multiple of 4.
__device__ __forceinline__ uint32_t layer_mask(const ParamDev& p, int64_t row, float E) {
  const int NL = p.NL;
  uint32_t mask = 0;
  if ((NL & 3) == 0) {
    const float4* f4 = reinterpret_cast<const float4*>(p.frac + row);
    float4 f[kMaxLayers / 4];
#pragma unroll
    for (int c = 0; c < kMaxLayers / 4; ++c) f[c] = (4 * c < NL) ? __ldg(f4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int c = 0; c < kMaxLayers / 4; ++c) {
      mask |= (uint32_t)(__fmul_rn(E, f[c].x) > 0.0f) << (4 * c);
      mask |= (uint32_t)(__fmul_rn(E, f[c].y) > 0.0f) << (4 * c + 1);
      mask |= (uint32_t)(__fmul_rn(E, f[c].z) > 0.0f) << (4 * c + 2);
      mask |= (uint32_t)(__fmul_rn(E, f[c].w) > 0.0f) << (4 * c + 3);
    }
  } else {
    for (int l = 0; l < NL; ++l) mask |= (uint32_t)(__fmul_rn(E, p.frac[row + l]) > 0.0f) << l;
  }
  return mask;
}

// Energy-bin interpolation: E = m 2^k (m in [1, 2)) takes the bin of the
// next point 2^(k+1), clamp(k + 1 - ebin_min, 0, NE - 1), with probability
// m - 1, decided exactly in integers: word 0 of Philox block (0, 2 << 16,
// particle in event, event) below the 23 mantissa bits of E shifted left by
// 9.  (Below the table's first point both points clamp to bin 0.)
__device__ __forceinline__ int32_t interp_entry(const ParamDev& p, int32_t entry, float E, uint32_t pin,
                                                uint32_t event, uint32_t k0, uint32_t k1) {
  const uint32_t x0 = philox4x32_10(make_uint4(0u, kPurposeEnergyBin << 16, pin, event), k0, k1).x;
  const uint32_t bits = __float_as_uint(E);
  if ((bits >> 23) == 0 || x0 >= ((bits & 0x7FFFFFu) << 9)) return entry;  // subnormal E: m < 1
  const int32_t hb = entry % p.NH, t = entry / (p.NH * p.NE);
  const int32_t eb = max(0, min((int32_t)((bits >> 23) & 0xFFu) - 127 + 1 - p.ebin_min, p.NE - 1));
  return (t * p.NE + eb) * p.NH + hb;
}

// Per particle: its checks, parametrisation entry, event and layer mask; the
// task count feeds the scan of task offsets.
__global__ void __launch_bounds__(128) k_particle_count(const ParamDev p, const fcs_particles parts, int32_t ev_lo,
                                                        int32_t ev_hi, WsDev w, int energy_interp, uint32_t k0,
                                                        uint32_t k1, uint32_t first_event_lo) {
  const int64_t pb = parts.event_offsets[ev_lo];
  const int64_t P = w.sizes->n_part;  // checked against the capacity and n_particles
  for (int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; li < P;
       li += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = pb + li;
    const int32_t t = parts.type[i];
    const float E = parts.E[i], eta = parts.eta[i], phi = parts.phi[i];
    uint4 info = make_uint4(0u, 0u, 0u, 0u);
    if (!particle_ok(p, t, E, eta, phi)) {
      atomicOr(&w.sizes->flags, (uint32_t)FCS_FLAG_BAD_PARTICLE);
    } else {
      int32_t entry = param_entry(p, t, E, eta);
      const int32_t e = event_of(parts.event_offsets, ev_lo, ev_hi, i);
      if (energy_interp)
        entry = interp_entry(p, entry, E, (uint32_t)(i - parts.event_offsets[e]), first_event_lo + (uint32_t)e, k0, k1);
      info = make_uint4((uint32_t)entry, (uint32_t)e, layer_mask(p, (int64_t)entry * p.NL, E), 0u);
    }
    w.pcount[li] = __popc(info.z);
    w.pinfo[li] = info;
  }
}

// Task records in (event, particle, layer) order and their Poisson means.
// A warp takes 32 consecutive particles, whose tasks are consecutive too
// (poff), and fills them 32 at a time: lane s of a round builds the task in
// slot s of the warp's range, so each round writes 32 consecutive 32-byte
// records.  The owner of a slot is found by a binary search over the lanes'
// inclusive task counts (shuffles); its data comes by shuffle from the lane
// that loaded the particle.
__global__ void __launch_bounds__(128) k_task_init(const GeoDev g, const ParamDev p, const fcs_particles parts,
                                                   int32_t ev_lo, WsDev w) {
  const int64_t pb = parts.event_offsets[ev_lo];
  const int64_t P = w.sizes->n_part;
  const int NL = p.NL;
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t wb = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; wb < P; wb += warps * 32) {
    const int64_t li = wb + lane;
    const bool have = li < P;
    const uint4 info = have ? w.pinfo[li] : make_uint4(0u, 0u, 0u, 0u);
    const int cnt = __popc(info.z);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) continue;
    const int64_t tbase = __shfl_sync(0xffffffffu, w.poff[have ? li : wb], 0);
    // the particle this lane loaded (lanes without tasks load nothing)
    float E = 0.0f, eta = 0.0f, phi = 0.0f, ch = 0.0f, sh = 0.0f, th = 0.0f;
    int32_t pin = 0;
    if (cnt) {
      const int64_t i = pb + li;
      E = parts.E[i];
      eta = parts.eta[i];
      phi = parts.phi[i];
      pin = (int32_t)(i - parts.event_offsets[info.y]);
      // FP32 scale factors of the (r, alpha) -> (eta, phi) map; the FP64
      // recheck recomputes them in double exactly as the oracle does
      const float ae = fabsf(eta);
      ch = coshf(eta);
      sh = sinhf(ae);
      th = tanhf(ae);
    }
    for (int s0 = 0; s0 < total; s0 += 32) {
      const int sl = s0 + lane;
      int o = 0;  // owner: the first lane whose inclusive count exceeds sl
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int v = __shfl_sync(0xffffffffu, incl, o + step - 1);
        if (v <= sl) o += step;
      }
      o = min(o, 31);
      const int j = sl - (__shfl_sync(0xffffffffu, incl, o) - __shfl_sync(0xffffffffu, cnt, o));
      const uint32_t entry = __shfl_sync(0xffffffffu, info.x, o);
      const uint32_t ev = __shfl_sync(0xffffffffu, info.y, o);
      const uint32_t mask = __shfl_sync(0xffffffffu, info.z, o);
      const float oE = __shfl_sync(0xffffffffu, E, o), oeta = __shfl_sync(0xffffffffu, eta, o);
      const float ophi = __shfl_sync(0xffffffffu, phi, o);
      const float och = __shfl_sync(0xffffffffu, ch, o), osh = __shfl_sync(0xffffffffu, sh, o);
      const float oth = __shfl_sync(0xffffffffu, th, o);
      const int32_t opin = __shfl_sync(0xffffffffu, pin, o);
      const int64_t to = tbase + sl;
      if (sl >= total || to >= w.task_cap) continue;  // the capacity is particles x layers: never
      const int l = (int)__fns(mask, 0u, j + 1);
      const int64_t e = (int64_t)entry * NL + l;
      const float El = __fmul_rn(oE, __ldg(p.frac + e));
      TaskRec r;
      r.entry = (int32_t)e;
      r.El = El;
      r.eta_c = oeta;
      r.phi_c = ophi;
      const float R = g.rz32[l];
      if (g.barrel[l]) {
        r.s_phi = 1.0f / R;
        r.s_eta = 1.0f / (R * och);
      } else {
        const float mm = (oth * osh) / R;
        r.s_phi = osh / R;
        r.s_eta = (oeta < 0.0f) ? mm : -mm;
      }
      r.particle = opin;
      r.ev_layer = (ev << 8) | (uint32_t)l;
      w.tasks[to] = r;
      w.tmu[to] = __fdiv_rn(El, __ldg(p.mhe + e));
    }
  }
}

// n = max(1, Poisson(mu)) in FP32.  Each warp takes windows of 256
// consecutive tasks, lists the window's inversion tasks (mu < 10) from the
// front and its PTRS tasks from the back of a per-warp shared array, and
// draws them 32 at a time, inversion rounds first: a round runs one method,
// and warps never wait for one another.  A PTRS round runs one iteration per
// lane (most draws accept at their first); a draw that rejects goes to the
// warp's retry list with its next iteration, and the list runs as a round
// whenever it holds 32, so that one long draw does not hold 31 idle lanes.
// Draws the FP32 path cannot certify are queued for k_task_poisson64, so that
// FP64 work runs in full warps instead of stalling a warp for one lane.
constexpr int kPoisWarps = 4;
constexpr int kPoisWin = 256;

// Appends the tasks of the lanes with `push` set to a list: warp-aggregated
// counter increment, entry q at list[q] (front) or list[cap - 1 - q] (back).
// Deferred draws are listed by method (inversion at the front of pdefer, PTRS
// at its back) so that the FP64 warps run one method.
__device__ __forceinline__ void warp_push(bool push, int64_t task, unsigned long long* counter, int32_t* list,
                                          bool back, int64_t cap) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, push);
  if (!m) return;
  unsigned long long b = 0;
  const int l0 = __ffs(m) - 1;
  if (lane == l0) b = atomicAdd(counter, (unsigned long long)__popc(m));
  b = __shfl_sync(0xffffffffu, b, l0);
  const int64_t q = (int64_t)b + __popc(m & ((1u << lane) - 1u));
  if (push) list[back ? cap - 1 - q : q] = (int32_t)task;
}

__global__ void __launch_bounds__(32 * kPoisWarps) k_task_poisson(WsDev w, PhiloxRoundKeys rk, uint32_t first_event_lo,
                                                                   const float* lfact, int32_t n_lfact) {
  __shared__ int s_list[kPoisWarps][kPoisWin];  // inversion tasks from the front, PTRS from the back
  __shared__ float s_mu[kPoisWarps][kPoisWin];
  __shared__ float s_rcp[kInvMax + 1];          // 1 / k, correctly rounded
  __shared__ int32_t s_rt[kPoisWarps][64];      // retry list: task
  __shared__ uint8_t s_ri[kPoisWarps][64];      //             and its next PTRS iteration
  for (int k = threadIdx.x; k <= kInvMax; k += blockDim.x) s_rcp[k] = __frcp_rn((float)k);
  __syncthreads();
  const int64_t T = min(w.sizes->n_tasks, w.task_cap);
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t nw = (int64_t)gridDim.x * kPoisWarps;
  unsigned long long* n_inv_defer = (unsigned long long*)&w.sizes->n_pdefer;
  unsigned long long* n_ptrs_defer = (unsigned long long*)&w.sizes->n_pdefer_ptrs;
  int n_r = 0;  // retry list length (warp-uniform, < 64)
  // the loop runs one window past the warp's last to drain the retry list
  for (int64_t win = ((int64_t)blockIdx.x * kPoisWarps + wi) * kPoisWin;; win += nw * kPoisWin) {
    const bool have = win < T;
    int n_i = 0, n_p = 0;
    if (have) {
#pragma unroll
      for (int c = 0; c < kPoisWin / 32; ++c) {
        const int idx = c * 32 + lane;
        const int64_t t = win + idx;
        const float mu = t < T ? w.tmu[t] : 0.0f;
        const bool inv = t < T && mu < 10.0f, pt = t < T && !(mu < 10.0f);
        const unsigned bi = __ballot_sync(0xffffffffu, inv), bp = __ballot_sync(0xffffffffu, pt);
        s_mu[wi][idx] = mu;
        if (inv) s_list[wi][n_i + __popc(bi & lt)] = idx;
        if (pt) s_list[wi][kPoisWin - 1 - (n_p + __popc(bp & lt))] = idx;
        n_i += __popc(bi);
        n_p += __popc(bp);
      }
      __syncwarp();
      for (int r0 = 0; r0 < n_i; r0 += 32) {
        const int j = r0 + lane;
        const bool valid = j < n_i;
        int32_t k = 0;
        int64_t t = 0;
        if (valid) {
          const int idx = s_list[wi][j];
          t = win + idx;
          const TaskRec& r = w.tasks[t];
          k = poisson_inv_fp32(s_mu[wi][idx], (uint32_t)r.layer(), (uint32_t)r.particle,
                               first_event_lo + (uint32_t)r.event(), rk, s_rcp);
          w.tn[t] = k < 1 ? 1 : k;  // provisional for a deferred draw
        }
        warp_push(valid && k < 0, t, n_inv_defer, w.pdefer, false, w.pdefer_cap);
      }
    }
    // PTRS rounds: new draws of the window 32 at a time, or 32 retries when
    // the list holds that many (after the warp's last window: all it holds)
    int p_next = 0;
    while (p_next < n_p || n_r >= (have ? 32 : 1)) {
      const bool from_retry = n_r >= 32 || p_next >= n_p;
      const int cnt = from_retry ? min(n_r, 32) : min(n_p - p_next, 32);
      const bool valid = lane < cnt;
      int64_t t = 0;
      uint32_t it = 0;
      float mu = 0.0f;
      if (valid) {
        if (from_retry) {
          t = s_rt[wi][lane];
          it = s_ri[wi][lane];
          mu = w.tmu[t];
        } else {
          const int idx = s_list[wi][kPoisWin - 1 - (p_next + lane)];
          t = win + idx;
          mu = s_mu[wi][idx];
        }
      }
      if (from_retry) {  // the entries past the round move to the front
        const int rest = n_r - cnt;
        const int32_t mt = lane < rest ? s_rt[wi][cnt + lane] : 0;
        const uint8_t mi = lane < rest ? s_ri[wi][cnt + lane] : 0;
        __syncwarp();
        if (lane < rest) {
          s_rt[wi][lane] = mt;
          s_ri[wi][lane] = mi;
        }
        __syncwarp();
        n_r = rest;
      } else {
        p_next += cnt;
      }
      int32_t k = 0;
      if (valid) {
        const TaskRec& r = w.tasks[t];
        k = ptrs_step_fp32(mu, (uint32_t)r.layer(), (uint32_t)r.particle, first_event_lo + (uint32_t)r.event(), rk,
                           lfact, n_lfact, it);
        if (k == -1 && it + 1 >= kPtrsMaxIter) k = (int32_t)floorf(mu);  // every iteration rejected
        if (k >= 0) w.tn[t] = k < 1 ? 1 : k;
        else if (k == -2) w.tn[t] = it;  // the FP64 definition resumes here
      }
      warp_push(valid && k == -2, t, n_ptrs_defer, w.pdefer, true, w.pdefer_cap);
      const bool rt = valid && k == -1;
      const unsigned rm = __ballot_sync(0xffffffffu, rt);
      if (rt) {
        const int q = n_r + __popc(rm & lt);
        s_rt[wi][q] = (int32_t)t;
        s_ri[wi][q] = (uint8_t)(it + 1);
      }
      n_r += __popc(rm);
      __syncwarp();
    }
    if (!have) break;
    __syncwarp();  // the window's lists are reused
  }
}

// A deferred PTRS draw from its uncertain iteration i0 on: iteration i0 in
// FP64 (the definition), each later one in FP32 where its decisions are
// certain (they are then the FP64 ones) and in FP64 where they are not.  A
// warp's time is its longest chain of FP64 iterations, and most draws that
// reject at i0 are decided in FP32 after it.
__device__ __noinline__ int64_t ptrs_resume(float mu32, uint32_t layer, uint32_t particle, uint32_t event,
                                            uint32_t k0, uint32_t k1, const PhiloxRoundKeys& rk,
                                            const float* lfact, const double* lfact64, int32_t n_lfact, uint32_t i0) {
  const double mu = (double)mu32;
  const PtrsConst64 c = ptrs_const64(mu);
  for (uint32_t i = i0; i < kPtrsMaxIter; ++i) {
    if (i != i0) {
      const int32_t k32 = ptrs_step_fp32(mu32, layer, particle, event, rk, lfact, n_lfact, i);
      if (k32 >= 0) return k32;
      if (k32 == -1) continue;
    }
    double u, V;
    draw_pair(i, layer, particle, event, k0, k1, &u, &V);
    const int64_t k = ptrs_iter64(mu, c, u, V, lfact64, n_lfact);
    if (k >= 0) return k;
  }
  return (int64_t)floor(mu);
}

// The deferred draws: the inversion list (front of pdefer) by the FP64
// definition, then the PTRS list (back of pdefer) resumed at the iteration
// the FP32 path could not decide; 32 per warp, so that a warp runs one method
// except at the seam.
__global__ void __launch_bounds__(128) k_task_poisson64(WsDev w, uint32_t k0, uint32_t k1, PhiloxRoundKeys rk,
                                                         uint32_t first_event_lo, const float* lfact,
                                                         const double* lfact64, int32_t n_lfact) {
  const int64_t n_inv = w.sizes->n_pdefer, n_ptrs = w.sizes->n_pdefer_ptrs;
  const int64_t n = n_inv + n_ptrs;
  if (blockIdx.x == 0 && threadIdx.x == 0) w.sizes->n_poisson_fp64 += (uint32_t)n;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const bool inv = q < n_inv;
    const int32_t t = w.pdefer[inv ? q : w.pdefer_cap - 1 - (q - n_inv)];
    const TaskRec& r = w.tasks[t];
    const uint32_t layer = (uint32_t)r.layer(), particle = (uint32_t)r.particle;
    const uint32_t event = first_event_lo + (uint32_t)r.event();
    int64_t k = inv ? poisson_draw((double)w.tmu[t], layer, particle, event, k0, k1, lfact64, n_lfact, 0u)
                    : ptrs_resume(w.tmu[t], layer, particle, event, k0, k1, rk, lfact, lfact64, n_lfact,
                                  (uint32_t)w.tn[t]);
    if (k < 1) k = 1;
    if (k > 0x7FFFFFFF) k = 0x7FFFFFFF;
    w.tn[t] = k;
  }
}

// One thread per task: in deterministic mode the hit energy into tmu (the
// fold's compact copy); validation dumps; the tile map (granule -> task
// holding its first hit) again when the call grew it after the scan that
// wrote it (fill_map).
__global__ void k_task_finish(WsDev w, fcs_debug dbg, int has_dbg, int det, int fill_map) {
  const int64_t T = min(w.sizes->n_tasks, w.task_cap);
  const int64_t H = w.sizes->n_hits;
  const bool map_ok = fill_map && H <= w.gmap_cap * (int64_t)kGranule;
  const int64_t task_base = w.sizes->task_base;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = w.tn[t];
    if (map_ok) {
      const int64_t b = w.th[t];
      for (int64_t gi = (b + kGranule - 1) / kGranule; gi * kGranule < b + n; ++gi) w.gmap[gi] = (int32_t)t;
    }
    if (det || has_dbg) {
      const TaskRec& r = w.tasks[t];
      const float Ehit = __fdiv_rn(r.El, (float)n);
      if (det) w.tmu[t] = Ehit;
      if (has_dbg) {
        const int64_t dt = task_base + t;
        if (dt < dbg.task_capacity) {
          if (dbg.task_event) dbg.task_event[dt] = r.event();
          if (dbg.task_particle) dbg.task_particle[dt] = r.particle;
          if (dbg.task_layer) dbg.task_layer[dt] = r.layer();
          if (dbg.task_n) dbg.task_n[dt] = (int32_t)n;
          if (dbg.task_Ehit) dbg.task_Ehit[dt] = Ehit;
        }
      }
    }
  }
}

// Blocks of 128 threads for n items, at most 16 per SM (a full SM's worth).
int grid_for(int64_t n, const Launch& L) {
  const int64_t b = (std::max<int64_t>(n, 1) + 127) / 128;
  return (int)std::min<int64_t>(b, (int64_t)L.num_sms * 16);
}

// Blocks of `block` threads of `kernel` that one SM holds at once (its
// registers and shared memory decide).  Grid-stride kernels launched with
// more blocks than that run the surplus as a second, mostly empty wave.
int resident_blocks(const void* kernel, int block) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    n = 1;
  }
  return std::max(n, 1);
}

// The same, cached per device for the two task kernels (the stores are
// ordered so that a non-zero `init` implies `pois` is set).
constexpr int kMaxDevices = 64;
struct TaskOccupancy {
  std::atomic<int> init{0}, pois{0};
};

}  // namespace

cudaError_t launch_task_counts(const GeoDev& g, const ParamDev& p, const fcs_particles& parts, int32_t ev_lo,
                               int32_t ev_hi, uint32_t k0, uint32_t k1, int64_t first_event, WsDev w, ScanTmp tmp,
                               int64_t n_part_max, int energy_interp, const Launch& L) {
  // one thread per particle / task where the grid allows (these kernels wait
  // on dependent loads: more threads in flight, not fewer, hide them)
  const int gp = grid_for(n_part_max, L);
  k_particle_count<<<gp, 128, 0, L.s>>>(p, parts, ev_lo, ev_hi, w, energy_interp, k0, k1, (uint32_t)first_event);
  cudaError_t e = launch_scan_i64(w.pcount, w.poff, &w.sizes->n_part, 0, &w.sizes->n_tasks, 0, tmp, L.s);
  if (e != cudaSuccess) return e;
  // the task kernels loop grid-stride: one wave of resident blocks
  static TaskOccupancy occ_by_device[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = kMaxDevices - 1;
  TaskOccupancy& occ = occ_by_device[dev];
  int occ_init = occ.init.load(std::memory_order_acquire), occ_pois;
  if (occ_init) {
    occ_pois = occ.pois.load(std::memory_order_relaxed);
  } else {
    occ_pois = resident_blocks((const void*)k_task_poisson, 32 * kPoisWarps);
    occ_init = resident_blocks((const void*)k_task_init, 128);
    occ.pois.store(occ_pois, std::memory_order_relaxed);
    occ.init.store(occ_init, std::memory_order_release);
  }
  k_task_init<<<std::min(gp, L.num_sms * occ_init), 128, 0, L.s>>>(g, p, parts, ev_lo, w);
  const int gpois = (int)std::min<int64_t>(
      (std::max<int64_t>(n_part_max * p.NL, 1) + kPoisWarps * kPoisWin - 1) / (kPoisWarps * kPoisWin),
      (int64_t)L.num_sms * occ_pois);
  k_task_poisson<<<gpois, 32 * kPoisWarps, 0, L.s>>>(w, philox_round_keys(k0, k1), (uint32_t)first_event, p.lfact,
                                                     p.n_lfact);
  // the FP64 pipe is narrow: one warp per block spreads the few deferred draws
  // over every SM
  k_task_poisson64<<<L.num_sms * 8, 32, 0, L.s>>>(w, k0, k1, philox_round_keys(k0, k1), (uint32_t)first_event,
                                                   p.lfact, p.lfact64, p.n_lfact);
  // the scan counts the tasks actually written (n_tasks <= task_cap by construction)
  return launch_scan_hits(w.tn, w.th, &w.sizes->n_tasks, &w.sizes->n_hits, w.gmap, w.gmap_cap, tmp, L.s);
}

cudaError_t launch_task_finish(WsDev w, const fcs_debug* dbg, int det, int fill_map, int64_t n_task_max,
                               const Launch& L) {
  if (!dbg && !det && !fill_map) return cudaSuccess;  // the scan wrote the tile map
  fcs_debug d{};
  if (dbg) d = *dbg;
  k_task_finish<<<grid_for(n_task_max, L), 128, 0, L.s>>>(w, d, dbg ? 1 : 0, det, fill_map);
  return cudaGetLastError();
}

}  // namespace fcs
