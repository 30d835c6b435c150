// fcs_tasks.cu - task build of the hit loop (Listing 1): per particle the
// parametrisation entry and its layers with a non-zero float layer energy;
// per task the Poisson hit count (get_number_of_hits) and the float hit
// energy; task records in (event, particle, layer) order.  One kernel writes
// the records and draws their counts, keeping the Poisson draws of a warp
// together in per-method queues.  (The hit-offset scan writes the tile -> task
// map; the task finish kernel here writes it again when a call grew the map
// after that scan.)
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
constexpr int kInvMax = 200;  // even: the FP32 search takes two steps a trip
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
// the iteration (PTRS) or the whole inversion is redone in FP64.  Rounding to
// nearest costs at most 2^-24 relative; expf and logf are within 2 and 1 ulp
// (2^-22 and 2^-23 relative), __fdividef within 2 ulp for divisors in
// [2^-126, 2^126] (every divisor here is), as documented.  Bounds:
//   inversion: p_0 = expf(-mu) is within 2^-22 relative; each step's two
//     products by mu and by the rounded 1/k add 3 2^-24, so p_k is within
//     (4 + 3k) 2^-24 relative and, with one rounding per partial sum (F <= 1),
//     |F32_k - F_k| <= (4 + 4k) 2^-24; the 53-bit uniform rounded to FP32 is
//     off by <= 2^-24, so u - F is known to (4k + 5) 2^-24 = (k + 1.25) 2^-22.
//     Used: (k + 2) 2^-22.
//   PTRS constants: sqrtf, the FP32 images of the decimal constants and one
//     rounding per operation put b within 2^-22 relative, a within 2^-21,
//     1/alpha within 2^-22 and v_r within 2^-21 absolute.  The quotients
//     2a/us and a/us^2 of an iteration are within 2^-20 relative.
//   PTRS acceptance test, d = (log V + log 1/alpha - log(a/us^2 + b))
//     - (-mu + k log mu - log k!): its three logs take __logf, within
//     2^-21.41 absolute on [1/2, 2] and 3 ulp (3 2^-23 relative) elsewhere,
//     as documented, so the left side is known to
//     3.0 2^-20 + 1.25 2^-20 (|l1| + |l2| + |l3|); the right side (log mu
//     within 1 ulp, log k! a correctly rounded table entry, two sums) to
//     2^-23 (2.5 |k log mu| + |log k!| + mu).  Used: 2^-18 + 2^-19 (|l1| + |l2|
//     + |l3|) + 2^-20 (|k log mu| + |log k!| + mu), above each term.
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
  const int32_t ki = (int32_t)kf;
  if (ki >= c.n_lfact) return -2;  // past the log k! table (never below kPtrsFastMaxMu): FP64
  const float l1 = __logf(Vf), l2 = __logf(c.invalpha), l3 = __logf(__fdividef(c.a, usf * usf) + c.b);
  const float kl = kf * c.loglam, lg = __ldg(c.lfact + ki);
  const float d = (l1 + l2 - l3) - ((-mu + kl) - lg);
  const float bd = fmaf(fabsf(l1) + fabsf(l2) + fabsf(l3), 0x1p-19f,
                        fmaf(fabsf(kl) + fabsf(lg) + mu, 0x1p-20f, 0x1p-18f));
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
  static_assert(kInvMax % 2 == 0, "two steps a trip end exactly at kInvMax");
  if (!(mu32 > 0.0f)) return 0;
  const uint4 x = philox4x32_10_rk(make_uint4(0u, layer | (kPurposePoisson << 16), particle, event), rk);
  const float uf = u53f(x.x, x.y);
  float p = expf(-mu32);
  float F = p;
  float e = 0x1p-21f;  // (k + 2) 2^-22, exact in FP32 for k <= kInvMax
  float d = uf - F;
  int k = 0;
  if (d > e) {  // u > F_0 for certain: the search goes on
    // two steps a trip: F_{k+2} >= F_{k+1} in FP32 too and the bound grows,
    // so a certain u > F_{k+2} makes u > F_{k+1} certain as well
    for (;;) {
      const float p1 = (p * mu32) * rcp[k + 1];
      const float F1 = F + p1;
      const float p2 = (p1 * mu32) * rcp[k + 2];
      const float F2 = F1 + p2;
      const float d2 = uf - F2, e2 = e + 0x1p-21f;
      if (d2 > e2 && k + 2 < kInvMax) {
        k += 2;
        p = p2;
        F = F2;
        e = e2;
        continue;
      }
      const float d1 = uf - F1, e1 = e + 0x1p-22f;
      if (d1 > e1) {  // the search passes k + 1 and stops at k + 2 (or is uncertain there)
        k += 2;
        d = d2;
        e = e2;
      } else {
        k += 1;
        d = d1;
        e = e1;
      }
      break;
    }
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

// Task records in (event, particle, layer) order and their FP32 Poisson hit
// counts, n = max(1, Poisson(mu)), in one pass: a task's draw runs while its
// record is still at hand, so the records are written once and not read back.
//
// Building: a warp takes 32 consecutive particles, whose tasks are consecutive
// too (poff), and fills them 32 at a time: lane s of a round builds the task in
// slot s of the warp's range, so each round writes 32 consecutive 32-byte
// records.  Each lane first lists its particle's tasks in shared memory (slot
// -> its lane and the layer of its k-th set mask bit); a slot's builder reads
// its owner and layer there and the owner's data by shuffle.
//
// Drawing: each new task joins one of two per-warp queues in shared memory,
// inversion (mu < 10) or PTRS, with its Philox counter fields.  Whenever a
// queue holds 32 draws the warp runs one round of that method on 32 of them,
// so a round runs one method in full lanes and warps never wait for one
// another.  A PTRS round runs one iteration per lane (most draws accept at
// their first); a draw that rejects goes back into the queue with its next
// iteration, so one long draw does not hold 31 idle lanes.  Draws the FP32 path
// cannot certify (a few in 1e4) are listed for k_task_poisson64, which runs
// them in full warps: an FP64 instruction holds the narrow FP64 pipe as long
// for one lane as for 32.  A warp drains its queues after its last particles.
constexpr int kBuildWarps = 4;
constexpr int kDrawQ = 64;  // < 32 left after the rounds + 32 new (or 32 retried)

struct DrawEnt {
  float mu;
  int32_t t;          // task
  uint32_t particle;  // particle in its event
  uint32_t evl;       // event in the range << 8 | layer
};

// Per-warp queues in shared memory: entries [0, n) of each, n warp-uniform.
struct WarpQueue {
  DrawEnt* e;
  uint8_t* it;  // PTRS queue: the entry's next iteration
  int n;
};

// Appends the draws of the lanes with `push` set to a queue (n + 32 <= kDrawQ).
__device__ __forceinline__ void queue_push(WarpQueue& q, bool push, const DrawEnt& d, uint8_t it) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, push);
  if (push) {
    const int j = q.n + __popc(m & ((1u << lane) - 1u));
    q.e[j] = d;
    q.it[j] = it;
  }
  q.n += __popc(m);
  __syncwarp();
}

// Takes the last min(n, 32) entries of a queue, one per lane; false for the
// lanes past them.
__device__ __forceinline__ bool queue_take(WarpQueue& q, DrawEnt* d, uint32_t* it) {
  const int lane = threadIdx.x & 31;
  const int cnt = min(q.n, 32);
  const bool valid = lane < cnt;
  if (valid) {
    *d = q.e[q.n - cnt + lane];
    *it = q.it[q.n - cnt + lane];
  }
  q.n -= cnt;
  __syncwarp();  // read before the queue grows again
  return valid;
}

// Appends the tasks of the lanes with `push` set to a global list:
// warp-aggregated counter increment, entry q at list[q] (front) or
// list[cap - 1 - q] (back).  Deferred draws are listed by method (inversion at
// the front of pdefer, PTRS at its back) so that the FP64 warps run one method.
__device__ __forceinline__ void warp_push(bool push, int32_t task, unsigned long long* counter, int32_t* list,
                                          bool back, int64_t cap) {
  const int lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, push);
  if (!m) return;
  unsigned long long b = 0;
  const int l0 = __ffs(m) - 1;
  if (lane == l0) b = atomicAdd(counter, (unsigned long long)__popc(m));
  b = __shfl_sync(0xffffffffu, b, l0);
  const int64_t q = (int64_t)b + __popc(m & ((1u << lane) - 1u));
  if (push) list[back ? cap - 1 - q : q] = task;
}

// One inversion round; uncertain draws are listed for k_task_poisson64.
__device__ __forceinline__ void inversion_round(WarpQueue& q, const WsDev& w, const PhiloxRoundKeys& rk,
                                                uint32_t first_event_lo, const float* rcp) {
  DrawEnt d{};
  uint32_t it = 0;
  const bool valid = queue_take(q, &d, &it);
  int32_t k = 0;
  if (valid) {
    k = poisson_inv_fp32(d.mu, d.evl & 0xFFu, d.particle, first_event_lo + (d.evl >> 8), rk, rcp);
    if (k >= 0) w.tn[d.t] = k < 1 ? 1 : k;
  }
  warp_push(valid && k < 0, d.t, (unsigned long long*)&w.sizes->n_pdefer, w.pdefer, false, w.pdefer_cap);
}

// One PTRS round: iteration it of each of up to 32 draws; the draws that
// reject for certain go back into the queue with it + 1, the uncertain ones
// are listed for k_task_poisson64 (tn holds the iteration to resume at).
__device__ __forceinline__ void ptrs_round(WarpQueue& q, const WsDev& w, const PhiloxRoundKeys& rk,
                                           uint32_t first_event_lo, const float* lfact, int32_t n_lfact) {
  DrawEnt d{};
  uint32_t it = 0;
  const bool valid = queue_take(q, &d, &it);
  int32_t k = 0;
  if (valid) {
    k = ptrs_step_fp32(d.mu, d.evl & 0xFFu, d.particle, first_event_lo + (d.evl >> 8), rk, lfact, n_lfact, it);
    if (k == -1 && it + 1 >= kPtrsMaxIter) k = (int32_t)floorf(d.mu);  // every iteration rejected
    if (k >= 0) w.tn[d.t] = k < 1 ? 1 : k;
    else if (k == -2) w.tn[d.t] = (int32_t)it;
  }
  queue_push(q, valid && k == -1, d, (uint8_t)(it + 1));
  warp_push(valid && k == -2, d.t, (unsigned long long*)&w.sizes->n_pdefer_ptrs, w.pdefer, true, w.pdefer_cap);
}

__global__ void __launch_bounds__(32 * kBuildWarps) k_task_build(const GeoDev g, const ParamDev p,
                                                                 const fcs_particles parts, int32_t ev_lo, WsDev w,
                                                                 PhiloxRoundKeys rk, uint32_t first_event_lo) {
  __shared__ DrawEnt s_e[2][kBuildWarps][kDrawQ];  // inversion and PTRS queues
  __shared__ uint8_t s_it[2][kBuildWarps][kDrawQ];
  __shared__ float s_rcp[kInvMax + 1];  // 1 / k, correctly rounded
  __shared__ uint16_t s_slot[kBuildWarps][32 * kMaxLayers];  // owner lane | layer << 8 of the group's tasks
  for (int k = threadIdx.x; k <= kInvMax; k += blockDim.x) s_rcp[k] = __frcp_rn((float)k);
  __syncthreads();
  const int64_t pb = parts.event_offsets[ev_lo];
  const int64_t P = w.sizes->n_part;
  const int NL = p.NL;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  WarpQueue qi{s_e[0][wi], s_it[0][wi], 0}, qp{s_e[1][wi], s_it[1][wi], 0};
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
    uint16_t* slot = s_slot[wi];
    __syncwarp();  // the previous group's rounds have read their slots
    for (uint32_t m = info.z, k = (uint32_t)(incl - cnt); m; m &= m - 1u, ++k)
      slot[k] = (uint16_t)(lane | ((__ffs(m) - 1) << 8));
    __syncwarp();
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
      const uint32_t sv = sl < total ? slot[sl] : 0u;
      const int o = (int)(sv & 31u);  // the particle's lane
      const int l = (int)(sv >> 8);    // the task's layer
      const uint32_t entry = __shfl_sync(0xffffffffu, info.x, o);
      const uint32_t ev = __shfl_sync(0xffffffffu, info.y, o);
      const float oE = __shfl_sync(0xffffffffu, E, o), oeta = __shfl_sync(0xffffffffu, eta, o);
      const float ophi = __shfl_sync(0xffffffffu, phi, o);
      const float och = __shfl_sync(0xffffffffu, ch, o), osh = __shfl_sync(0xffffffffu, sh, o);
      const float oth = __shfl_sync(0xffffffffu, th, o);
      const int32_t opin = __shfl_sync(0xffffffffu, pin, o);
      const int64_t to = tbase + sl;
      // the capacity is particles x layers: `to` never reaches it
      const bool valid = sl < total && to < w.task_cap;
      float mu = 0.0f;
      uint32_t evl = 0;
      if (valid) {
        const int64_t e = (int64_t)entry * NL + l;
        const float El = __fmul_rn(oE, __ldg(p.frac + e));
        TaskRec r;
        r.entry = (int32_t)e;
        r.El = El;
        r.eta_c = oeta;
        r.phi_c = ophi;
        // barrel 1/R and 1/(R cosh eta), end cap sinh|eta|/R and
        // -+tanh|eta| sinh|eta|/R, each a few ulp off (see the hit kernel's
        // error bound)
        const float rinv = __ldg(g.rinv32 + l);
        if (g.barrel[l]) {
          r.s_phi = rinv;
          r.s_eta = rinv * __frcp_rn(och);
        } else {
          const float mm = (oth * osh) * rinv;
          r.s_phi = osh * rinv;
          r.s_eta = (oeta < 0.0f) ? mm : -mm;
        }
        r.particle = opin;
        evl = (ev << 8) | (uint32_t)l;
        r.ev_layer = evl;
        w.tasks[to] = r;
        mu = __fdiv_rn(El, __ldg(p.mhe + e));
      }
      const DrawEnt d{mu, (int32_t)to, (uint32_t)opin, evl};
      queue_push(qi, valid && mu < 10.0f, d, 0);
      queue_push(qp, valid && !(mu < 10.0f), d, 0);
      if (qi.n >= 32) inversion_round(qi, w, rk, first_event_lo, s_rcp);
      while (qp.n >= 32) ptrs_round(qp, w, rk, first_event_lo, p.lfact, p.n_lfact);
    }
  }
  while (qi.n > 0) inversion_round(qi, w, rk, first_event_lo, s_rcp);
  while (qp.n > 0) ptrs_round(qp, w, rk, first_event_lo, p.lfact, p.n_lfact);
}

// The deferred draws: the inversion list (front of pdefer) by the FP64
// definition, then the PTRS list (back of pdefer) resumed at the iteration
// the FP32 path could not decide; 32 per warp, so that a warp runs one method
// except at the seam.  A task's mean is recomputed from its record as the
// build kernel computed it.
__global__ void __launch_bounds__(128) k_task_poisson64(WsDev w, const float* mhe, PhiloxRoundKeys rk,
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
    const float mu = __fdiv_rn(r.El, __ldg(mhe + r.entry));
    int64_t k = inv ? poisson_draw((double)mu, layer, particle, event, rk.k[0], rk.k[1], lfact64, n_lfact, 0u)
                    : ptrs_resume(mu, layer, particle, event, rk.k[0], rk.k[1], rk, lfact, lfact64, n_lfact,
                                  (uint32_t)w.tn[t]);
    if (k < 1) k = 1;
    if (k > 0x7FFFFFFF) k = 0x7FFFFFFF;
    w.tn[t] = (int32_t)k;
  }
}

// Audit of the FP32 path against the FP64 definition: draw i with mean mu[i]
// (Philox counter fields layer i & 0xFF, particle i >> 8, event 0) by the FP32
// path alone, which stops at its first uncertain decision, and by the FP64
// definition.  n32[i]: the FP32 count, -1 where an inversion was uncertain,
// -2 - i0 where PTRS iteration i0 was; n64[i]: the definition's count (both
// before max(1, .)).
__global__ void __launch_bounds__(128) k_poisson_audit(const float* mu, int64_t n, uint32_t k0, uint32_t k1,
                                                        PhiloxRoundKeys rk, const float* lfact,
                                                        const double* lfact64, int32_t n_lfact, int32_t* n32,
                                                        int32_t* n64) {
  __shared__ float s_rcp[kInvMax + 1];
  for (int k = threadIdx.x; k <= kInvMax; k += blockDim.x) s_rcp[k] = __frcp_rn((float)k);
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float m = mu[i];
    const uint32_t layer = (uint32_t)(i & 0xFF), particle = (uint32_t)(i >> 8);
    int32_t r = -1;
    if (m < 10.0f) {
      r = poisson_inv_fp32(m, layer, particle, 0u, rk, s_rcp);
    } else {
      for (uint32_t it = 0; it < kPtrsMaxIter; ++it) {
        const int32_t k = ptrs_step_fp32(m, layer, particle, 0u, rk, lfact, n_lfact, it);
        if (k == -1) {
          if (it + 1 >= kPtrsMaxIter) r = (int32_t)floorf(m);
          continue;
        }
        r = k >= 0 ? k : -2 - (int32_t)it;
        break;
      }
    }
    int64_t k64 = poisson_draw((double)m, layer, particle, 0u, k0, k1, lfact64, n_lfact, 0u);
    if (k64 > 0x7FFFFFFF) k64 = 0x7FFFFFFF;
    n32[i] = r;
    n64[i] = (int32_t)k64;
  }
}

// One thread per task: validation dumps; the tile map (granule -> task
// holding its first hit) again when the call grew it after the scan that
// wrote it (fill_map).
__global__ void k_task_finish(WsDev w, fcs_debug dbg, int has_dbg, int fill_map) {
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
    if (has_dbg) {
      const TaskRec& r = w.tasks[t];
      const float Ehit = __fdiv_rn(r.El, (float)n);
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

constexpr int kMaxDevices = 64;

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
  // the build kernel loops grid-stride: one wave of resident blocks
  static std::atomic<int> occ_by_device[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = kMaxDevices - 1;
  int occ = occ_by_device[dev].load(std::memory_order_relaxed);
  if (!occ) {
    occ = resident_blocks((const void*)k_task_build, 32 * kBuildWarps);
    occ_by_device[dev].store(occ, std::memory_order_relaxed);
  }
  const PhiloxRoundKeys rk = philox_round_keys(k0, k1);
  const int gb = (int)std::min<int64_t>((std::max<int64_t>(n_part_max, 1) + 32 * kBuildWarps - 1) / (32 * kBuildWarps),
                                        (int64_t)L.num_sms * occ);
  k_task_build<<<gb, 32 * kBuildWarps, 0, L.s>>>(g, p, parts, ev_lo, w, rk, (uint32_t)first_event);
  // the FP64 pipe is narrow: one warp per block spreads the few deferred draws
  // over every SM
  k_task_poisson64<<<L.num_sms * 8, 32, 0, L.s>>>(w, p.mhe, rk, (uint32_t)first_event, p.lfact, p.lfact64,
                                                   p.n_lfact);
  // the scan counts the tasks actually written (n_tasks <= task_cap by construction)
  return launch_scan_hits(w.tn, w.th, &w.sizes->n_tasks, &w.sizes->n_hits, w.gmap, w.gmap_cap, tmp, L.s);
}

cudaError_t launch_task_finish(WsDev w, const fcs_debug* dbg, int fill_map, int64_t n_task_max, const Launch& L) {
  if (!dbg && !fill_map) return cudaSuccess;  // the scan wrote the tile map
  fcs_debug d{};
  if (dbg) d = *dbg;
  k_task_finish<<<grid_for(n_task_max, L), 128, 0, L.s>>>(w, d, dbg ? 1 : 0, fill_map);
  return cudaGetLastError();
}

cudaError_t launch_poisson_audit(const ParamDev& p, const float* mu, int64_t n, uint32_t k0, uint32_t k1,
                                 int32_t* n32, int32_t* n64, const Launch& L) {
  if (n <= 0) return cudaSuccess;
  k_poisson_audit<<<grid_for(n, L), 128, 0, L.s>>>(mu, n, k0, k1, philox_round_keys(k0, k1), p.lfact, p.lfact64,
                                                   p.n_lfact, n32, n64);
  return cudaGetLastError();
}

}  // namespace fcs
