/*
 * fcs_oracle.c - plain, slow, single-threaded oracle of the parameterised
 * calorimeter hit path of arXiv:2103.14737 (FastCaloSim ported to GPUs).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke entry and the
 * benchmark's CPU-baseline leg.  It shares no code with the CUDA library.
 *
 * What the paper fixes, and where:
 *   - the per-layer hit loop: nhit = number of hits, Ehit = E(layer)/nhit in
 *     float, every hit carries Ehit, and a chain of per-hit steps decides the
 *     cell each hit deposits into (Sec. 4, Listing 1);
 *   - three random numbers per hit (Sec. 4);
 *   - the hit-to-cell mapping by region then cell, and the energy deposit by
 *     accumulation into the cell array (Sec. 7.3, Listing 2);
 *   - geometry of regions and cells flattened into arrays (Sec. 4);
 *   - results as (cell id, E) pairs of the hit cells (Sec. 4).
 * The paper does not give the random generator, the hit-count distribution,
 * the parametrisation lookup, the shape sampling or the (r, alpha) -> (eta,
 * phi) map.  The readings adopted here (Philox4x32-10; Poisson with
 * inversion / PTRS; power-of-two energy bins and 0.05 |eta| bins; inverse
 * CDF over a 16x8 (r, alpha) histogram with uniform-in-bin positions; a
 * linear barrel / end-cap map around the particle's direction) are listed
 * with reasons in the design notes and pinned by the CPU tests.
 *
 * Precision: FP64 throughout, except the FP32 steps the paper fixes (the
 * float layer energy and hit energy of Listing 1) and the canonical FP32 cell
 * fold of deterministic mode.  Built with -ffp-contract=off.
 */
#include "fcs_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

const char* orc_version(void) { return "fcs-oracle 1"; }

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As    */
/* Easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the  */
/* published multipliers, the key bumped by the published Weyl constants      */
/* between rounds.  Random draws of the method: Sec. 4 (3 per hit).           */
/* ------------------------------------------------------------------------- */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
    uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c[0];
  out[1] = c[1];
  out[2] = c[2];
  out[3] = c[3];
}

void orc_philox_n(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out) {
  for (int64_t i = 0; i < n; ++i) orc_philox(ctr + 4 * i, key, out + 4 * i);
}

/* 24-bit uniform on [0, 1): top 24 bits of a word. */
static double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }
/* 53-bit uniform on [0, 1) from two words (27 + 26 bits). */
static double u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

/* Counter layout: (index, layer | purpose << 16, particle in event, event). */
enum { PURPOSE_HIT = 0, PURPOSE_POISSON = 1, PURPOSE_EBIN = 2 };

static void draw_pair(const uint32_t key[2], uint32_t i, uint32_t layer, uint32_t particle,
                      uint32_t event, double* u, double* v) {
  uint32_t ctr[4] = {i, layer | ((uint32_t)PURPOSE_POISSON << 16), particle, event};
  uint32_t x[4];
  orc_philox(ctr, key, x);
  *u = u53(x[0], x[1]);
  *v = u53(x[2], x[3]);
}

/* ------------------------------------------------------------------------- */
/* Hit count (Listing 1, get_number_of_hits).  The paper gives only the range  */
/* (1 to 15,000 hits per layer, Sec. 4); the count is read as Poisson(mu):    */
/*   mu < 10 : inversion by sequential search from p0 = exp(-mu);             */
/*   mu >= 10: PTRS, the transformed rejection with squeeze of W. Hoermann,   */
/*             "The transformed rejection method for generating Poisson       */
/*             random variables", Insurance: Math. Econ. 12 (1993).           */
/* Draw i of a task uses Philox block (i, layer | 1 << 16, particle, event);  */
/* its four words give two 53-bit uniforms (u, v).                            */
/* ------------------------------------------------------------------------- */
#define POISSON_INV_MAX 200
#define PTRS_MAX_ITER 64

/* PTRS constants of a mean mu >= 10 (Hoermann 1993, Table 2 of the        */
/* transformed-rejection paper: b, a, the hat's 1/alpha and the squeeze v_r). */
typedef struct ptrs_c {
  double mu, loglam, b, a, invalpha, vr;
} ptrs_c;

static ptrs_c ptrs_constants(double mu) {
  ptrs_c c;
  const double slam = sqrt(mu);
  c.mu = mu;
  c.loglam = log(mu);
  c.b = 0.931 + 2.53 * slam;
  c.a = -0.059 + 0.02483 * c.b;
  c.invalpha = 1.1239 + 1.1328 / (c.b - 3.4);
  c.vr = 0.9277 - 3.6224 / (c.b - 2.0);
  return c;
}

/* One PTRS iteration from its uniforms u, V in [0, 1): the accepted count,  */
/* or -1 when the iteration rejects.  k = floor((2a/us + b) U + mu + 0.43)    */
/* with U = u - 1/2, us = 1/2 - |U|; quick acceptance (squeeze) when us >=   */
/* 0.07 and V <= v_r; rejection when k < 0 or (us < 0.013 and V > us); else  */
/* acceptance when log V + log(1/alpha) - log(a/us^2 + b) <= log p_mu(k).     */
static int64_t ptrs_iter(const ptrs_c* c, double u, double V) {
  const double U = u - 0.5;
  const double us = 0.5 - fabs(U);
  if (us <= 0.0) return -1; /* u == 0 exactly */
  const double kd = floor((2.0 * c->a / us + c->b) * U + c->mu + 0.43);
  if (us >= 0.07 && V <= c->vr) return (int64_t)kd;
  if (kd < 0.0 || (us < 0.013 && V > us)) return -1;
  const double lhs = log(V) + log(c->invalpha) - log(c->a / (us * us) + c->b);
  const double rhs = -c->mu + kd * c->loglam - lgamma(kd + 1.0);
  return (lhs <= rhs) ? (int64_t)kd : -1;
}

void orc_ptrs_iter_n(int64_t n, double mu, const double* u, const double* V, int64_t* out) {
  const ptrs_c c = ptrs_constants(mu);
  for (int64_t i = 0; i < n; ++i) out[i] = ptrs_iter(&c, u[i], V[i]);
}

int64_t orc_poisson(double mu, const uint32_t key[2], uint32_t layer, uint32_t particle,
                    uint32_t event) {
  if (!(mu > 0.0)) return 0;
  if (mu < 10.0) {
    double u, v;
    draw_pair(key, 0u, layer, particle, event, &u, &v);
    double p = exp(-mu);
    double F = p;
    int64_t k = 0;
    /* smallest k with u < F_k */
    while (u >= F && k < POISSON_INV_MAX) {
      k += 1;
      p = (p * mu) / (double)k;
      F = F + p;
    }
    return k;
  }
  const ptrs_c c = ptrs_constants(mu);
  for (uint32_t i = 0; i < PTRS_MAX_ITER; ++i) {
    double u, V;
    draw_pair(key, i, layer, particle, event, &u, &V);
    const int64_t k = ptrs_iter(&c, u, V);
    if (k >= 0) return k;
  }
  return (int64_t)floor(mu);
}

void orc_poisson_n(int64_t n, const double* mu, const uint32_t key[2], const uint32_t* layer,
                   const uint32_t* particle, const uint32_t* event, int64_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_poisson(mu[i], key, layer[i], particle[i], event[i]);
}

/* ------------------------------------------------------------------------- */
/* Parametrisation selection by particle type, energy and |eta| (Sec. 1: the  */
/* optimal parametrisation is selected by type, energy and location).         */
/* Energy bin: floor(log2 E) - ebin_log2_min, clamped (the paper's samples    */
/* are at powers of two in MeV, Tables 1 and 3).  |eta| bin: floor(|eta| *    */
/* scale) clamped to NH - 1.                                                  */
/* ------------------------------------------------------------------------- */
int32_t orc_param_entry(const orc_params* P, int32_t type, float E, float eta) {
  int ex = 0;
  (void)frexp((double)E, &ex); /* E = m * 2^ex, m in [0.5, 1) */
  int32_t eb = (ex - 1) - P->ebin_log2_min;
  if (eb < 0) eb = 0;
  if (eb > P->NE - 1) eb = P->NE - 1;
  double ae = fabs((double)eta) * P->eta_bin_scale;
  int32_t hb;
  if (ae >= (double)(P->NH - 1)) hb = P->NH - 1;
  else hb = (int32_t)floor(ae);
  return (type * P->NE + eb) * P->NH + hb;
}

/* Energy-bin interpolation (a reading: the paper selects "the optimal"     */
/* parametrisation, Sec. 1, and leaves interpolation out).  The bins' points */
/* are the powers of two 2^k; E = m 2^k, m in [1, 2), takes bin k + 1 with  */
/* probability m - 1 (linear in E between the two points).                  */
int32_t orc_param_entry_rng(const orc_params* P, int32_t type, float E, float eta, const uint32_t key[2],
                            uint32_t particle, uint32_t event) {
  const int32_t base = orc_param_entry(P, type, E, eta);
  if (!P->energy_interp || E < FLT_MIN) return base; /* subnormal energies are not interpolated */
  int ex = 0;
  const double m = 2.0 * frexp((double)E, &ex); /* E = m * 2^(ex - 1), m in [1, 2) */
  const uint32_t ctr[4] = {0u, (uint32_t)PURPOSE_EBIN << 16, particle, event};
  uint32_t x[4];
  orc_philox(ctr, key, x);
  const double u = (double)x[0] * (1.0 / 4294967296.0);
  if (!(u < m - 1.0)) return base;
  int32_t eb = (ex - 1) - P->ebin_log2_min + 1;
  if (eb < 0) eb = 0;
  if (eb > P->NE - 1) eb = P->NE - 1;
  const int32_t hb = base % P->NH;
  return (type * P->NE + eb) * P->NH + hb;
}

/* ------------------------------------------------------------------------- */
/* Inverse-CDF thresholds of a shape histogram.  With C_k the FP64            */
/* left-to-right prefix sum of the first k weights and K the last bin of      */
/* nonzero weight: T[k] = min(2^32 - 1, floor(2^32 C_{k+1} / C_nb)) for k < K */
/* and T[k] = 2^32 - 1 for k >= K.  Bin of a 32-bit word x: the first k < K   */
/* with x < T[k], else K.  Zero-weight bins are never chosen.                 */
/* ------------------------------------------------------------------------- */
int32_t orc_thresholds(const float* w, int32_t nb, uint32_t* T, int32_t* k_last) {
  double C = 0.0;
  int32_t K = -1;
  for (int32_t k = 0; k < nb; ++k) {
    C = C + (double)w[k];
    if (w[k] > 0.0f) K = k;
  }
  if (!(C > 0.0) || K < 0) return -1;
  double c = 0.0;
  for (int32_t k = 0; k < nb; ++k) {
    c = c + (double)w[k];
    if (k < K) {
      double t = floor((4294967296.0 * c) / C);
      if (t > 4294967295.0) t = 4294967295.0;
      T[k] = (uint32_t)t;
    } else {
      T[k] = 0xFFFFFFFFu;
    }
  }
  *k_last = K;
  return 0;
}

int32_t orc_sample_bin(const uint32_t* T, int32_t k_last, uint32_t x0) {
  for (int32_t k = 0; k < k_last; ++k)
    if (x0 < T[k]) return k;
  return k_last;
}

/* ------------------------------------------------------------------------- */
/* (r, alpha) -> (eta, phi) around the layer centre (Listing 1: extrapol).    */
/* Straight line from the origin: the layer centre is the particle's (eta,   */
/* phi).  Barrel layer at radius R: d(eta)/dz = 1/(R cosh eta), d(phi) =      */
/* dy/R.  End-cap layer at |z|: rho = |z| / sinh|eta|, d(eta)/d(rho) =        */
/* -sign(eta) tanh|eta| / rho, d(phi) = dy/rho.  r cos(alpha) runs along the  */
/* eta direction, r sin(alpha) along phi.                                     */
/* ------------------------------------------------------------------------- */
void orc_scales(const orc_geometry* g, int32_t layer, double eta_c, double* s_eta,
                double* s_phi) {
  const double R = g->layers[layer].rz;
  if (g->layers[layer].barrel) {
    *s_phi = 1.0 / R;
    *s_eta = 1.0 / (R * cosh(eta_c));
  } else {
    const double ae = fabs(eta_c);
    const double sh = sinh(ae);
    const double m = (tanh(ae) * sh) / R;
    *s_phi = sh / R;
    *s_eta = (eta_c < 0.0) ? m : -m;
  }
}

/* ------------------------------------------------------------------------- */
/* Cell lookup (Listing 2, getDDE).  Regions of a layer are sorted by eta_lo; */
/* region r owns eta in [s_r, s_{r+1}) where s_r is the midpoint between the  */
/* top of region r-1 (eta_lo + n_eta * deta) and eta_lo of region r (s of the */
/* first region is -inf), so a point in a gap or beyond the coverage goes to */
/* the nearest region.  i_eta = floor((eta - eta_lo) / deta) clamped to       */
/* [0, n_eta - 1]; i_phi = floor((phi - phi_lo) / dphi) mod n_phi.            */
/* cell = cell_offset + i_eta * n_phi + i_phi.                                */
/* ------------------------------------------------------------------------- */
static double region_split(const orc_geometry* g, int32_t r) {
  const orc_region* lo = &g->regions[r - 1];
  const double top = lo->eta_lo + (double)lo->n_eta * lo->deta;
  return 0.5 * (top + g->regions[r].eta_lo);
}

int32_t orc_cell(const orc_geometry* g, int32_t layer, double eta, double phi) {
  const int32_t rb = g->layer_region_begin[layer], re = g->layer_region_begin[layer + 1];
  int32_t r = rb;
  for (int32_t k = rb + 1; k < re; ++k)
    if (eta >= region_split(g, k)) r = k;
  const orc_region* R = &g->regions[r];
  const double te = (eta - R->eta_lo) / R->deta;
  int64_t ie;
  if (te < 0.0) ie = 0;
  else if (te >= (double)R->n_eta) ie = R->n_eta - 1;
  else ie = (int64_t)floor(te);
  if (ie > R->n_eta - 1) ie = R->n_eta - 1;
  double tp = (phi - R->phi_lo) / R->dphi;
  const double lim = 4503599627370496.0; /* 2^52 */
  if (tp > lim) tp = lim;
  if (tp < -lim) tp = -lim;
  int64_t ip = (int64_t)floor(tp) % (int64_t)R->n_phi;
  if (ip < 0) ip += R->n_phi;
  return R->cell_offset + (int32_t)ie * R->n_phi + (int32_t)ip;
}

void orc_cell_n(const orc_geometry* g, int64_t n, const int32_t* layer, const double* eta,
                const double* phi, int32_t* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = orc_cell(g, layer[i], eta[i], phi[i]);
}

/* ------------------------------------------------------------------------- */
/* Whole batch: for each event, particle, layer (in that order) a task with   */
/* E_l = fl32(E * f_l) (float, Listing 1), mu = fl32(E_l / mean hit energy),  */
/* n = max(1, Poisson(mu)) (at least one hit, Sec. 4), Ehit = fl32(E_l / n).  */
/* Layers with E_l == 0 have no task.  Hit h of a task draws Philox block     */
/* (h, layer, particle in event, event): word 0 picks the shape bin, words 1  */
/* and 2 the position in the bin (three numbers per hit, Sec. 4).  Energies   */
/* accumulate in FP64; the canonical FP32 value of a cell folds              */
/* fl32(fl32(n_cell,task) * Ehit) over tasks in ascending order from 0.0f.    */
/* ------------------------------------------------------------------------- */
int32_t orc_simulate(const orc_geometry* g, const orc_params* P, int64_t n_particles,
                     const int32_t* type, const float* E, const float* eta, const float* phi,
                     int32_t n_events, const int64_t* event_offsets, uint64_t seed,
                     int64_t first_event, orc_outputs* out) {
  if (P->NL != g->n_layers) return -1;
  if (event_offsets[0] != 0 || event_offsets[n_events] != n_particles) return -1;
  const int32_t NB = P->NR * P->NA;
  const int64_t n_entries = (int64_t)P->NT * P->NE * P->NH * P->NL;
  uint32_t* Tcache = (uint32_t*)malloc((size_t)n_entries * (size_t)NB * sizeof(uint32_t));
  int32_t* Kcache = (int32_t*)malloc((size_t)n_entries * sizeof(int32_t));
  int32_t* cnt = (int32_t*)calloc((size_t)g->n_cells, sizeof(int32_t));
  int32_t* touched = (int32_t*)malloc((size_t)g->n_cells * sizeof(int32_t));
  if (!Tcache || !Kcache || !cnt || !touched) {
    free(Tcache); free(Kcache); free(cnt); free(touched);
    return -1;
  }
  for (int64_t i = 0; i < n_entries; ++i) Kcache[i] = -2; /* not yet built */
  const uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
  int32_t status = 0;
  int64_t nt = 0, nh = 0;
  double E_layers = 0.0;

  for (int32_t e = 0; e < n_events; ++e) {
    const uint32_t ev = (uint32_t)(first_event + e);
    for (int64_t p = event_offsets[e]; p < event_offsets[e + 1]; ++p) {
      const uint32_t pin = (uint32_t)(p - event_offsets[e]);
      if (type[p] < 0 || type[p] >= P->NT || !(E[p] > 0.0f) || !isfinite(E[p]) ||
          !isfinite(eta[p]) || !isfinite(phi[p])) {
        status = -1;
        continue;
      }
      const int32_t base = orc_param_entry_rng(P, type[p], E[p], eta[p], key, pin, ev);
      for (int32_t l = 0; l < P->NL; ++l) {
        const int64_t entry = (int64_t)base * P->NL + l;
        const float El = E[p] * P->frac[entry];
        if (!(El > 0.0f)) continue;
        const float mu = El / P->mean_hit_E[entry];
        int64_t n = orc_poisson((double)mu, key, (uint32_t)l, pin, ev);
        if (n < 1) n = 1;
        const float Ehit = El / (float)n;
        if (Kcache[entry] == -2) {
          int32_t K = -1;
          if (orc_thresholds(P->shape_w + entry * NB, NB, Tcache + entry * NB, &K) != 0) K = -1;
          Kcache[entry] = K;
        }
        if (Kcache[entry] < 0) { status = -1; continue; }
        const uint32_t* T = Tcache + entry * NB;
        const int32_t K = Kcache[entry];
        if (nt < out->task_cap) {
          if (out->task_event) out->task_event[nt] = e;
          if (out->task_particle) out->task_particle[nt] = (int32_t)pin;
          if (out->task_layer) out->task_layer[nt] = l;
          if (out->task_n) out->task_n[nt] = (int32_t)n;
          if (out->task_Ehit) out->task_Ehit[nt] = Ehit;
        } else if (status == 0 && (out->task_event || out->task_particle || out->task_layer ||
                                   out->task_n || out->task_Ehit)) {
          status = -2;
        }
        E_layers += (double)El;
        double s_eta, s_phi;
        orc_scales(g, l, (double)eta[p], &s_eta, &s_phi);
        int32_t n_touched = 0;
        for (int64_t h = 0; h < n; ++h) {
          const uint32_t ctr[4] = {(uint32_t)h, (uint32_t)l | ((uint32_t)PURPOSE_HIT << 16), pin, ev};
          uint32_t x[4];
          orc_philox(ctr, key, x);
          const int32_t bin = orc_sample_bin(T, K, x[0]);
          const int32_t ir = bin / P->NA, ia = bin % P->NA;
          const double r_lo = (double)P->r_edges[ir], r_hi = (double)P->r_edges[ir + 1];
          const double a_lo = (double)P->a_edges[ia], a_hi = (double)P->a_edges[ia + 1];
          const double r = r_lo + u24(x[1]) * (r_hi - r_lo);
          const double alpha = a_lo + u24(x[2]) * (a_hi - a_lo);
          const double deta = (r * cos(alpha)) * s_eta;
          const double dphi = (r * sin(alpha)) * s_phi;
          const double heta = (double)eta[p] + deta;
          const double hphi = (double)phi[p] + dphi;
          const int32_t cell = orc_cell(g, l, heta, hphi);
          if (nh < out->hit_cap) {
            if (out->hit_cell) out->hit_cell[nh] = cell;
            if (out->hit_bin) out->hit_bin[nh] = (int16_t)bin;
            if (out->hit_eta) out->hit_eta[nh] = heta;
            if (out->hit_phi) out->hit_phi[nh] = hphi;
            if (out->hit_r) out->hit_r[nh] = r;
            if (out->hit_alpha) out->hit_alpha[nh] = alpha;
          } else if (status == 0 && (out->hit_cell || out->hit_bin || out->hit_eta ||
                                     out->hit_phi || out->hit_r || out->hit_alpha)) {
            status = -2;
          }
          nh += 1;
          if (out->cells64) out->cells64[(int64_t)e * g->n_cells + cell] += (double)Ehit;
          if (cnt[cell] == 0) touched[n_touched++] = cell;
          cnt[cell] += 1;
        }
        for (int32_t j = 0; j < n_touched; ++j) {
          const int32_t c = touched[j];
          if (out->cells_canon) {
            float* dst = &out->cells_canon[(int64_t)e * g->n_cells + c];
            const float add = (float)cnt[c] * Ehit;
            *dst = *dst + add;
          }
          cnt[c] = 0;
        }
        nt += 1;
      }
    }
  }
  out->n_tasks = nt;
  out->n_hits = nh;
  out->E_layers = E_layers;
  free(Tcache);
  free(Kcache);
  free(cnt);
  free(touched);
  return status;
}

/* ------------------------------------------------------------------------- */
/* Gradients by reweighting (the differentiable form of the hit loop).  For a */
/* seed, the base parametrisation fixes every hit: its task's count n, its    */
/* shape bin b and its cell.  Perturbed parameters change only the hits'     */
/* energies: E * f / n (FP64) for the layer fraction f of the task's entry,  */
/* times the shape likelihood ratio p_b(w) / p_b(w0) with p_b(w) = w_b /      */
/* sum(w).  walk_hits visits the hits in orc_simulate's order with the same  */
/* element functions.                                                         */
/* ------------------------------------------------------------------------- */
typedef struct orc_hit {
  int32_t event;  /* batch-local */
  int64_t entry;  /* parametrisation entry including the layer */
  int64_t n;      /* hits of the task */
  float E;        /* particle energy, MeV */
  int32_t bin, cell;
} orc_hit;

typedef void (*orc_hit_fn)(void* user, const orc_hit* h);

static int32_t walk_hits(const orc_geometry* g, const orc_params* P, int64_t n_particles,
                         const int32_t* type, const float* E, const float* eta, const float* phi,
                         int32_t n_events, const int64_t* event_offsets, uint64_t seed,
                         int64_t first_event, orc_hit_fn fn, void* user) {
  if (P->NL != g->n_layers) return -1;
  if (event_offsets[0] != 0 || event_offsets[n_events] != n_particles) return -1;
  const int32_t NB = P->NR * P->NA;
  uint32_t* T = (uint32_t*)malloc((size_t)NB * sizeof(uint32_t));
  if (!T) return -1;
  const uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
  int32_t status = 0;
  for (int32_t e = 0; e < n_events; ++e) {
    const uint32_t ev = (uint32_t)(first_event + e);
    for (int64_t p = event_offsets[e]; p < event_offsets[e + 1]; ++p) {
      const uint32_t pin = (uint32_t)(p - event_offsets[e]);
      if (type[p] < 0 || type[p] >= P->NT || !(E[p] > 0.0f) || !isfinite(E[p]) ||
          !isfinite(eta[p]) || !isfinite(phi[p])) {
        status = -1;
        continue;
      }
      const int32_t base = orc_param_entry_rng(P, type[p], E[p], eta[p], key, pin, ev);
      for (int32_t l = 0; l < P->NL; ++l) {
        const int64_t entry = (int64_t)base * P->NL + l;
        const float El = E[p] * P->frac[entry];
        if (!(El > 0.0f)) continue;
        const float mu = El / P->mean_hit_E[entry];
        int64_t n = orc_poisson((double)mu, key, (uint32_t)l, pin, ev);
        if (n < 1) n = 1;
        int32_t K = -1;
        if (orc_thresholds(P->shape_w + entry * NB, NB, T, &K) != 0) { status = -1; continue; }
        double s_eta, s_phi;
        orc_scales(g, l, (double)eta[p], &s_eta, &s_phi);
        orc_hit hit = {e, entry, n, E[p], 0, 0};
        for (int64_t h = 0; h < n; ++h) {
          const uint32_t ctr[4] = {(uint32_t)h, (uint32_t)l | ((uint32_t)PURPOSE_HIT << 16), pin, ev};
          uint32_t x[4];
          orc_philox(ctr, key, x);
          const int32_t bin = orc_sample_bin(T, K, x[0]);
          const int32_t ir = bin / P->NA, ia = bin % P->NA;
          const double r_lo = (double)P->r_edges[ir], r_hi = (double)P->r_edges[ir + 1];
          const double a_lo = (double)P->a_edges[ia], a_hi = (double)P->a_edges[ia + 1];
          const double r = r_lo + u24(x[1]) * (r_hi - r_lo);
          const double alpha = a_lo + u24(x[2]) * (a_hi - a_lo);
          const double heta = (double)eta[p] + (r * cos(alpha)) * s_eta;
          const double hphi = (double)phi[p] + (r * sin(alpha)) * s_phi;
          hit.bin = bin;
          hit.cell = orc_cell(g, l, heta, hphi);
          fn(user, &hit);
        }
      }
    }
  }
  free(T);
  return status;
}

static double weight_sum(const orc_params* P, int64_t entry) {
  const int32_t NB = P->NR * P->NA;
  double W = 0.0;
  for (int32_t k = 0; k < NB; ++k) W = W + (double)P->shape_w[entry * NB + k];
  return W;
}

typedef struct rw_ctx {
  const orc_params* P;
  int32_t n_cells;
  int64_t f_entry, w_entry;
  int32_t w_bin;
  double f_delta, w_delta, W0;
  double* cells;
} rw_ctx;

static void rw_hit(void* user, const orc_hit* h) {
  rw_ctx* c = (rw_ctx*)user;
  const int32_t NB = c->P->NR * c->P->NA;
  double f = (double)c->P->frac[h->entry];
  if (h->entry == c->f_entry) f = f + c->f_delta;
  double ratio = 1.0;
  if (h->entry == c->w_entry) {
    const double w0 = (double)c->P->shape_w[h->entry * NB + h->bin];
    const double w1 = w0 + (h->bin == c->w_bin ? c->w_delta : 0.0);
    ratio = (w1 / (c->W0 + c->w_delta)) / (w0 / c->W0);
  }
  c->cells[(int64_t)h->event * c->n_cells + h->cell] += (((double)h->E * f) / (double)h->n) * ratio;
}

int32_t orc_reweighted_cells(const orc_geometry* g, const orc_params* P, int64_t n_particles,
                             const int32_t* type, const float* E, const float* eta,
                             const float* phi, int32_t n_events, const int64_t* event_offsets,
                             uint64_t seed, int64_t first_event, int64_t f_entry, double f_delta,
                             int64_t w_entry, int32_t w_bin, double w_delta, double* cells) {
  rw_ctx c = {P, g->n_cells, f_entry, w_entry, w_bin, f_delta, w_delta, 1.0, cells};
  if (w_entry >= 0) c.W0 = weight_sum(P, w_entry);
  return walk_hits(g, P, n_particles, type, E, eta, phi, n_events, event_offsets, seed, first_event,
                   rw_hit, &c);
}

typedef struct bw_ctx {
  const orc_params* P;
  int32_t n_cells;
  const double* g;
  double* d_frac;
  double* A;
} bw_ctx;

static void bw_hit(void* user, const orc_hit* h) {
  bw_ctx* c = (bw_ctx*)user;
  const int32_t NB = c->P->NR * c->P->NA;
  const double gc = c->g[(int64_t)h->event * c->n_cells + h->cell];
  /* dE_hit / df = E / n; the hit energy itself weights the shape score */
  c->d_frac[h->entry] += ((double)h->E / (double)h->n) * gc;
  c->A[h->entry * NB + h->bin] += (((double)h->E * (double)c->P->frac[h->entry]) / (double)h->n) * gc;
}

/* d_frac, d_w: accumulated (the caller zeroes them).  With A[e][k] the sum of  */
/* E_hit * dL/dE_cell over the hits of entry e in bin k and W = sum(w[e]):     */
/*   dL/df[e]    = sum over its hits of (E / n) dL/dE_cell                     */
/*   dL/dw[e][k] = A[e][k] / w[e][k] - sum_j A[e][j] / W   (first term 0 when  */
/*                 w[e][k] == 0: such bins have no hits)                        */
int32_t orc_backward(const orc_geometry* g, const orc_params* P, int64_t n_particles,
                     const int32_t* type, const float* E, const float* eta, const float* phi,
                     int32_t n_events, const int64_t* event_offsets, uint64_t seed,
                     int64_t first_event, const double* dL_dcells, double* d_frac, double* d_w) {
  const int32_t NB = P->NR * P->NA;
  const int64_t n_entries = (int64_t)P->NT * P->NE * P->NH * P->NL;
  double* A = (double*)calloc((size_t)n_entries * (size_t)NB, sizeof(double));
  if (!A) return -1;
  bw_ctx c = {P, g->n_cells, dL_dcells, d_frac, A};
  const int32_t st = walk_hits(g, P, n_particles, type, E, eta, phi, n_events, event_offsets, seed,
                               first_event, bw_hit, &c);
  for (int64_t e = 0; e < n_entries; ++e) {
    double S = 0.0;
    int any = 0;
    for (int32_t k = 0; k < NB; ++k) {
      S = S + A[e * NB + k];
      any |= A[e * NB + k] != 0.0;
    }
    if (!any) continue;
    const double W = weight_sum(P, e);
    for (int32_t k = 0; k < NB; ++k) {
      const double w = (double)P->shape_w[e * NB + k];
      d_w[e * NB + k] += (w > 0.0 ? A[e * NB + k] / w : 0.0) - S / W;
    }
  }
  free(A);
  return st;
}
