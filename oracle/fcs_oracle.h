/*
 * fcs_oracle.h - plain single-threaded FP64 oracle of the parameterised
 * calorimeter hit path (arXiv:2103.14737, Sec. 4 and Listing 1).
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle exists to check the CUDA library; it
 * shares no code, header or table with it.  Only the tests, the smoke entry
 * and the benchmark's CPU-baseline leg may load it.
 *
 * All functions are pure, single threaded and allocate only what they free
 * before returning.  Floating-point work is FP64 except where the paper fixes
 * FP32 (the layer energy and hit energy are floats in Listing 1); the file is
 * compiled with -ffp-contract=off so that every FP32 step rounds once.
 */
#ifndef FCS_ORACLE_H
#define FCS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Geometry as the library receives it: regions sorted by (layer, eta_lo). */
typedef struct orc_region {
  double eta_lo, deta, phi_lo, dphi;
  int32_t n_eta, n_phi, cell_offset, layer;
} orc_region;

typedef struct orc_layer {
  double rz;      /* barrel radius or end-cap |z|, mm */
  int32_t barrel; /* 1 barrel, 0 end-cap */
  int32_t pad;
} orc_layer;

typedef struct orc_geometry {
  int32_t n_layers, n_regions, n_cells;
  const orc_region* regions;
  const int32_t* layer_region_begin; /* [n_layers + 1] */
  const orc_layer* layers;           /* [n_layers] */
} orc_geometry;

typedef struct orc_params {
  int32_t NT, NE, NH, NL, NR, NA;
  const float* frac;       /* [NT][NE][NH][NL] */
  const float* mean_hit_E; /* [NT][NE][NH][NL] */
  const float* shape_w;    /* [NT][NE][NH][NL][NR][NA] */
  const float* r_edges;    /* [NR + 1] */
  const float* a_edges;    /* [NA + 1] */
  double eta_bin_scale;    /* eta bins per unit |eta| */
  int32_t ebin_log2_min;   /* energy bin 0 starts at 2^ebin_log2_min MeV */
  int32_t energy_interp;   /* 1: probabilistic energy-bin interpolation (orc_energy_bin) */
} orc_params;

const char* orc_version(void);

/* Philox4x32-10 block cipher (Salmon et al., SC'11). */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Vector form for tests: n blocks, ctr and out as [n][4]. */
void orc_philox_n(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out);

/* Poisson draw used for the per-layer hit count (Listing 1, get_number_of_hits). */
int64_t orc_poisson(double mu, const uint32_t key[2], uint32_t layer, uint32_t particle,
                    uint32_t event);
void orc_poisson_n(int64_t n, const double* mu, const uint32_t key[2], const uint32_t* layer,
                   const uint32_t* particle, const uint32_t* event, int64_t* out);
/* One iteration of the PTRS draw (mu >= 10) from given uniforms u[i], V[i]:
 * the accepted count, or -1 where the iteration rejects. */
void orc_ptrs_iter_n(int64_t n, double mu, const double* u, const double* V, int64_t* out);

/* Parametrisation entry (without the layer index) for a particle. */
int32_t orc_param_entry(const orc_params* P, int32_t type, float E, float eta);
/* The same with the energy bin interpolated when P->energy_interp: E = m 2^k
 * (m in [1, 2)) lies the fraction x = m - 1 of the way from the bin's point
 * 2^k to the next bin's 2^(k+1), and takes the next bin when the uniform
 * u = x0 2^-32 of Philox block (0, 2 << 16, particle in event, event) is
 * below x (exact in FP64); subnormal E keeps its bin. */
int32_t orc_param_entry_rng(const orc_params* P, int32_t type, float E, float eta, const uint32_t key[2],
                            uint32_t particle, uint32_t event);

/* Inverse-CDF thresholds of one shape histogram; returns -1 if all weights are 0. */
int32_t orc_thresholds(const float* w, int32_t nb, uint32_t* T, int32_t* k_last);
int32_t orc_sample_bin(const uint32_t* T, int32_t k_last, uint32_t x0);

/* Per-task (r, alpha) -> (eta, phi) scale factors. */
void orc_scales(const orc_geometry* g, int32_t layer, double eta_c, double* s_eta,
                double* s_phi);

/* Cell of a point in a layer (region search then grid index). */
int32_t orc_cell(const orc_geometry* g, int32_t layer, double eta, double phi);
void orc_cell_n(const orc_geometry* g, int64_t n, const int32_t* layer, const double* eta,
                const double* phi, int32_t* out);

/* Whole-batch simulation.  Any output pointer may be NULL.  Returns 0, or -1
 * for invalid input, or -2 when task_cap / hit_cap were too small (counting
 * continues; only the capped dumps are truncated). */
typedef struct orc_outputs {
  double* cells64;    /* [n_events][n_cells], accumulated (caller zeroes) */
  float* cells_canon; /* [n_events][n_cells], canonical FP32 fold (caller zeroes) */
  int64_t task_cap;
  int32_t* task_event, *task_particle, *task_layer, *task_n;
  float* task_Ehit;
  int64_t hit_cap;
  int32_t* hit_cell;
  int16_t* hit_bin;
  double* hit_eta, *hit_phi, *hit_r, *hit_alpha;
  int64_t n_tasks, n_hits; /* written */
  double E_layers;         /* sum over tasks of the FP32 layer energy (FP64 sum) */
} orc_outputs;

int32_t orc_simulate(const orc_geometry* g, const orc_params* P, int64_t n_particles,
                     const int32_t* type, const float* E, const float* eta, const float* phi,
                     int32_t n_events, const int64_t* event_offsets, uint64_t seed,
                     int64_t first_event, orc_outputs* out);

/* Differentiable form (gradients by reweighting hit energies, hit positions
 * held fixed for the seed).  orc_reweighted_cells: FP64 cells [n_events][n_cells]
 * (accumulated) of the hits of P with the layer fraction of entry f_entry
 * moved by f_delta and the weight of (w_entry, w_bin) moved by w_delta
 * (entries < 0: no change).  orc_backward: gradients of a loss with the given
 * dL/dE_cell [n_events][n_cells] with respect to the layer fractions
 * [entries] and shape weights [entries][NR * NA] (accumulated). */
int32_t orc_reweighted_cells(const orc_geometry* g, const orc_params* P, int64_t n_particles,
                             const int32_t* type, const float* E, const float* eta,
                             const float* phi, int32_t n_events, const int64_t* event_offsets,
                             uint64_t seed, int64_t first_event, int64_t f_entry, double f_delta,
                             int64_t w_entry, int32_t w_bin, double w_delta, double* cells);
int32_t orc_backward(const orc_geometry* g, const orc_params* P, int64_t n_particles,
                     const int32_t* type, const float* E, const float* eta, const float* phi,
                     int32_t n_events, const int64_t* event_offsets, uint64_t seed,
                     int64_t first_event, const double* dL_dcells, double* d_frac, double* d_w);

#ifdef __cplusplus
}
#endif
#endif
