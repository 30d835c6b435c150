/*
 * fcs.h - C ABI of the GB300 (sm_103a) parameterised calorimeter hit path.
 *
 * The library simulates the hot loop of FastCaloSim as ported to GPUs in
 * arXiv:2103.14737: for every particle, calorimeter layer and hit it draws
 * counter-based random numbers, picks the hit count and hit energy of the
 * selected parametrisation, samples the hit's (r, alpha) from a 2-D shape
 * histogram by inverse CDF, maps it to (eta, phi) around the particle's
 * direction, finds the cell (region search, then grid index) and adds the
 * hit energy into the cell array (Sec. 4, Listing 1; Sec. 7.3, Listing 2).
 * Many events run in one launch sequence, the paper's grouped simulation
 * (GPU_g, Sec. 4, last paragraph) taken to whole batches of events.
 *
 * Conventions for every entry point:
 *   - Return value: FCS_OK (0) or one of the FCS_E_* codes below; the text of
 *     the last error of the calling thread is available from
 *     fcs_last_error().  No entry point aborts the process.
 *   - Pointers documented "host" are read during the call only.  Pointers
 *     documented "device" must be CUDA device memory of the current device,
 *     owned by the caller (typically torch tensors); the library never frees
 *     them and reads or writes them only in work enqueued on the given
 *     stream.
 *   - Objects created by fcs_load_* / fcs_workspace_create belong to the
 *     library; release them with the matching fcs_free_* call after all work
 *     that uses them has completed.
 *   - Work is enqueued on the caller's stream `s` (may be 0 for the legacy
 *     default stream).  Calls with config->sync != 0 wait for that stream
 *     before returning and report device-side checks in their status; calls
 *     with sync == 0 return as soon as the work is enqueued and report
 *     device-side failures through fcs_workspace_status().
 *   - A workspace must not be used by two calls whose work overlaps on the
 *     GPU (two streams, or two host threads): it holds the intermediate
 *     buffers of one call.
 */
#ifndef FCS_H
#define FCS_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
enum fcs_status_code {
  FCS_OK = 0,
  FCS_E_ARG = 1,          /* invalid argument: NULL where required, bad size, bad table value */
  FCS_E_RANGE = 2,        /* an output or workspace capacity is too small (see each call) */
  FCS_E_OOM = 3,          /* a device allocation of the library failed */
  FCS_E_CUDA = 4,         /* a CUDA runtime call failed (message in fcs_last_error) */
  FCS_E_DEVICE_CHECK = 5, /* a device-side input check failed (bad particle type, NaN, ...) */
  FCS_E_TIMEOUT = 6,      /* a bounded device wait gave up (FCS_FLAG_WAIT_TIMEOUT) */
  FCS_E_UNSUPPORTED = 7   /* the call or option is not implemented */
};

/* Device-side check bits reported in fcs_stats.device_flags. */
enum fcs_device_flag {
  FCS_FLAG_BAD_PARTICLE = 1u << 0,  /* type out of range, E <= 0 or non-finite, eta/phi non-finite */
  FCS_FLAG_HIT_CAPACITY = 1u << 1,  /* more hits than the workspace was sized for (sync == 0) */
  FCS_FLAG_OUT_CAPACITY = 1u << 2,  /* more non-zero cells than `capacity` */
  FCS_FLAG_KEY_BITS = 1u << 3,      /* deterministic mode: (cell, task) keys need > 63 bits, or an
                                       event holds 2^27 tasks or more */
  FCS_FLAG_RECHECK_SPILL = 1u << 4, /* informational: FP64 recheck queue full, done inline */
  FCS_FLAG_BAD_OFFSETS = 1u << 5,   /* event_offsets not within [0, n_particles] or decreasing */
  FCS_FLAG_WAIT_TIMEOUT = 1u << 6   /* a bounded device wait gave up: the call's results are invalid */
};

/* ---- geometry (Sec. 4: 187,652 cells, 24 layers, 78 regions, flattened) -- */
/* One region: a regular eta x phi grid within one layer.  Cell (i_eta, i_phi)
 * of the region spans [eta_lo + i_eta*deta, eta_lo + (i_eta+1)*deta) x
 * [phi_lo + i_phi*dphi, ...) and has id cell_offset + i_eta*n_phi + i_phi.
 * 48 bytes, no padding. */
typedef struct fcs_region {
  double eta_lo, deta, phi_lo, dphi;
  int32_t n_eta, n_phi, cell_offset, layer;
} fcs_region;

/* One layer: barrel radius or end-cap |z| (mm) and a barrel flag. */
typedef struct fcs_layer_geom {
  double rz;
  int32_t barrel; /* 1 barrel (cylinder at radius rz), 0 end-cap (disk at |z| = rz) */
  int32_t pad;
} fcs_layer_geom;

typedef struct fcs_geo fcs_geo;             /* opaque, device-resident geometry */
typedef struct fcs_params fcs_params;       /* opaque, device-resident parametrisation */
typedef struct fcs_workspace fcs_workspace; /* opaque, device buffers of one call */

/* Particles of n_events events as device SoA; event e owns the particles
 * [event_offsets[e], event_offsets[e+1]).  type: 0 electron, 1 photon,
 * 2 charged pion (any value < NT of the parametrisation).  The four particle
 * arrays may be NULL when n_particles == 0; event_offsets is always required. */
typedef struct fcs_particles {
  const int32_t* type;          /* device [n_particles] */
  const float* E;               /* device [n_particles], MeV, > 0 */
  const float* eta;             /* device [n_particles] */
  const float* phi;             /* device [n_particles], rad */
  const int64_t* event_offsets; /* device [n_events + 1], event_offsets[0] = 0 */
} fcs_particles;

enum fcs_mode {
  FCS_MODE_ATOMIC = 0,       /* warp-aggregated atomics (Sec. 4: atomicAdd) of the float count x Ehit of
                                each group of hits into FP64 cells, rounded once to float per cell */
  FCS_MODE_DETERMINISTIC = 1 /* records (cell, task, count) grouped by cell, sorted by task and folded
                                in that order in FP32; bit-reproducible */
};

typedef struct fcs_config {
  int32_t mode;            /* enum fcs_mode */
  int32_t batched;         /* 1: events in launch sequences of wave_events; 0: one sequence per
                              event; 2: per event, one hit-kernel launch per task (the paper's
                              non-grouped GPU mode, Sec. 4; the call waits for the stream per
                              event to read the task list; no graph capture) */
  int32_t hits_per_thread; /* hit kernel: hits per thread per tile, 1, 2, 4 or 8; 0 = default (8) */
  int32_t block;           /* hit kernel: threads per block, 128, 256 or 512; 0 = default (128) */
  int32_t sync;            /* != 0: wait for the stream, read the device status (see above) */
  int32_t use_graph;       /* != 0 (requires sync == 0): capture the launch sequence as a CUDA
                              graph keyed by every argument, replay it on identical calls */
  int32_t timing;          /* != 0: record CUDA events around each stage (fcs_workspace_timings) */
  int32_t wave_events;     /* batched: events per launch sequence (a wave), >= 0; 0 = all events of
                              the call.  A wave's accumulation rows (FP64: 8 B x cells per event)
                              stay in L2 while they fit; the workspace holds one wave's rows */
  int32_t energy_interp;   /* 1: probabilistic energy-bin interpolation.  A particle of energy
                              E = m 2^k (m in [1, 2)) takes the next energy bin with probability
                              m - 1: when word 0 of Philox block (0, 2 << 16, particle in event,
                              event) is below (mantissa bits of E) << 9.  0: the bin of E */
  int32_t reserved;        /* must be 0 */
} fcs_config;

/* Filled by fcs_simulate_events when non-NULL and config->sync != 0. */
typedef struct fcs_stats {
  int64_t n_tasks;    /* (event, particle, layer) tasks with E_layer > 0 */
  int64_t n_hits;     /* total hits */
  int64_t n_nonzero;  /* non-zero cells over all events (the compacted output size) */
  int64_t n_recheck;  /* hits whose cell the FP32 path could not certify, decided in FP64 */
  uint32_t device_flags; /* enum fcs_device_flag bits */
  uint32_t n_poisson_fp64; /* hit-count draws with a decision the FP32 path could not certify */
} fcs_stats;

/* Optional per-task / per-hit dumps for validation (device pointers; NULL
 * entries are skipped).  Tasks are in (event, particle, layer) order, hits in
 * (task, hit index) order.  Entries beyond the capacities are not written. */
typedef struct fcs_debug {
  int64_t task_capacity;
  int32_t* task_event;    /* batch-local event index */
  int32_t* task_particle; /* particle index within its event */
  int32_t* task_layer;
  int32_t* task_n;        /* hits of the task */
  float* task_Ehit;       /* hit energy, MeV */
  int64_t hit_capacity;
  int32_t* hit_cell;      /* cell id of each hit */
  int16_t* hit_bin;       /* shape-histogram bin of each hit (ir * n_alpha + ia) */
} fcs_debug;

/* ---- entry points ---------------------------------------------------------- */

const char* fcs_version(void);

/* Copies the message of the calling thread's last error into buf (always
 * NUL-terminated when len > 0).  Returns the status code of that error. */
int fcs_last_error(char* buf, size_t len);

/* Geometry (Sec. 4: detector description flattened to arrays of structs;
 * Listing 2: getDDE).  regions: host [n_regions], sorted by layer, then by
 * eta_lo within a layer, non-overlapping, n_eta, n_phi >= 1, deta, dphi > 0,
 * cell ids contiguous (layer-major, region, i_eta, i_phi); layer_region_begin:
 * host [n_layers + 1]; layers: host [n_layers].  Limits: n_layers <= 32,
 * n_regions <= 256, n_eta <= 2^22 per region, cells < 2^31.  FCS_E_ARG if
 * the table breaks a rule.
 * Copies everything to the device on stream s and waits for it. */
int fcs_load_geometry(fcs_geo** out, const fcs_region* regions, int32_t n_regions,
                      const int32_t* layer_region_begin, int32_t n_layers,
                      const fcs_layer_geom* layers, cudaStream_t s);
int fcs_geometry_info(const fcs_geo* geo, int32_t* n_cells, int32_t* n_layers, int32_t* n_regions);
void fcs_free_geometry(fcs_geo* geo);

/* Parametrisation (Sec. 1 and Sec. 4: tables selected by particle type,
 * energy and eta, flattened and copied to the GPU once).  Host arrays:
 *   frac, mean_hit_E: [NT][NE][NH][NL] (NL = the geometry's layer count);
 *     per entry the layer energy fraction (>= 0) and mean hit energy (MeV,
 *     > 0 wherever frac > 0);
 *   shape_w: [NT][NE][NH][NL][NR][NA] histogram weights (>= 0, finite, with a
 *     positive sum wherever frac > 0); NR * NA must be 128 (16 x 8);
 *   r_edges: [NR + 1] increasing, from 0 (mm); a_edges: [NA + 1] increasing
 *     (rad) spanning at most [0, 2 pi].
 * Energy bin = clamp(floor(log2 E) - ebin_log2_min, 0, NE - 1); |eta| bin =
 * min(floor(|eta| * eta_bin_scale), NH - 1).  The inverse-CDF thresholds
 * and guide tables are built on the device.  Waits for stream s. */
int fcs_load_params(fcs_params** out, const fcs_geo* geo, const float* frac,
                    const float* mean_hit_E, const float* shape_w, const float* r_edges,
                    const float* a_edges, int32_t NT, int32_t NE, int32_t NH, int32_t NR,
                    int32_t NA, double eta_bin_scale, int32_t ebin_log2_min, cudaStream_t s);
/* Replaces the parametrisation's tables from DEVICE arrays of the shapes of
 * fcs_load_params (a training step's update); NULL keeps an array.  The new
 * values are checked on the device with fcs_load_params' rules first (the
 * call waits for stream s for that); on a violation it returns FCS_E_ARG and
 * nothing changes.  Then the copies and the rebuild of the inverse-CDF tables
 * are enqueued on s: the source arrays must stay valid until s reaches them,
 * and simulation calls on other streams must be ordered after them. */
int fcs_update_params(fcs_params* prm, const float* frac, const float* mean_hit_E,
                      const float* shape_w, cudaStream_t s);
void fcs_free_params(fcs_params* prm);

/* Workspace: the intermediate device buffers of a simulation call (task
 * records, tile map, FP64-recheck queue, accumulation array, sort keys).  The
 * library allocates them with cudaMalloc and grows them on demand during
 * sync calls: the first sync call on a workspace reads the hit count back
 * mid-call to size it; later sync calls run without that round trip and, if
 * a call outgrows the workspace, grow it and run the call once more.
 * fcs_workspace_reserve sizes them ahead of sync == 0 calls and graph
 * capture.  Pointers stay fixed until the next growth. */
int fcs_workspace_create(fcs_workspace** out);
int fcs_workspace_reserve(fcs_workspace* ws, const fcs_geo* geo, int64_t n_particles,
                          int32_t n_events, int64_t n_hits, int32_t mode);
/* Reads the device status of the last call on ws: waits for stream s, then
 * fills *stats (may be NULL) and returns the call's status, as a synchronous
 * call would.  This completes a call made with config->sync == 0, on the
 * device (fcs_simulate_events) or from host buffers (fcs_simulate_events_host).
 * s: the stream of that call. */
int fcs_workspace_status(fcs_workspace* ws, fcs_stats* stats, cudaStream_t s);

/* Kernel launches of one replay of the CUDA graph the workspace launched
 * last: a call with config->use_graph != 0, or a host-buffer call replayed in
 * waves (fcs_simulate_events_host).  The kernel nodes of the captured
 * graph.  n_kernels: host, written.  FCS_E_ARG when no call on ws has run as a
 * graph. */
int fcs_workspace_graph_kernels(const fcs_workspace* ws, int64_t* n_kernels);

/* Self-test of the bounded device waits (the single-pass scans' look-back):
 * runs a three-tile scan, in buffers of its own, in which one tile never
 * publishes its status, so that the next tile's wait gives up after its poll
 * limit (2^20 polls, about 0.2 s) and sets FCS_FLAG_WAIT_TIMEOUT.  Returns
 * FCS_E_TIMEOUT, the status a call returns when one of its waits gives up;
 * the device stays usable.  FCS_E_DEVICE_CHECK if the wait did not report
 * giving up.  ms: host, written: the kernel's time.  Synchronous. */
int fcs_selftest_wait_timeout(float* ms, cudaStream_t s);

/* Stage times of the last call on ws that ran with config->timing != 0, in
 * milliseconds, summed over its event ranges (CUDA events on the call's
 * stream; waits for them): ms[FCS_STAGE_TASKS] particle tasks, scans, task
 * records and tile map; ms[FCS_STAGE_HITS] the hit kernel; ms[FCS_STAGE_RECHECK]
 * the FP64 recheck; ms[FCS_STAGE_REDUCE] compaction or sort + fold;
 * ms[FCS_STAGE_TOTAL] all of them.  ms: host [FCS_N_STAGES].  FCS_E_ARG when
 * no timed call has run. */
enum fcs_stage {
  FCS_STAGE_TASKS = 0,
  FCS_STAGE_HITS = 1,
  FCS_STAGE_RECHECK = 2,
  FCS_STAGE_REDUCE = 3,
  FCS_STAGE_TOTAL = 4,
  FCS_N_STAGES = 5
};
int fcs_workspace_timings(fcs_workspace* ws, float* ms);
void fcs_workspace_free(fcs_workspace* ws);

/* Simulate n_events events (the hit loop of Listing 1 for every particle and
 * layer, the cell mapping and deposit of Listing 2).  Event e of this batch
 * uses random-stream event number first_event + e, so a batch split across
 * calls or GPUs gives the same cells.  Outputs (device, any may be NULL):
 *   cells_out: [n_events][n_cells] dense cell energies (MeV);
 *   cell_ids / cell_E: the non-zero cells of all events, event-major and
 *     ascending cell id within an event, at most `capacity` entries
 *     (Sec. 4: results gathered as {cell_id, E});
 *   event_offsets_out: [n_events + 1]; event e's cells are
 *     [event_offsets_out[e], event_offsets_out[e+1]).  When the output does
 *     not fit, nothing beyond capacity is written, event_offsets_out[n_events]
 *     holds the size needed and the call returns FCS_E_RANGE (sync) or sets
 *     FCS_FLAG_OUT_CAPACITY (async).
 * dbg: optional validation dumps (NULL in production).
 * Errors: FCS_E_ARG for bad arguments, FCS_E_RANGE as above, when a
 * sync == 0 call needs more workspace than reserved or for 2^24 or more
 * events in one call, and in deterministic mode when an event range (a wave)
 * has 2^31 or more hit slots, when its (cell, task) keys need more than 63
 * bits, or when one event holds 2^27 tasks or more (use smaller waves),
 * FCS_E_DEVICE_CHECK when
 * a particle fails its checks (its tasks are skipped), FCS_E_CUDA / OOM. */
int fcs_simulate_events(const fcs_geo* geo, const fcs_params* prm, fcs_workspace* ws,
                        const fcs_particles* particles, int64_t n_particles, int32_t n_events,
                        uint64_t seed, int64_t first_event, const fcs_config* config,
                        float* cells_out, int32_t* cell_ids, float* cell_E,
                        int64_t* event_offsets_out, int64_t capacity, fcs_stats* stats,
                        const fcs_debug* dbg, cudaStream_t s);

/* End-to-end form of fcs_simulate_events for callers holding host data: the
 * particle arrays (host SoA, same layout as fcs_particles, event_offsets on
 * the host) are copied to the device, simulated, and the compacted result
 * copied back into host cell_ids / cell_E / event_offsets_out (capacity
 * entries).  Synchronous, except as config->sync == 0 allows (below).  When
 * every output array is mapped pinned host memory (cudaMallocHost,
 * cudaHostAlloc(Mapped) or a registered range; the device address is taken
 * with cudaPointerGetAttributes), the compaction kernel writes the results
 * there directly and no device-to-host copy runs.
 * When the particle arrays are pinned too, the call is in atomic mode in one
 * launch sequence (wave_events 0), has at least two events and offsets from
 * 0 to n_particles, and the workspace has been sized by an earlier call, it
 * runs as waves of events on three streams (one CUDA graph, replayed while
 * the arguments stay the same): a wave's particles are copied in while the
 * wave before it computes, and a wave's results move to the host while the
 * next computes.  Two waves (3/4 and 1/4 of the events) below 512 events,
 * four (1/4 each) from 512 on.  Each wave has its own accumulation rows.
 * Pageable memory works through device staging and copies.
 * config->sync == 0 asks for a call that does not wait: when the call runs
 * as the wave graph above, it returns FCS_OK once the graph is enqueued
 * on s, with *stats zeroed, and fcs_workspace_status(ws, stats, s) waits for
 * it and returns its status and statistics (FCS_E_RANGE when the workspace
 * held fewer hits than the call produced: repeat the call synchronously).
 * Until then the call's host buffers and ws stay in use.  A serving loop
 * alternates two workspaces on two streams, so that one call's copies and
 * results overlap the other's compute.  Any other call runs synchronously
 * whatever config->sync says. */
int fcs_simulate_events_host(const fcs_geo* geo, const fcs_params* prm, fcs_workspace* ws,
                             const int32_t* type, const float* E, const float* eta,
                             const float* phi, const int64_t* event_offsets,
                             int64_t n_particles, int32_t n_events, uint64_t seed,
                             int64_t first_event, const fcs_config* config, int32_t* cell_ids,
                             float* cell_E, int64_t* event_offsets_out, int64_t capacity,
                             fcs_stats* stats, cudaStream_t s);

/* Autotuner of the hit kernel's launch shape (the grouped launch of Sec. 4
 * with a tunable tile).  Runs the call described by the arguments (device
 * pointers as for fcs_simulate_events; no outputs are kept) once for every
 * supported (threads per block, hits per thread) pair in {128, 256, 512} x
 * {1, 2, 4, 8}, `reps` timed repetitions each after one warm-up, and writes
 * the pair with the smallest median hit-kernel time into config->block and
 * config->hits_per_thread (config->mode selects the kernel variant; other
 * fields are ignored).  ms: optional host [12] array, median milliseconds in
 * the order block-major, hits-per-thread-minor.  Synchronous.  Errors as for
 * fcs_simulate_events. */
#define FCS_AUTOTUNE_SHAPES 12
int fcs_autotune(const fcs_geo* geo, const fcs_params* prm, fcs_workspace* ws,
                 const fcs_particles* particles, int64_t n_particles, int32_t n_events,
                 uint64_t seed, int64_t first_event, int32_t reps, fcs_config* config,
                 float* ms, cudaStream_t s);

/* Throughput microbenchmarks of the units the hit path uses (the roofline
 * denominators): kind FCS_MB_PHILOX = Philox4x32-10 blocks/s; FCS_MB_MULWIDE =
 * 32x32->64-bit integer multiplies/s (each followed by a 2-input XOR);
 * FCS_MB_LOP3 = shift + 3-input XOR + add steps/s; FCS_MB_FFMA = FP32 FMAs/s;
 * FCS_MB_RED = float reductions into global memory at uniformly random
 * addresses of a `size`-float array per second; FCS_MB_MUFU = hardware sines
 * (__sinf)/s; FCS_MB_LDS = 32-bit words/s read by 128-bit shared-memory loads;
 * FCS_MB_RED64 = double reductions at uniformly random addresses of a
 * `size`-double array per second (the accumulation rows' atomics).  A full grid (4 waves of
 * 256-thread blocks) runs `iters` iterations per thread, once to warm up and
 * once timed with CUDA events on stream s; *rate receives operations per
 * second.  Allocates and frees its own device buffer.  Synchronous. */
enum fcs_microbench_kind {
  FCS_MB_PHILOX = 0,
  FCS_MB_MULWIDE = 1,
  FCS_MB_LOP3 = 2,
  FCS_MB_FFMA = 3,
  FCS_MB_RED = 4,
  FCS_MB_MUFU = 5,
  FCS_MB_LDS = 6,
  FCS_MB_RED64 = 7
};
int fcs_microbench(int32_t kind, int64_t size, int32_t iters, double* rate, cudaStream_t s);

/* Audit of the Poisson hit counts (Listing 1, get_number_of_hits: n = Poisson(mu),
 * by inversion for mu < 10 and by PTRS above).  The library draws each count in
 * FP32 where every comparison is certified by an error bound, and in FP64 (the
 * definition) where one is not; this call runs both for n draws so that a test
 * can check the certified FP32 decisions against the FP64 ones on many more
 * draws than a CPU reference can.  Draw i has mean mu[i] and the Philox
 * counter fields of a task with layer i & 0xFF, particle i >> 8 and event 0,
 * under key `seed`.  Outputs (device, n entries each):
 *   n_fp32[i]: the FP32 count; -1 where an inversion decision was uncertain,
 *     -2 - i0 where PTRS iteration i0 was (the library then draws in FP64);
 *   n_fp64[i]: the FP64 definition's count (before max(1, n), clamped to
 *     2^31 - 1).
 * mu: device, n positive finite means (callers' responsibility; others give
 * counts without meaning).  prm must live on the current device.
 * Synchronous on stream s.  Errors: FCS_E_ARG, FCS_E_CUDA. */
int fcs_poisson_audit(const fcs_params* prm, const float* mu, int64_t n, uint64_t seed,
                      int32_t* n_fp32, int32_t* n_fp64, cudaStream_t s);

/* Size of the library's static device scratch used by
 * fcs_simulate_events_static (16 MiB, held on every GPU that loads the
 * library until the process exits). */
#define FCS_STATIC_SCRATCH_BYTES (16 * 1024 * 1024)

/* Atomic-mode, batched fcs_simulate_events that allocates no device memory,
 * for callers that must not call cudaMalloc/cudaFree while they run: online
 * trigger or serving loops that cannot take the device-wide synchronisation
 * an allocation can cause, processes whose device memory is fully reserved by
 * another framework's pool, or clients running under a memory quota.  This
 * entry point has no counterpart in the paper; it only changes where the
 * intermediate buffers live.
 * Inputs and outputs are as for fcs_simulate_events (device pointers; the
 * dense cells_out and the validation dumps are not offered; n_events == 0
 * writes event_offsets_out[0] = 0, zeroes *stats and returns FCS_OK); the task
 * records, tile map, recheck queue and accumulation rows are carved out of
 * one static device array of FCS_STATIC_SCRATCH_BYTES.  The call is
 * synchronous on stream s and returns the device status like a sync call.
 * Limits: the particle tables (about 52 bytes x layers + 32 bytes per particle) plus the
 * accumulation rows (8 bytes x cells, padded, per event) must fit in the
 * array, and the hits of the call are bounded by what remains (128 hits per
 * 4 remaining bytes); otherwise FCS_E_RANGE with the sizes in the message.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * Every call uses the same array: calls that overlap on the GPU (two streams
 * or two threads) race and corrupt each other's results. */
int fcs_simulate_events_static(const fcs_geo* geo, const fcs_params* prm,
                               const fcs_particles* particles, int64_t n_particles,
                               int32_t n_events, uint64_t seed, int64_t first_event,
                               int32_t* cell_ids, float* cell_E, int64_t* event_offsets_out,
                               int64_t capacity, fcs_stats* stats, cudaStream_t s);

/* Adjoint of fcs_simulate_events: the gradient of a loss L of the dense cell
 * energies with respect to the layer-fraction table and the shape weights.
 * The hit energy E_hit = E f_l / n of Sec. 4 (Listing 1) is the only place
 * where the parameters enter once the seed fixes each hit's task, count n,
 * shape bin b and cell; the fraction enters linearly (dE_hit/df_l = E / n)
 * and the shape weights through the likelihood ratio p_b(w) / p_b(w0) of the
 * drawn bin, p_b = w_b / sum(w).  With A[e][b] = the sum of E_hit dL/dE_cell
 * over entry e's hits drawn in bin b (FP64):
 *   d_frac[e]       += sum_b A[e][b] / frac[e]
 *   d_shape_w[e][b] += A[e][b] / w_b - sum_j A[e][j] / sum_j w_j
 *                      (the first term is 0 where w_b = 0: no hits there)
 * Only entries that received hits change.  Hits are regenerated on the
 * device exactly as by the forward call with the same seed, first_event and
 * particles (FP64 recheck included), so no hit list is stored.
 *   dL_dcells: device [n_events][n_cells] FP32, the layout of cells_out.
 *   d_frac: device, shaped like frac; d_shape_w: device, shaped like
 *     shape_w; FP32, accumulated into (the caller zeroes them); either may
 *     be NULL.
 *   config: mode is ignored; batched, hits_per_thread, block and sync as for
 *     fcs_simulate_events; use_graph must be 0; timing is ignored.
 *   stats: host, optional (n_tasks, n_hits, n_recheck, device_flags).
 * The scores use a FP64 array of the workspace (8 bytes x 128 x entries),
 * allocated by the first call.  With sync != 0 the call waits for the stream
 * and returns the device status like fcs_simulate_events; with sync == 0 it
 * returns after enqueueing (the workspace must be reserved) and
 * fcs_workspace_status reports the status.  On a device error the gradients
 * are incomplete.  FCS_E_RANGE if n_events (batched) x n_cells >= 2^32. */
int fcs_simulate_backward(const fcs_geo* geo, const fcs_params* prm, fcs_workspace* ws,
                          const fcs_particles* particles, int64_t n_particles,
                          int32_t n_events, uint64_t seed, int64_t first_event,
                          const fcs_config* config, const float* dL_dcells, float* d_frac,
                          float* d_shape_w, fcs_stats* stats, cudaStream_t s);

#ifdef __cplusplus
}
#endif
#endif /* FCS_H */
