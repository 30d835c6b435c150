// fcs_api.cu - the C ABI of include/fcs.h: argument validation, device
// residency of geometry and parametrisation, the workspace, and the launch
// sequence of a simulation call:
//   per event range: range setup -> particle task counts -> task-offset scan
//   -> task records -> Poisson counts (FP32, then the deferred FP64 draws) ->
//   hit-offset scan with the tile map -> hit kernel -> FP64 recheck ->
//   compaction (atomic) or sort + fold (deterministic)
// between a starting and a finishing kernel.  Batched calls use one range for
// all events (the grouped simulation of Sec. 4) or waves of events; per-event
// calls use one range per event, as the paper's per-event GPU path did.  No
// launch depends on a host-read size except in sync calls, which read the hit
// count once to size the workspace.  Host-buffer calls with pinned buffers run
// as two waves on three streams so that the transfers overlap the compute.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <vector>

#include "fcs_internal.cuh"

using namespace fcs;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
namespace {
thread_local int g_err_code = FCS_OK;
thread_local char g_err_msg[512] = "";

int set_err(int code, const char* fmt, ...) {
  g_err_code = code;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err_msg, sizeof(g_err_msg), fmt, ap);
  va_end(ap);
  return code;
}
int ok() {
  g_err_code = FCS_OK;
  g_err_msg[0] = 0;
  return FCS_OK;
}
}  // namespace

#define FCS_CUDA(expr)                                                                     \
  do {                                                                                     \
    cudaError_t _e = (expr);                                                               \
    if (_e != cudaSuccess) {                                                               \
      if (_e == cudaErrorMemoryAllocation) {                                               \
        (void)cudaGetLastError();                                                          \
        return set_err(FCS_E_OOM, "%s: %s", #expr, cudaGetErrorString(_e));                \
      }                                                                                    \
      return set_err(FCS_E_CUDA, "%s (%s:%d): %s", #expr, __FILE__, __LINE__,              \
                     cudaGetErrorString(_e));                                              \
    }                                                                                      \
  } while (0)

#define FCS_TRY(expr)               \
  do {                              \
    int _rc = (expr);               \
    if (_rc != FCS_OK) return _rc;  \
  } while (0)

// ---------------------------------------------------------------------------
// opaque objects
// ---------------------------------------------------------------------------
struct fcs_geo {
  int device = -1;
  GeoDev d{};
  std::vector<void*> allocs;
  ~fcs_geo() {
    for (void* p : allocs) cudaFree(p);
  }
};

struct fcs_params {
  int device = -1;
  ParamDev d{};
  float* w = nullptr;           // device shape weights (the tables' source)
  int32_t* bad = nullptr;       // per-entry flags of the table build
  uint32_t* check = nullptr;    // validation word of fcs_update_params
  std::vector<void*> allocs;
  ~fcs_params() {
    for (void* p : allocs) cudaFree(p);
  }
};

namespace {
template <typename T>
int dev_alloc(T** p, size_t n, std::vector<void*>* owner = nullptr) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *p = nullptr;
    return set_err(e == cudaErrorMemoryAllocation ? FCS_E_OOM : FCS_E_CUDA, "cudaMalloc(%zu bytes): %s",
                   n * sizeof(T), cudaGetErrorString(e));
  }
  if (owner) owner->push_back((void*)*p);
  return FCS_OK;
}

// Grows a library-owned buffer to at least `need` elements (contents lost).
template <typename T>
int grow(T** p, int64_t* cap, int64_t need, bool zero = false) {
  if (need <= *cap && *p) return FCS_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const int64_t n = std::max<int64_t>(need, 1);
  FCS_TRY(dev_alloc(p, (size_t)n));
  if (zero) FCS_CUDA(cudaMemset(*p, 0, (size_t)n * sizeof(T)));
  *cap = n;
  return FCS_OK;
}

int bits_for(int64_t n) {  // bits to hold values 0 .. n - 1
  int b = 1;
  while (b < 63 && (int64_t(1) << b) < n) ++b;
  return b;
}

int current_device(int* dev) {
  FCS_CUDA(cudaGetDevice(dev));
  return FCS_OK;
}
}  // namespace

// Host-buffer calls run in waves of events (host_waves).  The shares, in
// eighths of the call's events: the first waves' results move over the link
// while the later waves compute, and only the last wave's results move after
// the last kernel.  Each wave repeats about 0.12 ms of latency-bound kernels,
// so small calls take two waves and large ones four.  Measured on 64
// pile-up events (one call at a time): 6/8 2/8 took 1.54 ms per call against
// 1.62-1.64 ms for splits of 2/3, 5/6 and 7/8, 1.68 ms on one stream, and
// 1.70-1.81 ms for three or four waves.  On 1024 events (the serving loop of
// two workspaces, the compaction on a third of the SMs): four waves of 2/8
// took 17.7 ms per call against 18.4 ms for 4/8 2/8 2/8, 19.0-19.6 ms for
// 6/8 2/8 and 18.2-18.8 ms for eight waves of 1/8.
constexpr int kHostWaveEighths[] = {6, 2};
constexpr int kHostWaveEighthsLarge[] = {2, 2, 2, 2};
constexpr int32_t kHostLargeEvents = 512;  // calls of this many events or more take the large table
constexpr int kMaxHostWaves = 4;
static_assert(sizeof(kHostWaveEighths) / sizeof(int) <= kMaxHostWaves &&
                  sizeof(kHostWaveEighthsLarge) / sizeof(int) <= kMaxHostWaves,
              "wave tables");

struct fcs_workspace {
  int device = -1;
  int num_sms = 0;
  Sizes* d_sizes = nullptr;
  Sizes* h_sizes = nullptr;  // pinned mirror
  int64_t sizes_cap = 0;
  int64_t* pcount = nullptr;
  int64_t* poff = nullptr;
  uint4* pinfo = nullptr;
  int64_t pc_cap = 0, po_cap = 0, pi_cap = 0, pcap = 0;
  TaskRec* tasks = nullptr;
  float* tehit = nullptr;
  int32_t* tn = nullptr;
  int64_t* th = nullptr;
  int32_t* pdefer = nullptr;
  int64_t task_cap = 0, tehit_cap = 0, tn_cap = 0, th_cap = 0, tl_cap = 0, pd_cap = 0;
  int32_t* gmap = nullptr;
  int64_t gmap_cap = 0;
  uint2* recheck = nullptr;
  int64_t recheck_cap = 0;
  double* acc = nullptr;  // FP64 accumulation rows
  int64_t acc_cap = 0, rows_cap = 0;
  int32_t acc_stride = 0;
  uint64_t* scan_state = nullptr;  // zero between scans (see ScanTmp)
  int64_t ss_cap = 0;
  uint64_t* keys = nullptr;
  uint64_t* keys_alt = nullptr;
  int64_t k_cap = 0, ka_cap = 0, rec_cap = 0;
  int64_t* cell_off = nullptr;  // deterministic mode: each cell's first record
  int64_t co_cells_cap = 0;
  // gradient scores [n_entries][128] (FP64) and their entry flags; zero
  // between backward calls (the finalize kernel clears what it reads)
  double* grad_acc = nullptr;
  uint8_t* grad_touched = nullptr;
  int64_t ga_cap = 0, gt_cap = 0;
  bool grad_dirty = false;  // a backward call stopped before its finalize
  // staging for the host-buffer entry point
  void* stage = nullptr;
  int64_t stage_cap = 0;
  // pinned copy of a range's first hits and hit counts (per-task launches)
  int64_t* h_tasks = nullptr;
  int64_t h_tasks_cap = 0;
  // CUDA graph cache (use_graph)
  cudaGraphExec_t graph = nullptr;
  std::vector<unsigned char> graph_key;
  int64_t graph_kernels = 0;     // kernel nodes of the cached graph
  int64_t launched_kernels = 0;  // kernel nodes of the graph launched last (either cache)
  // stage timing events: 5 per event range (begin, after tasks, after hits,
  // after recheck, after reduce) of the last timed call; recorded as external
  // events so that a captured call gets event-record nodes in its graph
  std::vector<cudaEvent_t> tev;
  int timed_ranges = 0;
  // host-buffer calls in waves: the copy-in and output streams, their
  // fork/join events, the output stream's scan state and the cached graph
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t pev[2 * kMaxHostWaves + 2] = {};
  uint64_t* scan_state2 = nullptr;
  int64_t ss2_cap = 0;
  cudaGraphExec_t pgraph = nullptr;
  std::vector<unsigned char> pgraph_key;
  int64_t pgraph_kernels = 0;

  ~fcs_workspace() {
    if (graph) cudaGraphExecDestroy(graph);
    if (pgraph) cudaGraphExecDestroy(pgraph);
    for (cudaEvent_t e : tev) cudaEventDestroy(e);
    for (cudaEvent_t e : pev)
      if (e) cudaEventDestroy(e);
    if (s_in) cudaStreamDestroy(s_in);
    if (s_out) cudaStreamDestroy(s_out);
    if (scan_state2) cudaFree(scan_state2);
    void* ps[] = {d_sizes, pcount, poff, pinfo, tasks, tehit, tn, th, pdefer, gmap,
                  recheck, acc, scan_state, keys, keys_alt, cell_off, stage, grad_acc, grad_touched};
    for (void* p : ps)
      if (p) cudaFree(p);
    if (h_sizes) cudaFreeHost(h_sizes);
    if (h_tasks) cudaFreeHost(h_tasks);
  }

  WsDev view() const {
    WsDev w{};
    w.sizes = d_sizes;
    w.pcount = pcount;
    w.poff = poff;
    w.pinfo = pinfo;
    w.pcap = pcap;
    w.tasks = tasks;
    w.tehit = tehit;
    w.tn = tn;
    w.th = th;
    w.pdefer = pdefer;
    w.gmap = gmap;
    w.recheck = recheck;
    w.acc = acc;
    w.task_cap = task_cap;
    w.gmap_cap = gmap_cap;
    w.recheck_cap = recheck_cap;
    w.rows_cap = rows_cap;
    w.pdefer_cap = pd_cap;
    w.keys = keys;
    w.keys_alt = keys_alt;
    w.rec_cap = rec_cap;
    return w;
  }

  ScanTmp scan_tmp() const {
    // three 256-thread CTAs per SM: the scans' 76 registers and 35 KB of tile buffer allow it
    return ScanTmp{scan_state, ss_cap - 2, d_sizes ? &d_sizes->flags : nullptr, num_sms * 3};
  }
};

namespace {

// Sizes every buffer that depends only on host-known quantities.
int ws_reserve_static(fcs_workspace* ws, const fcs_geo* geo, int64_t P, int32_t rows, int mode) {
  if (ws->device < 0) {
    FCS_TRY(current_device(&ws->device));
    FCS_CUDA(cudaDeviceGetAttribute(&ws->num_sms, cudaDevAttrMultiProcessorCount, ws->device));
  }
  if (!ws->d_sizes) {
    FCS_TRY(grow(&ws->d_sizes, &ws->sizes_cap, 1, true));
    FCS_CUDA(cudaMallocHost((void**)&ws->h_sizes, sizeof(Sizes)));
    std::memset(ws->h_sizes, 0, sizeof(Sizes));
  }
  const int NL = geo->d.n_layers;
  const int64_t Pc = std::max<int64_t>(P, 1);
  if (Pc > ws->pcap || !ws->pcount) {
    FCS_TRY(grow(&ws->pcount, &ws->pc_cap, Pc));
    FCS_TRY(grow(&ws->poff, &ws->po_cap, Pc));
    FCS_TRY(grow(&ws->pinfo, &ws->pi_cap, Pc));
    ws->pcap = Pc;
  }
  FCS_TRY(grow(&ws->tasks, &ws->task_cap, Pc * NL));
  FCS_TRY(grow(&ws->tehit, &ws->tehit_cap, Pc * NL));
  FCS_TRY(grow(&ws->tn, &ws->tn_cap, Pc * NL));
  FCS_TRY(grow(&ws->th, &ws->th_cap, Pc * NL));
  FCS_TRY(grow(&ws->pdefer, &ws->pd_cap, Pc * NL));
  const int32_t stride = geo->d.acc_stride;
  if (stride != ws->acc_stride || rows > ws->rows_cap || !ws->acc) {
    int64_t cap = 0;
    if (ws->acc) cudaFree(ws->acc);
    ws->acc = nullptr;
    ws->acc_cap = 0;
    FCS_TRY(grow(&ws->acc, &cap, (int64_t)std::max(rows, 1) * stride, true));
    ws->acc_cap = cap;
    ws->rows_cap = std::max(rows, 1);
    ws->acc_stride = stride;
  }
  const int64_t chunks = compact_chunks(geo->d.n_cells, std::max(rows, 1));
  // scan state for the largest array any scan of a call covers, and a status
  // word per compaction chunk (zeroed; the scans and the compaction leave it
  // zero)
  FCS_TRY(grow(&ws->scan_state, &ws->ss_cap,
               std::max(scan_state_words(std::max({Pc * NL, (int64_t)std::max(rows, 1) * stride, chunks})), chunks + 2),
               true));
  if (mode == FCS_MODE_DETERMINISTIC)
    FCS_TRY(grow(&ws->cell_off, &ws->co_cells_cap, (int64_t)std::max(rows, 1) * (stride + 1)));
  return FCS_OK;
}

// Sizes the hit-dependent buffers for H hits.
int ws_reserve_hits(fcs_workspace* ws, int64_t H, int mode) {
  const int64_t g = H / kGranule + 2;
  if (g > ws->gmap_cap) FCS_TRY(grow(&ws->gmap, &ws->gmap_cap, g + g / 4));
  const int64_t rq = std::max<int64_t>(1 << 16, H / 16);
  if (rq > ws->recheck_cap) FCS_TRY(grow(&ws->recheck, &ws->recheck_cap, rq + rq / 4));
  if (mode == FCS_MODE_DETERMINISTIC) {
    // the cells' segment offsets are int32: at most 2^31 - 1 record slots
    const int64_t kMaxSlots = INT32_MAX;
    const int64_t need = std::max<int64_t>(H, 1) + kRecordSlack;
    if (need > kMaxSlots)
      return set_err(FCS_E_RANGE, "deterministic mode: %lld hits in one event range exceed 2^31 record slots; use "
                     "smaller waves", (long long)H);
    if (need > ws->rec_cap) {
      const int64_t cap = std::min(need + need / 8, kMaxSlots);
      int64_t c1 = ws->k_cap, c2 = ws->ka_cap;
      FCS_TRY(grow(&ws->keys, &c1, cap));
      FCS_TRY(grow(&ws->keys_alt, &c2, cap));
      ws->k_cap = c1;
      ws->ka_cap = c2;
      ws->rec_cap = cap;
    }
  }
  return FCS_OK;
}

// ---- small kernels of the launch sequence ----------------------------------
__global__ void k_call_begin(Sizes* s) {
  Sizes z{};
  *s = z;
}

// One block of kRangeThreads: the range's offsets are checked in parallel
// (non-decreasing, within [0, n_particles] and the particle capacity), then
// thread 0 resets the range's counters.
constexpr int kRangeThreads = 256;
__global__ void __launch_bounds__(kRangeThreads) k_range_begin(Sizes* s, const int64_t* __restrict__ off,
                                                               int32_t ev_lo, int32_t ev_hi, int64_t n_particles,
                                                               int64_t pcap) {
  bool bad = false;
  for (int32_t e = ev_lo + (int32_t)threadIdx.x; e < ev_hi; e += kRangeThreads) bad |= off[e + 1] < off[e];
  bad = __syncthreads_or(bad);
  if (threadIdx.x != 0) return;
  const int64_t a = off[ev_lo], b = off[ev_hi];
  bad = bad || a < 0 || b < a || b > n_particles || (b - a) > pcap;
  s->n_part = bad ? 0 : (b - a);
  if (bad) s->flags |= FCS_FLAG_BAD_OFFSETS;
  s->n_tasks = 0;
  s->n_hits = 0;
  s->n_recheck = 0;
  s->n_records = 0;
  s->n_slots = 0;
  s->n_big = 0;
  s->n_mid = 0;
  s->n_mid32 = 0;
  s->n_pdefer = 0;
  s->n_pdefer_ptrs = 0;
  s->queue = 0;
}

__global__ void k_range_end(Sizes* s) {
  s->task_base += s->n_tasks;
  s->hit_base += s->n_hits;
  s->recheck_total += s->n_recheck;
}

__global__ void k_call_end(Sizes* s, int64_t* event_offsets_out, int32_t n_events, int64_t capacity,
                           int32_t want_cells) {
  if (event_offsets_out) event_offsets_out[n_events] = s->nnz_total;
  if (want_cells && s->nnz_total > capacity) s->flags |= FCS_FLAG_OUT_CAPACITY;
}

__global__ void k_empty_offsets(int64_t* event_offsets_out, int32_t n_events) {
  for (int i = threadIdx.x; i <= n_events; i += blockDim.x) event_offsets_out[i] = 0;
}

int status_from(const Sizes& s, fcs_stats* st) {
  if (st) {
    st->n_tasks = s.task_base;
    st->n_hits = s.hit_base;
    st->n_nonzero = s.nnz_total;
    st->n_recheck = s.recheck_total;
    st->device_flags = s.flags;
    st->n_poisson_fp64 = s.n_poisson_fp64;
  }
  if (s.flags & FCS_FLAG_WAIT_TIMEOUT)
    return set_err(FCS_E_TIMEOUT, "a bounded device wait gave up; the call's results are invalid");
  if (s.flags & FCS_FLAG_BAD_OFFSETS)
    return set_err(FCS_E_ARG, "event_offsets must be non-decreasing within [0, n_particles]");
  if (s.flags & FCS_FLAG_BAD_PARTICLE)
    return set_err(FCS_E_DEVICE_CHECK, "a particle failed its checks (type, E > 0, finite eta/phi); its tasks were skipped");
  if (s.flags & FCS_FLAG_HIT_CAPACITY)
    return set_err(FCS_E_RANGE, "the workspace holds fewer hits than the call produced (%lld); reserve more",
                   (long long)s.hit_base);
  if (s.flags & FCS_FLAG_KEY_BITS)
    return set_err(FCS_E_RANGE, "deterministic mode: keys exceed 63 bits, or an event holds 2^27 tasks or more");
  if (s.flags & FCS_FLAG_OUT_CAPACITY)
    return set_err(FCS_E_RANGE, "output capacity too small: %lld non-zero cells", (long long)s.nnz_total);
  return ok();
}

int check_particles(const fcs_particles* p, int64_t n_particles) {
  if (!p || !p->event_offsets) return set_err(FCS_E_ARG, "particles and event_offsets must be non-NULL");
  if (n_particles > 0 && (!p->type || !p->E || !p->eta || !p->phi))
    return set_err(FCS_E_ARG, "particles: every array must be non-NULL when n_particles > 0");
  return FCS_OK;
}

struct CallArgs {
  const fcs_geo* geo;
  const fcs_params* prm;
  fcs_workspace* ws;
  fcs_particles parts;
  int64_t n_particles;
  int32_t n_events;
  uint64_t seed;
  int64_t first_event;
  fcs_config cfg;
  float* cells_out;
  int32_t* cell_ids;
  float* cell_E;
  int64_t* event_offsets_out;
  int64_t capacity;
  const fcs_debug* dbg;
  cudaStream_t s;
};

// Stage events: inside a stream capture they must be external events to
// become event-record nodes of the graph; outside a capture plain records.
cudaError_t record_stage(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t err = cudaStreamIsCapturing(s, &cs);
  if (err != cudaSuccess) return err;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                             : cudaEventRecord(e, s);
}

// Kernel nodes of a captured graph.
int64_t graph_kernel_nodes(cudaGraph_t g) {
  int64_t kernels = 0;
  size_t n_nodes = 0;
  if (cudaGraphGetNodes(g, nullptr, &n_nodes) == cudaSuccess && n_nodes > 0) {
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    if (cudaGraphGetNodes(g, nodes.data(), &n_nodes) == cudaSuccess)
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
      }
  }
  return kernels;
}

// The task and hit stages of one event range on a.s: range begin, tasks and
// Poisson counts, hit offsets and tile map, the hit kernel (or one launch per
// task) and the FP64 recheck.  sync_size: read the hit count back after the
// scans and grow the hit-dependent buffers.  The range's accumulation rows
// start at row acc_row0 of the workspace's; *w_out: the view the range used.
int enqueue_range_hits(const CallArgs& a, int32_t ev_lo, int32_t ev_hi, int32_t range, bool sync_size,
                       const HitCfg& hc, int key_task_bits, int64_t acc_row0, WsDev* w_out) {
  fcs_workspace* ws = a.ws;
  const Launch L{a.s, ws->num_sms};
  const int det = a.cfg.mode == FCS_MODE_DETERMINISTIC;
  cudaEvent_t* tev = a.cfg.timing ? &ws->tev[(size_t)range * 5] : nullptr;
  if (tev) FCS_CUDA(record_stage(tev[0], a.s));
  k_range_begin<<<1, kRangeThreads, 0, a.s>>>(ws->d_sizes, a.parts.event_offsets, ev_lo, ev_hi, a.n_particles,
                                              ws->pcap);
  const uint32_t k0 = (uint32_t)(a.seed & 0xFFFFFFFFu), k1 = (uint32_t)(a.seed >> 32);
  const ScanTmp tmp = ws->scan_tmp();
  auto view = [&]() {
    WsDev v = ws->view();
    v.acc = ws->acc + acc_row0 * ws->acc_stride;
    return v;
  };
  WsDev w = view();
  FCS_CUDA(launch_task_counts(a.geo->d, a.prm->d, a.parts, ev_lo, ev_hi, k0, k1, a.first_event, w, tmp,
                              a.n_particles, a.cfg.energy_interp, L));
  if (sync_size || a.cfg.batched == 2) {
    FCS_CUDA(cudaMemcpyAsync(ws->h_sizes, ws->d_sizes, sizeof(Sizes), cudaMemcpyDeviceToHost, a.s));
    FCS_CUDA(cudaStreamSynchronize(a.s));
    FCS_TRY(ws_reserve_hits(ws, ws->h_sizes->n_hits, a.cfg.mode));
    w = view();
  }
  FCS_CUDA(launch_task_finish(w, a.dbg, (sync_size || a.cfg.batched == 2) ? 1 : 0,
                              a.n_particles * a.geo->d.n_layers, L));
  if (tev) FCS_CUDA(record_stage(tev[1], a.s));
  if (a.cfg.batched == 2) {
    // per-task launches: read the range's first hits and hit counts, then
    // one hit-kernel launch over each task's hits
    const int64_t nt = ws->h_sizes->n_tasks;
    if (2 * nt > ws->h_tasks_cap) {
      if (ws->h_tasks) cudaFreeHost(ws->h_tasks);
      ws->h_tasks = nullptr;
      ws->h_tasks_cap = 0;
      FCS_CUDA(cudaMallocHost((void**)&ws->h_tasks, (size_t)(2 * nt) * sizeof(int64_t)));
      ws->h_tasks_cap = 2 * nt;
    }
    if (nt > 0) {
      FCS_CUDA(cudaMemcpyAsync(ws->h_tasks, ws->th, (size_t)nt * sizeof(int64_t), cudaMemcpyDeviceToHost, a.s));
      FCS_CUDA(cudaMemcpyAsync(ws->h_tasks + nt, ws->tn, (size_t)nt * sizeof(int32_t), cudaMemcpyDeviceToHost, a.s));
      FCS_CUDA(cudaStreamSynchronize(a.s));
    }
    for (int64_t t = 0; t < nt; ++t) {
      const int64_t hb = ws->h_tasks[t];
      FCS_CUDA(launch_hits_task(a.geo->d, a.prm->d, w, ev_lo, k0, k1, a.first_event, hc, key_task_bits, a.dbg, hb,
                                hb + reinterpret_cast<const int32_t*>(ws->h_tasks + nt)[t], (int32_t)t, L));
    }
  } else {
    FCS_CUDA(launch_hits(a.geo->d, a.prm->d, w, ev_lo, k0, k1, a.first_event, hc, key_task_bits, a.dbg, L));
  }
  if (tev) FCS_CUDA(record_stage(tev[2], a.s));
  FCS_CUDA(launch_recheck(a.geo->d, a.prm->d, w, ev_lo, k0, k1, a.first_event, det, key_task_bits, a.dbg, L));
  if (tev) FCS_CUDA(record_stage(tev[3], a.s));
  *w_out = w;
  return FCS_OK;
}

// The reduction of one event range on stream s with scan state tmp: the
// deterministic sort and fold, then the compaction into the call's outputs.
int enqueue_range_reduce(const CallArgs& a, WsDev w, int32_t ev_lo, int32_t rows, int key_task_bits, ScanTmp tmp,
                         cudaStream_t s, int max_ctas = 0) {
  fcs_workspace* ws = a.ws;
  const Launch L{s, ws->num_sms};
  if (a.cfg.mode == FCS_MODE_DETERMINISTIC)
    FCS_CUDA(launch_det_reduce(a.geo->d, w, rows, key_task_bits, ws->cell_off, a.parts.event_offsets, ev_lo, tmp, L));
  FCS_CUDA(launch_compact(a.geo->d, w, rows, ev_lo, tmp, a.cells_out, a.cell_ids, a.cell_E, a.event_offsets_out,
                          a.capacity, max_ctas, L));
  return FCS_OK;
}

// Enqueues one event range on a.s (its rows start at row 0 of the workspace's).
int enqueue_range(const CallArgs& a, int32_t ev_lo, int32_t ev_hi, int32_t range, bool sync_size, const HitCfg& hc,
                  int key_task_bits) {
  fcs_workspace* ws = a.ws;
  WsDev w{};
  FCS_TRY(enqueue_range_hits(a, ev_lo, ev_hi, range, sync_size, hc, key_task_bits, 0, &w));
  FCS_TRY(enqueue_range_reduce(a, w, ev_lo, ev_hi - ev_lo, key_task_bits, ws->scan_tmp(), a.s));
  if (a.cfg.timing) FCS_CUDA(record_stage(ws->tev[(size_t)range * 5 + 4], a.s));
  k_range_end<<<1, 1, 0, a.s>>>(ws->d_sizes);
  return FCS_OK;
}

// Events per launch sequence: all (batched, wave_events == 0), waves of
// wave_events, or one (per-event launches).
int32_t range_events(const fcs_config& c, int32_t n_events) {
  if (c.batched != 1) return 1;
  if (c.wave_events > 0 && c.wave_events < n_events) return c.wave_events;
  return std::max(n_events, 1);
}

int32_t n_ranges(const fcs_config& c, int32_t n_events) {
  const int32_t W = range_events(c, n_events);
  return (n_events + W - 1) / W;
}

int ensure_timing_events(fcs_workspace* ws, int ranges) {
  while ((int)ws->tev.size() < ranges * 5) {
    cudaEvent_t e;
    FCS_CUDA(cudaEventCreate(&e));
    ws->tev.push_back(e);
  }
  ws->timed_ranges = ranges;
  return FCS_OK;
}

int enqueue_call(const CallArgs& a, bool sync_size, const HitCfg& hc, int key_task_bits) {
  fcs_workspace* ws = a.ws;
  k_call_begin<<<1, 1, 0, a.s>>>(ws->d_sizes);
  const int32_t W = range_events(a.cfg, a.n_events);
  for (int32_t lo = 0, r = 0; lo < a.n_events; lo += W, ++r)
    FCS_TRY(enqueue_range(a, lo, std::min(a.n_events, lo + W), r, sync_size, hc, key_task_bits));
  k_call_end<<<1, 1, 0, a.s>>>(ws->d_sizes, a.event_offsets_out, a.n_events, a.capacity, a.cell_ids ? 1 : 0);
  FCS_CUDA(cudaGetLastError());
  return FCS_OK;
}

HitCfg hit_cfg(const fcs_config& c) {
  HitCfg h;
  h.block = c.block ? c.block : 128;  // the shape fcs_autotune picks on GB300 for pile-up batches
  h.hpt = c.hits_per_thread ? c.hits_per_thread : 8;
  h.det = c.mode == FCS_MODE_DETERMINISTIC;
  return h;
}

int validate_config(const fcs_config& c) {
  if (c.mode != FCS_MODE_ATOMIC && c.mode != FCS_MODE_DETERMINISTIC) return set_err(FCS_E_ARG, "config.mode");
  if (c.batched < 0 || c.batched > 2) return set_err(FCS_E_ARG, "config.batched must be 0, 1 or 2");
  if (c.batched == 2 && c.use_graph) return set_err(FCS_E_ARG, "per-task launches (batched = 2) cannot be captured");
  const int hpt = c.hits_per_thread, blk = c.block;
  if (!(hpt == 0 || hpt == 1 || hpt == 2 || hpt == 4 || hpt == 8))
    return set_err(FCS_E_ARG, "config.hits_per_thread must be 0, 1, 2, 4 or 8");
  if (!(blk == 0 || blk == 128 || blk == 256 || blk == 512))
    return set_err(FCS_E_ARG, "config.block must be 0, 128, 256 or 512");
  if (c.wave_events < 0) return set_err(FCS_E_ARG, "config.wave_events must be >= 0");
  if (c.energy_interp != 0 && c.energy_interp != 1) return set_err(FCS_E_ARG, "config.energy_interp must be 0 or 1");
  if (c.reserved) return set_err(FCS_E_ARG, "config.reserved must be 0");
  if (c.use_graph && c.sync) return set_err(FCS_E_ARG, "config.use_graph requires sync == 0");
  return FCS_OK;
}

// Device address of a mapped pinned host allocation, else NULL.
void* mapped_host(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return (at.type == cudaMemoryTypeHost && at.devicePointer) ? at.devicePointer : nullptr;
}

// Wave boundaries of a host-buffer call: the events bnd[i] .. bnd[i + 1] - 1
// form wave i.  The shares come from kHostWaveEighths; empty waves are
// dropped, and a call of two or more events gets at least two waves.
int host_wave_bounds(int32_t n, int32_t* bnd) {
  int nw = 0, cum = 0;
  bnd[0] = 0;
  auto take = [&](const int* shares, int count) {
    for (int q = 0; q < count; ++q) {
      cum += shares[q];
      const int32_t b = (int32_t)std::min<int64_t>(n, ((int64_t)n * cum + 7) / 8);
      if (b > bnd[nw]) bnd[++nw] = b;
    }
  };
  if (n >= kHostLargeEvents) take(kHostWaveEighthsLarge, (int)(sizeof(kHostWaveEighthsLarge) / sizeof(int)));
  else take(kHostWaveEighths, (int)(sizeof(kHostWaveEighths) / sizeof(int)));
  if (nw == 1 && n >= 2) {
    bnd[1] = (n + 1) / 2;
    bnd[2] = n;
    nw = 2;
  }
  return nw;
}

// Host-buffer call in waves of events on three streams, captured as one CUDA
// graph: each later wave's particles are copied in while the waves before it
// compute, and each wave's cells are compacted into the mapped output buffers
// (over the CPU-GPU link) while the next wave computes.  Each wave has its own
// accumulation rows; the output stream has its own scan state.
int enqueue_waves(const CallArgs& a, const int32_t* type, const float* E, const float* eta, const float* phi,
                      const int64_t* event_offsets, const int32_t* bnd, int nw, int key_task_bits) {
  fcs_workspace* ws = a.ws;
  const cudaStream_t cs = a.s, s_in = ws->s_in, s_out = ws->s_out;
  const HitCfg hc = hit_cfg(a.cfg);
  const ScanTmp tmp2{ws->scan_state2, ws->ss2_cap - 2, &ws->d_sizes->flags, ws->num_sms * 3};
  const fcs_particles& d = a.parts;
  auto copy_in = [&](int64_t lo, int64_t hi) -> cudaError_t {
    if (hi <= lo) return cudaSuccess;
    const size_t n = (size_t)(hi - lo) * 4;
    cudaError_t e = cudaMemcpyAsync((void*)(d.type + lo), type + lo, n, cudaMemcpyHostToDevice, s_in);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)(d.E + lo), E + lo, n, cudaMemcpyHostToDevice, s_in);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)(d.eta + lo), eta + lo, n, cudaMemcpyHostToDevice, s_in);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void*)(d.phi + lo), phi + lo, n, cudaMemcpyHostToDevice, s_in);
    return e;
  };
  k_call_begin<<<1, 1, 0, cs>>>(ws->d_sizes);
  FCS_CUDA(cudaEventRecord(ws->pev[0], cs));
  FCS_CUDA(cudaStreamWaitEvent(s_in, ws->pev[0], 0));
  FCS_CUDA(cudaStreamWaitEvent(s_out, ws->pev[0], 0));
  FCS_CUDA(cudaMemcpyAsync((void*)d.event_offsets, event_offsets, (size_t)(a.n_events + 1) * 8,
                           cudaMemcpyHostToDevice, s_in));
  for (int k = 0; k < nw; ++k) {
    FCS_CUDA(copy_in(event_offsets[bnd[k]], event_offsets[bnd[k + 1]]));
    FCS_CUDA(cudaEventRecord(ws->pev[1 + k], s_in));
  }
  for (int k = 0; k < nw; ++k) {
    FCS_CUDA(cudaStreamWaitEvent(cs, ws->pev[1 + k], 0));
    WsDev w{};
    FCS_TRY(enqueue_range_hits(a, bnd[k], bnd[k + 1], k, false, hc, key_task_bits, bnd[k], &w));
    k_range_end<<<1, 1, 0, cs>>>(ws->d_sizes);
    FCS_CUDA(cudaEventRecord(ws->pev[1 + nw + k], cs));
    FCS_CUDA(cudaStreamWaitEvent(s_out, ws->pev[1 + nw + k], 0));
    // the compaction runs beside the next wave on a third of the SMs: its
    // stores over the CPU-GPU link need few CTAs to keep the link busy, and
    // the next wave's kernels keep the rest (a quarter starved the link on
    // small calls; half slowed the next wave on large ones)
    FCS_TRY(enqueue_range_reduce(a, w, bnd[k], bnd[k + 1] - bnd[k], key_task_bits, tmp2, s_out, ws->num_sms / 3));
  }
  k_call_end<<<1, 1, 0, s_out>>>(ws->d_sizes, a.event_offsets_out, a.n_events, a.capacity, a.cell_ids ? 1 : 0);
  FCS_CUDA(cudaEventRecord(ws->pev[1 + 2 * nw], s_out));
  FCS_CUDA(cudaStreamWaitEvent(cs, ws->pev[1 + 2 * nw], 0));
  FCS_CUDA(cudaGetLastError());
  return FCS_OK;
}

// Replays (capturing it first when its arguments changed) the two-wave graph
// of a host-buffer call on stream s.  FCS_E_UNSUPPORTED when the call does not
// qualify: atomic mode in one launch sequence, at least two events, pinned
// inputs, offsets from 0 to n_particles, a workspace sized for the hits.
int host_waves(const fcs_geo* geo, const fcs_params* prm, fcs_workspace* ws, const int32_t* type, const float* E,
                   const float* eta, const float* phi, const int64_t* event_offsets, int64_t n_particles,
                   int32_t n_events, uint64_t seed, int64_t first_event, const fcs_config& cfg,
                   const fcs_particles& dparts, int32_t* m_ids, float* m_cE, int64_t* m_oout, int64_t capacity,
                   cudaStream_t s) {
  if (cfg.mode != FCS_MODE_ATOMIC || cfg.batched != 1 || cfg.timing || n_events < 2 || n_particles <= 0 ||
      (cfg.wave_events > 0 && cfg.wave_events < n_events) || !m_ids || !m_oout || ws->gmap_cap == 0)
    return FCS_E_UNSUPPORTED;
  for (const void* p : {(const void*)type, (const void*)E, (const void*)eta, (const void*)phi,
                        (const void*)event_offsets})
    if (!mapped_host(p)) return FCS_E_UNSUPPORTED;
  if (event_offsets[0] != 0 || event_offsets[n_events] != n_particles) return FCS_E_UNSUPPORTED;
  for (int32_t e = 0; e < n_events; ++e)
    if (event_offsets[e + 1] < event_offsets[e]) return FCS_E_UNSUPPORTED;
  int32_t bnd[kMaxHostWaves + 1];
  const int nw = host_wave_bounds(n_events, bnd);
  if ((int64_t)n_events * geo->d.acc_stride >= (int64_t(1) << 32)) return FCS_E_UNSUPPORTED;
  FCS_TRY(ws_reserve_static(ws, geo, n_particles, n_events, cfg.mode));
  if (ws->ss2_cap < ws->ss_cap) {
    if (ws->scan_state2) cudaFree(ws->scan_state2);
    ws->scan_state2 = nullptr;
    ws->ss2_cap = 0;
    FCS_TRY(grow(&ws->scan_state2, &ws->ss2_cap, ws->ss_cap, true));
  }
  if (!ws->s_in) FCS_CUDA(cudaStreamCreateWithFlags(&ws->s_in, cudaStreamNonBlocking));
  if (!ws->s_out) FCS_CUDA(cudaStreamCreateWithFlags(&ws->s_out, cudaStreamNonBlocking));
  for (cudaEvent_t& e : ws->pev)
    if (!e) FCS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  const int key_task_bits = bits_for(n_particles * geo->d.n_layers);
  // key of the captured sequence: every argument and buffer that shapes it
  std::vector<unsigned char> key;
  auto put = [&](const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    key.insert(key.end(), c, c + n);
  };
  const void* hp[5] = {type, E, eta, phi, event_offsets};
  const WsDev view = ws->view();
  put(&geo, sizeof(geo));
  put(&prm, sizeof(prm));
  put(hp, sizeof(hp));
  put(&n_particles, sizeof(n_particles));
  put(&n_events, sizeof(n_events));
  put(bnd, sizeof(int32_t) * (nw + 1));
  put(&seed, sizeof(seed));
  put(&first_event, sizeof(first_event));
  put(&cfg, sizeof(cfg));
  put(&dparts, sizeof(dparts));
  put(&m_ids, sizeof(m_ids));
  put(&m_cE, sizeof(m_cE));
  put(&m_oout, sizeof(m_oout));
  put(&capacity, sizeof(capacity));
  put(&view, sizeof(view));
  put(&ws->acc_stride, sizeof(ws->acc_stride));
  put(&ws->scan_state, sizeof(void*));
  put(&ws->ss_cap, sizeof(ws->ss_cap));
  put(&ws->scan_state2, sizeof(void*));
  put(&ws->ss2_cap, sizeof(ws->ss2_cap));
  if (!ws->pgraph || key != ws->pgraph_key) {
    if (ws->pgraph) {
      cudaGraphExecDestroy(ws->pgraph);
      ws->pgraph = nullptr;
    }
    cudaStream_t cs;
    FCS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    CallArgs a{geo, prm, ws, dparts, n_particles, n_events, seed, first_event, cfg, nullptr,
               m_ids, m_cE, m_oout, capacity, nullptr, cs};
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = FCS_OK;
    if (e == cudaSuccess) rc = enqueue_waves(a, type, E, eta, phi, event_offsets, bnd, nw, key_task_bits);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess || rc != FCS_OK || e2 != cudaSuccess) {
      // the forked streams took part in a failed capture: start them afresh
      (void)cudaGetLastError();
      cudaStreamDestroy(ws->s_in);
      cudaStreamDestroy(ws->s_out);
      ws->s_in = ws->s_out = nullptr;
    }
    if (e != cudaSuccess) return set_err(FCS_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
    if (rc != FCS_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e2 != cudaSuccess) return set_err(FCS_E_CUDA, "graph capture: %s", cudaGetErrorString(e2));
    ws->pgraph_kernels = graph_kernel_nodes(g);
    e = cudaGraphInstantiate(&ws->pgraph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      ws->pgraph = nullptr;
      return set_err(FCS_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    ws->pgraph_key = key;
  }
  FCS_CUDA(cudaGraphLaunch(ws->pgraph, s));
  ws->launched_kernels = ws->pgraph_kernels;
  return FCS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* fcs_version(void) { return "libfcs 0.1 (sm_103a)"; }

int fcs_last_error(char* buf, size_t len) {
  if (buf && len) {
    std::strncpy(buf, g_err_msg, len - 1);
    buf[len - 1] = 0;
  }
  return g_err_code;
}

int fcs_load_geometry(fcs_geo** out, const fcs_region* regions, int32_t n_regions,
                      const int32_t* layer_region_begin, int32_t n_layers, const fcs_layer_geom* layers,
                      cudaStream_t s) {
  if (!out) return set_err(FCS_E_ARG, "out is NULL");
  *out = nullptr;
  if (!regions || !layer_region_begin || !layers) return set_err(FCS_E_ARG, "NULL table");
  if (n_layers < 1 || n_layers > kMaxLayers) return set_err(FCS_E_ARG, "n_layers must be in [1, %d]", kMaxLayers);
  if (n_regions < 1 || n_regions > kMaxRegions) return set_err(FCS_E_ARG, "n_regions must be in [1, %d]", kMaxRegions);
  const int32_t* lrb = layer_region_begin;
  if (lrb[0] != 0 || lrb[n_layers] != n_regions) return set_err(FCS_E_ARG, "layer_region_begin must span [0, n_regions]");
  int64_t cells = 0;
  std::vector<RegionF> rf(n_regions);
  std::vector<float> split32(n_regions);
  std::vector<double> eta_lo(n_regions), deta(n_regions), phi_lo(n_regions), dphi(n_regions), split(n_regions);
  std::vector<int32_t> ne(n_regions), np(n_regions), co(n_regions);
  for (int l = 0; l < n_layers; ++l) {
    if (lrb[l + 1] <= lrb[l]) return set_err(FCS_E_ARG, "layer %d has no region", l);
    const double R = layers[l].rz;
    if (!(R > 0.0) || !std::isfinite(R)) return set_err(FCS_E_ARG, "layer %d: rz must be > 0", l);
    if (layers[l].barrel != 0 && layers[l].barrel != 1) return set_err(FCS_E_ARG, "layer %d: barrel flag", l);
    for (int r = lrb[l]; r < lrb[l + 1]; ++r) {
      const fcs_region& g = regions[r];
      if (g.layer != l) return set_err(FCS_E_ARG, "region %d: layer %d != %d", r, g.layer, l);
      if (g.n_eta < 1 || g.n_phi < 1) return set_err(FCS_E_ARG, "region %d: empty grid", r);
      if (g.n_eta > (1 << 22)) return set_err(FCS_E_ARG, "region %d: more than 2^22 eta cells", r);
      if (!(g.deta > 0.0) || !(g.dphi > 0.0) || !std::isfinite(g.deta) || !std::isfinite(g.dphi) ||
          !std::isfinite(g.eta_lo) || !std::isfinite(g.phi_lo))
        return set_err(FCS_E_ARG, "region %d: bad bounds", r);
      if (g.cell_offset != cells) return set_err(FCS_E_ARG, "region %d: cell ids must be contiguous", r);
      cells += (int64_t)g.n_eta * g.n_phi;
      if (cells >= (int64_t(1) << 31)) return set_err(FCS_E_ARG, "more than 2^31 - 1 cells");
      eta_lo[r] = g.eta_lo;
      deta[r] = g.deta;
      phi_lo[r] = g.phi_lo;
      dphi[r] = g.dphi;
      ne[r] = g.n_eta;
      np[r] = g.n_phi;
      co[r] = g.cell_offset;
      if (r == lrb[l]) {
        split[r] = -std::numeric_limits<double>::infinity();
      } else {
        // midpoint between the top of the previous region and this eta_lo
        const double top = eta_lo[r - 1] + (double)ne[r - 1] * deta[r - 1];
        if (!(g.eta_lo >= top - 1e-9)) return set_err(FCS_E_ARG, "region %d overlaps region %d", r, r - 1);
        split[r] = 0.5 * (top + g.eta_lo);
      }
      RegionF& f = rf[r];
      f = RegionF{};
      f.ek = (float)(-g.eta_lo / g.deta);
      f.inv_deta = (float)(1.0 / g.deta);
      f.pk = (float)(-g.phi_lo / g.dphi);
      f.inv_dphi = (float)(1.0 / g.dphi);
      split32[r] = (float)split[r];
      f.n_eta_hf = (float)g.n_eta - 0.5f;
      // bounds of the FP32 index beyond the position's error (fcs_hits.cuh: fast_cell), rounded up
      f.ce = (float)(std::fabs((double)f.ek) * 0x1p-23 + 0x1p-22) * 1.0001f;
      f.cp = (float)(std::fabs((double)f.pk) * 0x1p-23 + 0x1p-22) * 1.0001f;
      f.n_phi = g.n_phi;
      f.cell_off = g.cell_offset;
    }
  }
  fcs_geo* geo = new fcs_geo();
  int rc = FCS_OK;
  auto fail = [&](int code) {
    delete geo;
    return code;
  };
  if ((rc = current_device(&geo->device)) != FCS_OK) return fail(rc);
  RegionF* d_rf;
  double *d_el, *d_de, *d_pl, *d_dp, *d_sp, *d_rz;
  float *d_rinv32, *d_sp32;
  int32_t *d_ne, *d_np, *d_co, *d_lrb, *d_bar;
  if ((rc = dev_alloc(&d_rf, n_regions, &geo->allocs)) || (rc = dev_alloc(&d_el, n_regions, &geo->allocs)) ||
      (rc = dev_alloc(&d_de, n_regions, &geo->allocs)) || (rc = dev_alloc(&d_pl, n_regions, &geo->allocs)) ||
      (rc = dev_alloc(&d_dp, n_regions, &geo->allocs)) || (rc = dev_alloc(&d_sp, n_regions, &geo->allocs)) ||
      (rc = dev_alloc(&d_ne, n_regions, &geo->allocs)) || (rc = dev_alloc(&d_np, n_regions, &geo->allocs)) ||
      (rc = dev_alloc(&d_co, n_regions, &geo->allocs)) || (rc = dev_alloc(&d_lrb, n_layers + 1, &geo->allocs)) ||
      (rc = dev_alloc(&d_rz, n_layers, &geo->allocs)) || (rc = dev_alloc(&d_bar, n_layers, &geo->allocs)) ||
      (rc = dev_alloc(&d_rinv32, n_layers, &geo->allocs)) || (rc = dev_alloc(&d_sp32, n_regions, &geo->allocs)))
    return fail(rc);
  std::vector<double> rz(n_layers);
  std::vector<float> rinv32(n_layers);
  std::vector<int32_t> bar(n_layers);
  for (int l = 0; l < n_layers; ++l) {
    rz[l] = layers[l].rz;
    rinv32[l] = 1.0f / (float)layers[l].rz;  // correctly rounded, as on the device
    bar[l] = layers[l].barrel;
  }
  const struct {
    void* d;
    const void* h;
    size_t n;
  } copies[] = {{d_rf, rf.data(), n_regions * sizeof(RegionF)}, {d_el, eta_lo.data(), n_regions * sizeof(double)},
                {d_de, deta.data(), n_regions * sizeof(double)},  {d_pl, phi_lo.data(), n_regions * sizeof(double)},
                {d_dp, dphi.data(), n_regions * sizeof(double)},  {d_sp, split.data(), n_regions * sizeof(double)},
                {d_ne, ne.data(), n_regions * sizeof(int32_t)},   {d_np, np.data(), n_regions * sizeof(int32_t)},
                {d_co, co.data(), n_regions * sizeof(int32_t)},   {d_lrb, lrb, (n_layers + 1) * sizeof(int32_t)},
                {d_rz, rz.data(), n_layers * sizeof(double)},     {d_bar, bar.data(), n_layers * sizeof(int32_t)},
                {d_rinv32, rinv32.data(), n_layers * sizeof(float)},  {d_sp32, split32.data(), n_regions * sizeof(float)}};
  for (const auto& c : copies) {
    cudaError_t e = cudaMemcpyAsync(c.d, c.h, c.n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(set_err(FCS_E_CUDA, "geometry copy: %s", cudaGetErrorString(e)));
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(set_err(FCS_E_CUDA, "geometry copy: %s", cudaGetErrorString(e)));
  GeoDev& d = geo->d;
  d.n_layers = n_layers;
  d.n_regions = n_regions;
  d.n_cells = (int32_t)cells;
  d.acc_stride = (int32_t)((cells + 63) / 64 * 64);
  d.regf = d_rf;
  d.eta_lo = d_el;
  d.deta = d_de;
  d.phi_lo = d_pl;
  d.dphi = d_dp;
  d.split = d_sp;
  d.split32 = d_sp32;
  d.n_eta = d_ne;
  d.n_phi = d_np;
  d.cell_off = d_co;
  d.lrb = d_lrb;
  d.rz = d_rz;
  d.rinv32 = d_rinv32;
  d.barrel = d_bar;
  *out = geo;
  return ok();
}

int fcs_geometry_info(const fcs_geo* geo, int32_t* n_cells, int32_t* n_layers, int32_t* n_regions) {
  if (!geo) return set_err(FCS_E_ARG, "geo is NULL");
  if (n_cells) *n_cells = geo->d.n_cells;
  if (n_layers) *n_layers = geo->d.n_layers;
  if (n_regions) *n_regions = geo->d.n_regions;
  return ok();
}

void fcs_free_geometry(fcs_geo* geo) { delete geo; }

int fcs_load_params(fcs_params** out, const fcs_geo* geo, const float* frac, const float* mean_hit_E,
                    const float* shape_w, const float* r_edges, const float* a_edges, int32_t NT, int32_t NE,
                    int32_t NH, int32_t NR, int32_t NA, double eta_bin_scale, int32_t ebin_log2_min,
                    cudaStream_t s) {
  if (!out) return set_err(FCS_E_ARG, "out is NULL");
  *out = nullptr;
  if (!geo || !frac || !mean_hit_E || !shape_w || !r_edges || !a_edges) return set_err(FCS_E_ARG, "NULL argument");
  if (NT < 1 || NE < 1 || NH < 1) return set_err(FCS_E_ARG, "NT, NE, NH must be >= 1");
  if (NR != kNR || NA != kNA) return set_err(FCS_E_ARG, "the shape histogram must be %d (r) x %d (alpha)", kNR, kNA);
  if (!(eta_bin_scale > 0.0) || !std::isfinite(eta_bin_scale)) return set_err(FCS_E_ARG, "eta_bin_scale must be > 0");
  if (ebin_log2_min < -1000 || ebin_log2_min > 1000) return set_err(FCS_E_ARG, "ebin_log2_min out of range");
  const int NL = geo->d.n_layers;
  const int64_t n_entries = (int64_t)NT * NE * NH * NL;
  if (n_entries >= (int64_t(1) << 24)) return set_err(FCS_E_ARG, "parametrisation has 2^24 or more entries");
  if (!(r_edges[0] >= 0.0f)) return set_err(FCS_E_ARG, "r_edges[0] must be >= 0");
  for (int i = 0; i < NR; ++i)
    if (!(r_edges[i + 1] > r_edges[i]) || !std::isfinite(r_edges[i + 1])) return set_err(FCS_E_ARG, "r_edges must increase");
  if (!(a_edges[0] >= 0.0f) || !(a_edges[NA] <= 6.2831855f)) return set_err(FCS_E_ARG, "a_edges must lie in [0, 2 pi]");
  for (int i = 0; i < NA; ++i)
    if (!(a_edges[i + 1] > a_edges[i])) return set_err(FCS_E_ARG, "a_edges must increase");
  for (int64_t e = 0; e < n_entries; ++e) {
    const float f = frac[e], m = mean_hit_E[e];
    if (!(f >= 0.0f) || !std::isfinite(f)) return set_err(FCS_E_ARG, "frac[%lld] must be finite and >= 0", (long long)e);
    const float* w = shape_w + e * kNBins;
    double sum = 0.0;
    for (int k = 0; k < kNBins; ++k) {
      if (!(w[k] >= 0.0f) || !std::isfinite(w[k]))
        return set_err(FCS_E_ARG, "shape_w[%lld][%d] must be finite and >= 0", (long long)e, k);
      sum += w[k];
    }
    if (f > 0.0f) {
      if (!(m > 0.0f) || !std::isfinite(m))
        return set_err(FCS_E_ARG, "mean_hit_E[%lld] must be > 0 where frac > 0", (long long)e);
      if (!(sum > 0.0)) return set_err(FCS_E_ARG, "shape_w of entry %lld sums to 0 where frac > 0", (long long)e);
    }
  }
  fcs_params* prm = new fcs_params();
  int rc = FCS_OK;
  auto fail = [&](int code) {
    delete prm;
    return code;
  };
  if ((rc = current_device(&prm->device)) != FCS_OK) return fail(rc);
  float *d_frac, *d_mhe, *d_re, *d_ae, *d_lf, *d_w = nullptr;
  double* d_lf64 = nullptr;
  uint32_t* d_thr;
  uint2* d_guide;
  int32_t* d_bad = nullptr;
  if ((rc = dev_alloc(&d_frac, n_entries, &prm->allocs)) || (rc = dev_alloc(&d_mhe, n_entries, &prm->allocs)) ||
      (rc = dev_alloc(&d_re, NR + 1, &prm->allocs)) || (rc = dev_alloc(&d_ae, NA + 1, &prm->allocs)) ||
      (rc = dev_alloc(&d_thr, n_entries * kNBins, &prm->allocs)) ||
      (rc = dev_alloc(&d_guide, n_entries * kGuideCells, &prm->allocs)) ||
      (rc = dev_alloc(&d_lf, kLfactEntries, &prm->allocs)) ||
      (rc = dev_alloc(&d_lf64, kLfactEntries, &prm->allocs)))
    return fail(rc);
  // log k! from the host's FP64 lgamma: as is for the FP64 Poisson acceptance
  // test (the value the C definition computes), rounded once for the FP32 test
  std::vector<float> lf(kLfactEntries);
  std::vector<double> lf64(kLfactEntries);
  for (int k = 0; k < kLfactEntries; ++k) {
    lf64[k] = std::lgamma((double)k + 1.0);
    lf[k] = (float)lf64[k];
  }
  if ((rc = dev_alloc(&d_w, n_entries * kNBins, &prm->allocs)) || (rc = dev_alloc(&d_bad, n_entries, &prm->allocs)) ||
      (rc = dev_alloc(&prm->check, 1, &prm->allocs)))
    return fail(rc);
  cudaError_t e = cudaSuccess;
  if ((e = cudaMemcpyAsync(d_frac, frac, n_entries * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_mhe, mean_hit_E, n_entries * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_re, r_edges, (NR + 1) * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_ae, a_edges, (NA + 1) * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_lf, lf.data(), kLfactEntries * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_lf64, lf64.data(), kLfactEntries * sizeof(double), cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(d_w, shape_w, n_entries * kNBins * sizeof(float), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = launch_build_tables(d_w, (int)n_entries, d_thr, d_guide, d_bad, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    return fail(set_err(FCS_E_CUDA, "parametrisation upload: %s", cudaGetErrorString(e)));
  }
  prm->w = d_w;
  prm->bad = d_bad;
  ParamDev& d = prm->d;
  d.NT = NT;
  d.NE = NE;
  d.NH = NH;
  d.NL = NL;
  d.eta_scale = eta_bin_scale;
  d.ebin_min = ebin_log2_min;
  d.eta_scale_int = (eta_bin_scale == std::floor(eta_bin_scale) && eta_bin_scale >= 1.0 && eta_bin_scale <= 255.0)
                        ? (int32_t)eta_bin_scale
                        : 0;
  d.n_lfact = kLfactEntries;
  d.lfact = d_lf;
  d.lfact64 = d_lf64;
  d.n_entries = (int32_t)n_entries;
  d.frac = d_frac;
  d.shape_w = d_w;
  d.mhe = d_mhe;
  d.thr = d_thr;
  d.guide = d_guide;
  d.r_edges = d_re;
  d.a_edges = d_ae;
  *out = prm;
  return ok();
}

int fcs_update_params(fcs_params* prm, const float* frac, const float* mean_hit_E, const float* shape_w,
                      cudaStream_t s) {
  if (!prm) return set_err(FCS_E_ARG, "params is NULL");
  int dev = 0;
  FCS_TRY(current_device(&dev));
  if (dev != prm->device) return set_err(FCS_E_ARG, "the parametrisation lives on another device");
  ParamDev& d = prm->d;
  const int64_t n = d.n_entries;
  FCS_CUDA(cudaMemsetAsync(prm->check, 0, sizeof(uint32_t), s));
  FCS_CUDA(launch_check_params(frac ? frac : d.frac, mean_hit_E ? mean_hit_E : d.mhe, shape_w ? shape_w : prm->w,
                               (int)n, prm->check, s));
  uint32_t bad = 0;
  FCS_CUDA(cudaMemcpyAsync(&bad, prm->check, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  FCS_CUDA(cudaStreamSynchronize(s));
  if (bad & 1u) return set_err(FCS_E_ARG, "frac must be finite and >= 0");
  if (bad & 2u) return set_err(FCS_E_ARG, "mean_hit_E must be finite and > 0 where frac > 0");
  if (bad & 4u) return set_err(FCS_E_ARG, "shape_w must be finite and >= 0");
  if (bad & 8u) return set_err(FCS_E_ARG, "shape_w of an entry with frac > 0 sums to 0");
  if (frac) FCS_CUDA(cudaMemcpyAsync((void*)d.frac, frac, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (mean_hit_E) FCS_CUDA(cudaMemcpyAsync((void*)d.mhe, mean_hit_E, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (shape_w) {
    FCS_CUDA(cudaMemcpyAsync(prm->w, shape_w, n * kNBins * sizeof(float), cudaMemcpyDeviceToDevice, s));
    FCS_CUDA(launch_build_tables(prm->w, (int)n, (uint32_t*)d.thr, (uint2*)d.guide, prm->bad, s));
  }
  return ok();
}

void fcs_free_params(fcs_params* prm) { delete prm; }

int fcs_workspace_create(fcs_workspace** out) {
  if (!out) return set_err(FCS_E_ARG, "out is NULL");
  *out = new fcs_workspace();
  return ok();
}

int fcs_workspace_reserve(fcs_workspace* ws, const fcs_geo* geo, int64_t n_particles, int32_t n_events,
                          int64_t n_hits, int32_t mode) {
  if (!ws || !geo) return set_err(FCS_E_ARG, "NULL argument");
  if (n_particles < 0 || n_events < 0 || n_hits < 0) return set_err(FCS_E_ARG, "negative size");
  if (mode != FCS_MODE_ATOMIC && mode != FCS_MODE_DETERMINISTIC) return set_err(FCS_E_ARG, "mode");
  FCS_TRY(ws_reserve_static(ws, geo, n_particles, n_events, mode));
  FCS_TRY(ws_reserve_hits(ws, n_hits, mode));
  return ok();
}

int fcs_workspace_status(fcs_workspace* ws, fcs_stats* stats, cudaStream_t s) {
  if (!ws) return set_err(FCS_E_ARG, "ws is NULL");
  if (!ws->d_sizes) {
    if (stats) std::memset(stats, 0, sizeof(*stats));
    return ok();
  }
  FCS_CUDA(cudaMemcpyAsync(ws->h_sizes, ws->d_sizes, sizeof(Sizes), cudaMemcpyDeviceToHost, s));
  FCS_CUDA(cudaStreamSynchronize(s));
  return status_from(*ws->h_sizes, stats);
}

int fcs_workspace_graph_kernels(const fcs_workspace* ws, int64_t* n_kernels) {
  if (!ws || !n_kernels) return set_err(FCS_E_ARG, "NULL argument");
  *n_kernels = 0;
  if (!ws->launched_kernels) return set_err(FCS_E_ARG, "no call on this workspace has run as a graph");
  *n_kernels = ws->launched_kernels;
  return ok();
}

int fcs_selftest_wait_timeout(float* ms, cudaStream_t s) {
  if (!ms) return set_err(FCS_E_ARG, "ms is NULL");
  *ms = 0.0f;
  uint32_t flags = 0;
  FCS_CUDA(scan_wait_selftest(&flags, ms, s));
  if (!(flags & FCS_FLAG_WAIT_TIMEOUT))
    return set_err(FCS_E_DEVICE_CHECK, "the self-test's wait did not report giving up (flags 0x%x)", flags);
  return set_err(FCS_E_TIMEOUT, "a bounded device wait gave up after %.0f ms (self-test)", *ms);
}

int fcs_poisson_audit(const fcs_params* prm, const float* mu, int64_t n, uint64_t seed, int32_t* n_fp32,
                      int32_t* n_fp64, cudaStream_t s) {
  if (!prm || n < 0 || (n > 0 && (!mu || !n_fp32 || !n_fp64))) return set_err(FCS_E_ARG, "bad argument");
  int dev = 0, sms = 0;
  FCS_TRY(current_device(&dev));
  if (dev != prm->device) return set_err(FCS_E_ARG, "the parametrisation must live on the current device");
  FCS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const Launch L{s, sms};
  FCS_CUDA(launch_poisson_audit(prm->d, mu, n, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), n_fp32, n_fp64,
                                L));
  FCS_CUDA(cudaStreamSynchronize(s));
  return ok();
}

int fcs_workspace_timings(fcs_workspace* ws, float* ms) {
  if (!ws || !ms) return set_err(FCS_E_ARG, "NULL argument");
  if (ws->timed_ranges <= 0) return set_err(FCS_E_ARG, "no timed call on this workspace");
  for (int k = 0; k < FCS_N_STAGES; ++k) ms[k] = 0.0f;
  FCS_CUDA(cudaEventSynchronize(ws->tev[(size_t)ws->timed_ranges * 5 - 1]));
  for (int r = 0; r < ws->timed_ranges; ++r) {
    const cudaEvent_t* e = &ws->tev[(size_t)r * 5];
    for (int k = 0; k < 4; ++k) {
      float t = 0.0f;
      FCS_CUDA(cudaEventElapsedTime(&t, e[k], e[k + 1]));
      ms[k] += t;
    }
  }
  ms[FCS_STAGE_TOTAL] = ms[0] + ms[1] + ms[2] + ms[3];
  return ok();
}

void fcs_workspace_free(fcs_workspace* ws) { delete ws; }

int fcs_simulate_events(const fcs_geo* geo, const fcs_params* prm, fcs_workspace* ws,
                        const fcs_particles* particles, int64_t n_particles, int32_t n_events, uint64_t seed,
                        int64_t first_event, const fcs_config* config, float* cells_out, int32_t* cell_ids,
                        float* cell_E, int64_t* event_offsets_out, int64_t capacity, fcs_stats* stats,
                        const fcs_debug* dbg, cudaStream_t s) {
  if (!geo || !prm || !ws) return set_err(FCS_E_ARG, "geo, params and workspace are required");
  FCS_TRY(check_particles(particles, n_particles));
  if (n_particles < 0 || n_events < 0 || capacity < 0) return set_err(FCS_E_ARG, "negative size");
  if (n_events >= kMaxEventsPerCall) return set_err(FCS_E_RANGE, "at most 2^24 - 1 events per call");
  if (prm->d.NL != geo->d.n_layers) return set_err(FCS_E_ARG, "parametrisation and geometry disagree on layers");
  if ((cell_ids == nullptr) != (cell_E == nullptr)) return set_err(FCS_E_ARG, "cell_ids and cell_E go together");
  fcs_config cfg{};
  cfg.batched = 1;
  cfg.sync = 1;
  if (config) cfg = *config;
  FCS_TRY(validate_config(cfg));
  int dev = 0;
  FCS_TRY(current_device(&dev));
  if (dev != geo->device || dev != prm->device || (ws->device >= 0 && ws->device != dev))
    return set_err(FCS_E_ARG, "geometry, parametrisation and workspace must live on the current device");
  if (n_events == 0) {
    if (event_offsets_out) k_empty_offsets<<<1, 32, 0, s>>>(event_offsets_out, 0);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    FCS_CUDA(cudaGetLastError());
    return ok();
  }
  const int32_t rows = range_events(cfg, n_events);
  if ((int64_t)rows * geo->d.acc_stride >= (int64_t(1) << 32))
    return set_err(FCS_E_RANGE, "%d events x %d cells exceed 2^32 accumulation cells; split the batch", rows,
                   geo->d.acc_stride);
  FCS_TRY(ws_reserve_static(ws, geo, n_particles, rows, cfg.mode));
  const int key_task_bits = bits_for(std::max<int64_t>(n_particles, 1) * geo->d.n_layers);
  if (cfg.mode == FCS_MODE_DETERMINISTIC &&
      kRecordCountBits + key_task_bits + bits_for((int64_t)rows * geo->d.acc_stride) > 63)
    return set_err(FCS_E_RANGE, "deterministic mode: (cell, task) keys exceed 63 bits; use smaller waves or split the batch");
  CallArgs a{geo, prm, ws, *particles, n_particles, n_events, seed, first_event, cfg, cells_out,
             cell_ids, cell_E, event_offsets_out, capacity, dbg, s};
  const HitCfg hc = hit_cfg(cfg);
  if (cfg.timing) FCS_TRY(ensure_timing_events(ws, n_ranges(cfg, n_events)));
  else ws->timed_ranges = 0;
  if (!cfg.sync && cfg.use_graph) {
    // key of the captured sequence: every argument that shapes it
    std::vector<unsigned char> key;
    auto put = [&](const void* p, size_t n) {
      const unsigned char* c = (const unsigned char*)p;
      key.insert(key.end(), c, c + n);
    };
    put(&geo, sizeof(geo));
    put(&prm, sizeof(prm));
    put(particles, sizeof(*particles));
    put(&n_particles, sizeof(n_particles));
    put(&n_events, sizeof(n_events));
    put(&seed, sizeof(seed));
    put(&first_event, sizeof(first_event));
    put(&cfg, sizeof(cfg));
    put(&cells_out, sizeof(cells_out));
    put(&cell_ids, sizeof(cell_ids));
    put(&cell_E, sizeof(cell_E));
    put(&event_offsets_out, sizeof(event_offsets_out));
    put(&capacity, sizeof(capacity));
    put(&dbg, sizeof(dbg));
    put(&ws->d_sizes, sizeof(void*));
    put(&ws->pcount, sizeof(void*));
    put(&ws->poff, sizeof(void*));
    put(&ws->pinfo, sizeof(void*));
    put(&ws->tasks, sizeof(void*));
    put(&ws->gmap, sizeof(void*));
    put(&ws->recheck, sizeof(void*));
    put(&ws->acc, sizeof(void*));
    put(&ws->keys, sizeof(void*));
    put(&ws->cell_off, sizeof(void*));
    if (!ws->graph || key != ws->graph_key) {
      if (ws->graph) {
        cudaGraphExecDestroy(ws->graph);
        ws->graph = nullptr;
      }
      cudaStream_t cs;
      FCS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      CallArgs ca = a;
      ca.s = cs;
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      int rc = FCS_OK;
      if (e == cudaSuccess) rc = enqueue_call(ca, false, hc, key_task_bits);
      cudaError_t e2 = cudaStreamEndCapture(cs, &g);
      cudaStreamDestroy(cs);
      if (e != cudaSuccess) return set_err(FCS_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
      if (rc != FCS_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (e2 != cudaSuccess) return set_err(FCS_E_CUDA, "graph capture: %s", cudaGetErrorString(e2));
      const int64_t kernels = graph_kernel_nodes(g);
      e = cudaGraphInstantiate(&ws->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        ws->graph = nullptr;
        return set_err(FCS_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
      }
      ws->graph_key = key;
      ws->graph_kernels = kernels;
    }
    FCS_CUDA(cudaGraphLaunch(ws->graph, s));
    ws->launched_kernels = ws->graph_kernels;
    return ok();
  }
  // A sync call reads the hit count back mid-call only while the workspace has
  // never been sized for hits; later calls run optimistically and are redone
  // once, with the workspace grown, if they outgrow it (a call that overflows
  // deposits nothing beyond the flag and leaves the accumulation rows zero).
  const bool size_mid_call = cfg.sync != 0 && cfg.batched == 1 && ws->gmap_cap == 0;
  FCS_TRY(enqueue_call(a, size_mid_call, hc, key_task_bits));
  if (!cfg.sync) return ok();
  FCS_CUDA(cudaMemcpyAsync(ws->h_sizes, ws->d_sizes, sizeof(Sizes), cudaMemcpyDeviceToHost, s));
  FCS_CUDA(cudaStreamSynchronize(s));
  if (ws->h_sizes->flags & FCS_FLAG_HIT_CAPACITY) {
    // the call outgrew the workspace: size it for the whole call's hits (they
    // bound every event range's) and run again
    FCS_TRY(ws_reserve_hits(ws, ws->h_sizes->hit_base, cfg.mode));
    FCS_TRY(enqueue_call(a, false, hc, key_task_bits));
    FCS_CUDA(cudaMemcpyAsync(ws->h_sizes, ws->d_sizes, sizeof(Sizes), cudaMemcpyDeviceToHost, s));
    FCS_CUDA(cudaStreamSynchronize(s));
  }
  return status_from(*ws->h_sizes, stats);
}

int fcs_autotune(const fcs_geo* geo, const fcs_params* prm, fcs_workspace* ws, const fcs_particles* particles,
                 int64_t n_particles, int32_t n_events, uint64_t seed, int64_t first_event, int32_t reps,
                 fcs_config* config, float* ms, cudaStream_t s) {
  if (!config) return set_err(FCS_E_ARG, "config is required");
  if (reps < 1 || reps > 1000) return set_err(FCS_E_ARG, "reps must be in [1, 1000]");
  static const int kBlocks[3] = {128, 256, 512};
  static const int kHpt[4] = {1, 2, 4, 8};
  fcs_config c{};
  c.mode = config->mode;
  c.batched = 1;
  c.wave_events = config->wave_events;
  c.energy_interp = config->energy_interp;
  c.sync = 1;
  // sizes the workspace and validates the arguments
  FCS_TRY(fcs_simulate_events(geo, prm, ws, particles, n_particles, n_events, seed, first_event, &c, nullptr, nullptr,
                              nullptr, nullptr, 0, nullptr, nullptr, s));
  if (n_events == 0) return ok();
  float best = 1e30f;
  int best_b = 256, best_h = 4;
  std::vector<float> t((size_t)reps);
  for (int ib = 0; ib < 3; ++ib) {
    for (int ih = 0; ih < 4; ++ih) {
      c.block = kBlocks[ib];
      c.hits_per_thread = kHpt[ih];
      c.sync = 0;
      c.timing = 1;
      for (int r = -1; r < reps; ++r) {
        FCS_TRY(fcs_simulate_events(geo, prm, ws, particles, n_particles, n_events, seed, first_event, &c, nullptr,
                                    nullptr, nullptr, nullptr, 0, nullptr, nullptr, s));
        float st[FCS_N_STAGES];
        FCS_TRY(fcs_workspace_timings(ws, st));
        if (r >= 0) t[(size_t)r] = st[FCS_STAGE_HITS];
      }
      std::sort(t.begin(), t.end());
      const float med = t[(size_t)reps / 2];
      if (ms) ms[ib * 4 + ih] = med;
      if (med < best) {
        best = med;
        best_b = kBlocks[ib];
        best_h = kHpt[ih];
      }
    }
  }
  fcs_stats st{};
  FCS_TRY(fcs_workspace_status(ws, &st, s));
  config->block = best_b;
  config->hits_per_thread = best_h;
  return ok();
}

int fcs_simulate_events_host(const fcs_geo* geo, const fcs_params* prm, fcs_workspace* ws, const int32_t* type,
                             const float* E, const float* eta, const float* phi, const int64_t* event_offsets,
                             int64_t n_particles, int32_t n_events, uint64_t seed, int64_t first_event,
                             const fcs_config* config, int32_t* cell_ids, float* cell_E,
                             int64_t* event_offsets_out, int64_t capacity, fcs_stats* stats, cudaStream_t s) {
  if (!geo || !prm || !ws) return set_err(FCS_E_ARG, "geo, params and workspace are required");
  if (n_particles < 0 || n_events < 0 || capacity < 0) return set_err(FCS_E_ARG, "negative size");
  if (!event_offsets || !event_offsets_out || (n_particles > 0 && (!type || !E || !eta || !phi)))
    return set_err(FCS_E_ARG, "host arrays must be non-NULL");
  if ((cell_ids == nullptr) != (cell_E == nullptr)) return set_err(FCS_E_ARG, "cell_ids and cell_E go together");
  fcs_config cfg{};
  cfg.batched = 1;
  if (config) cfg = *config;
  // sync == 0: a call that runs as the cached two-wave graph returns once it
  // is enqueued; every other call runs synchronously
  const bool enqueue_only = config && config->sync == 0;
  cfg.sync = 1;
  cfg.use_graph = 0;
  // staging: particles, offsets, outputs (16-byte aligned slices)
  auto al = [](int64_t b) { return (b + 255) / 256 * 256; };
  const int64_t b_type = al(n_particles * 4), b_f = al(n_particles * 4), b_off = al((int64_t)(n_events + 1) * 8);
  const int64_t b_ids = al(capacity * 4), b_E = al(capacity * 4);
  const int64_t need = b_type + 3 * b_f + 2 * b_off + b_ids + b_E;
  if (need > ws->stage_cap) {
    if (ws->stage) cudaFree(ws->stage);
    ws->stage = nullptr;
    ws->stage_cap = 0;
    unsigned char* p = nullptr;
    FCS_TRY(dev_alloc(&p, (size_t)need));
    ws->stage = p;
    ws->stage_cap = need;
  }
  unsigned char* base = (unsigned char*)ws->stage;
  int32_t* d_type = (int32_t*)base;
  float* d_E = (float*)(base + b_type);
  float* d_eta = (float*)(base + b_type + b_f);
  float* d_phi = (float*)(base + b_type + 2 * b_f);
  int64_t* d_off = (int64_t*)(base + b_type + 3 * b_f);
  int64_t* d_oout = (int64_t*)(base + b_type + 3 * b_f + b_off);
  int32_t* d_ids = (int32_t*)(base + b_type + 3 * b_f + 2 * b_off);
  float* d_cE = (float*)(base + b_type + 3 * b_f + 2 * b_off + b_ids);
  fcs_particles parts{d_type, d_E, d_eta, d_phi, d_off};
  fcs_stats st{};
  // Output buffers in mapped pinned host memory (cudaMallocHost, or torch's
  // pin_memory) are written by the compaction kernel directly, over the
  // CPU-GPU link, instead of through device staging and copies.
  int64_t* m_oout = (int64_t*)mapped_host(event_offsets_out);
  int32_t* m_ids = cell_ids ? (int32_t*)mapped_host(cell_ids) : nullptr;
  float* m_cE = cell_ids ? (float*)mapped_host(cell_E) : nullptr;
  const bool direct = m_oout && (!cell_ids || (m_ids && m_cE));
  if (direct && cfg.batched == 1 && ws->gmap_cap > 0) {
    // two waves on three streams: copies in, compute and the transfer of
    // results overlap (pinned inputs; see host_waves)
    const int rc2 = host_waves(geo, prm, ws, type, E, eta, phi, event_offsets, n_particles, n_events, seed,
                                   first_event, cfg, parts, m_ids, m_cE, m_oout, capacity, s);
    if (rc2 == FCS_OK && enqueue_only) {
      // fcs_workspace_status waits for the call and reports it
      if (stats) std::memset(stats, 0, sizeof(*stats));
      return ok();
    }
    if (rc2 == FCS_OK) {
      FCS_CUDA(cudaMemcpyAsync(ws->h_sizes, ws->d_sizes, sizeof(Sizes), cudaMemcpyDeviceToHost, s));
      FCS_CUDA(cudaStreamSynchronize(s));
      if (!(ws->h_sizes->flags & FCS_FLAG_HIT_CAPACITY)) return status_from(*ws->h_sizes, stats);
      FCS_TRY(ws_reserve_hits(ws, ws->h_sizes->hit_base, cfg.mode));
    } else if (rc2 != FCS_E_UNSUPPORTED) {
      return rc2;
    }
  }
  FCS_CUDA(cudaMemcpyAsync(d_type, type, n_particles * 4, cudaMemcpyHostToDevice, s));
  FCS_CUDA(cudaMemcpyAsync(d_E, E, n_particles * 4, cudaMemcpyHostToDevice, s));
  FCS_CUDA(cudaMemcpyAsync(d_eta, eta, n_particles * 4, cudaMemcpyHostToDevice, s));
  FCS_CUDA(cudaMemcpyAsync(d_phi, phi, n_particles * 4, cudaMemcpyHostToDevice, s));
  FCS_CUDA(cudaMemcpyAsync(d_off, event_offsets, (size_t)(n_events + 1) * 8, cudaMemcpyHostToDevice, s));
  if (direct) {
    // once the workspace is sized, replay the call's CUDA graph and read the
    // status; a call that outgrew the workspace runs again synchronously
    if (cfg.batched == 1 && ws->gmap_cap > 0) {
      fcs_config gcfg = cfg;
      gcfg.sync = 0;
      gcfg.use_graph = 1;
      gcfg.timing = 0;
      FCS_TRY(fcs_simulate_events(geo, prm, ws, &parts, n_particles, n_events, seed, first_event, &gcfg, nullptr,
                                  m_ids, m_cE, m_oout, capacity, nullptr, nullptr, s));
      FCS_CUDA(cudaMemcpyAsync(ws->h_sizes, ws->d_sizes, sizeof(Sizes), cudaMemcpyDeviceToHost, s));
      FCS_CUDA(cudaStreamSynchronize(s));
      if (!(ws->h_sizes->flags & FCS_FLAG_HIT_CAPACITY)) return status_from(*ws->h_sizes, stats);
      FCS_TRY(ws_reserve_hits(ws, ws->h_sizes->hit_base, cfg.mode));
    }
    const int rc = fcs_simulate_events(geo, prm, ws, &parts, n_particles, n_events, seed, first_event, &cfg, nullptr,
                                       m_ids, m_cE, m_oout, capacity, &st, nullptr, s);
    if (stats) *stats = st;
    return rc;
  }
  const int rc = fcs_simulate_events(geo, prm, ws, &parts, n_particles, n_events, seed, first_event, &cfg, nullptr,
                                     cell_ids ? d_ids : nullptr, cell_ids ? d_cE : nullptr, d_oout, capacity, &st,
                                     nullptr, s);
  if (stats) *stats = st;
  if (rc != FCS_OK && rc != FCS_E_RANGE && rc != FCS_E_DEVICE_CHECK) return rc;
  const int64_t n_out = std::min<int64_t>(st.n_nonzero, capacity);
  FCS_CUDA(cudaMemcpyAsync(event_offsets_out, d_oout, (size_t)(n_events + 1) * 8, cudaMemcpyDeviceToHost, s));
  if (cell_ids && n_out > 0) {
    FCS_CUDA(cudaMemcpyAsync(cell_ids, d_ids, n_out * 4, cudaMemcpyDeviceToHost, s));
    FCS_CUDA(cudaMemcpyAsync(cell_E, d_cE, n_out * 4, cudaMemcpyDeviceToHost, s));
  }
  FCS_CUDA(cudaStreamSynchronize(s));
  if (rc != FCS_OK) return rc;
  return ok();
}

int fcs_simulate_backward(const fcs_geo* geo, const fcs_params* prm, fcs_workspace* ws,
                          const fcs_particles* particles, int64_t n_particles, int32_t n_events, uint64_t seed,
                          int64_t first_event, const fcs_config* config, const float* dL_dcells, float* d_frac,
                          float* d_shape_w, fcs_stats* stats, cudaStream_t s) {
  if (!geo || !prm || !ws) return set_err(FCS_E_ARG, "geo, params and workspace are required");
  FCS_TRY(check_particles(particles, n_particles));
  if (n_particles < 0 || n_events < 0) return set_err(FCS_E_ARG, "negative size");
  if (n_events >= kMaxEventsPerCall) return set_err(FCS_E_RANGE, "at most 2^24 - 1 events per call");
  if (prm->d.NL != geo->d.n_layers) return set_err(FCS_E_ARG, "parametrisation and geometry disagree on layers");
  if (n_events > 0 && !dL_dcells) return set_err(FCS_E_ARG, "dL_dcells is required");
  fcs_config cfg{};
  cfg.batched = 1;
  cfg.sync = 1;
  if (config) cfg = *config;
  FCS_TRY(validate_config(cfg));
  if (cfg.use_graph) return set_err(FCS_E_ARG, "the backward pass runs without graph capture (use_graph = 0)");
  int dev = 0;
  FCS_TRY(current_device(&dev));
  if (dev != geo->device || dev != prm->device || (ws->device >= 0 && ws->device != dev))
    return set_err(FCS_E_ARG, "geometry, parametrisation and workspace must live on the current device");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n_events == 0) return ok();
  const int32_t rows = range_events(cfg, n_events);
  if ((int64_t)rows * geo->d.n_cells >= (int64_t(1) << 32))
    return set_err(FCS_E_RANGE, "%d events x %d cells exceed 2^32; split the batch", rows, geo->d.n_cells);
  FCS_TRY(ws_reserve_static(ws, geo, n_particles, 1, FCS_MODE_ATOMIC));
  const int64_t n_scores = (int64_t)prm->d.n_entries * kNBins;
  if (n_scores > ws->ga_cap || prm->d.n_entries > ws->gt_cap || ws->grad_dirty) {
    FCS_TRY(grow(&ws->grad_acc, &ws->ga_cap, n_scores, true));
    FCS_TRY(grow(&ws->grad_touched, &ws->gt_cap, (int64_t)prm->d.n_entries, true));
    if (ws->grad_dirty) {
      FCS_CUDA(cudaMemset(ws->grad_acc, 0, (size_t)ws->ga_cap * sizeof(double)));
      FCS_CUDA(cudaMemset(ws->grad_touched, 0, (size_t)ws->gt_cap));
      ws->grad_dirty = false;
    }
  }
  ws->timed_ranges = 0;
  const HitCfg hc = hit_cfg(cfg);
  const Launch L{s, ws->num_sms};
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
  const ScanTmp tmp = ws->scan_tmp();
  ws->grad_dirty = true;
  k_call_begin<<<1, 1, 0, s>>>(ws->d_sizes);
  for (int32_t lo = 0; lo < n_events; lo += rows) {
    const int32_t hi = std::min(n_events, lo + rows);
    k_range_begin<<<1, kRangeThreads, 0, s>>>(ws->d_sizes, particles->event_offsets, lo, hi, n_particles,
                                              ws->pcap);
    WsDev w = ws->view();
    FCS_CUDA(launch_task_counts(geo->d, prm->d, *particles, lo, hi, k0, k1, first_event, w, tmp, n_particles,
                                cfg.energy_interp, L));
    if (cfg.sync) {
      FCS_CUDA(cudaMemcpyAsync(ws->h_sizes, ws->d_sizes, sizeof(Sizes), cudaMemcpyDeviceToHost, s));
      FCS_CUDA(cudaStreamSynchronize(s));
      FCS_TRY(ws_reserve_hits(ws, ws->h_sizes->n_hits, FCS_MODE_ATOMIC));
      w = ws->view();
    }
    FCS_CUDA(launch_task_finish(w, nullptr, cfg.sync ? 1 : 0, n_particles * geo->d.n_layers, L));
    const float* g = dL_dcells + (int64_t)lo * geo->d.n_cells;
    FCS_CUDA(launch_hits_grad(geo->d, prm->d, w, lo, k0, k1, first_event, hc, g, ws->grad_acc, ws->grad_touched, L));
    FCS_CUDA(launch_recheck_grad(geo->d, prm->d, w, lo, k0, k1, first_event, g, ws->grad_acc, ws->grad_touched, L));
    k_range_end<<<1, 1, 0, s>>>(ws->d_sizes);
  }
  FCS_CUDA(launch_grad_finalize(prm->d, ws->grad_acc, ws->grad_touched, d_frac, d_shape_w, L));
  FCS_CUDA(cudaGetLastError());
  ws->grad_dirty = false;
  if (!cfg.sync) return ok();
  FCS_CUDA(cudaMemcpyAsync(ws->h_sizes, ws->d_sizes, sizeof(Sizes), cudaMemcpyDeviceToHost, s));
  FCS_CUDA(cudaStreamSynchronize(s));
  return status_from(*ws->h_sizes, stats);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Simulation without device allocation: the scratch buffers of the launch
// sequence live in one file-scope device array of fixed size instead of a
// cudaMalloc'd workspace.
// ---------------------------------------------------------------------------
namespace {

// Holds the intermediate buffers of fcs_simulate_events_static.  Every GPU
// that loads the library keeps this array until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[FCS_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};  // device address of g_static_scratch, per device
int g_static_sms[kMaxDevices] = {};

// Device address of the array on the current device (host code must not use
// the symbol itself, which is only a host-side stand-in).
int static_scratch(int dev, void** ptr, int* sms) {
  if (dev < 0 || dev >= kMaxDevices) return set_err(FCS_E_ARG, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return set_err(FCS_E_CUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_err(FCS_E_CUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
    g_static_ptr[dev] = p;
    g_static_sms[dev] = n;
  }
  *ptr = g_static_ptr[dev];
  *sms = g_static_sms[dev];
  return FCS_OK;
}

// Bump allocator over the array (256-byte aligned slices).
struct Carve {
  unsigned char* base;
  size_t off, cap;
  template <typename T>
  T* take(int64_t n) {
    const size_t bytes = ((size_t)std::max<int64_t>(n, 1) * sizeof(T) + 255) / 256 * 256;
    if (off + bytes > cap) return nullptr;
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

}  // namespace

extern "C" int fcs_simulate_events_static(const fcs_geo* geo, const fcs_params* prm,
                                          const fcs_particles* particles, int64_t n_particles,
                                          int32_t n_events, uint64_t seed, int64_t first_event,
                                          int32_t* cell_ids, float* cell_E, int64_t* event_offsets_out,
                                          int64_t capacity, fcs_stats* stats, cudaStream_t s) {
  if (!geo || !prm) return set_err(FCS_E_ARG, "geo and params are required");
  FCS_TRY(check_particles(particles, n_particles));
  if (n_particles < 0 || n_events < 0 || capacity < 0) return set_err(FCS_E_ARG, "bad size");
  if (n_events >= kMaxEventsPerCall) return set_err(FCS_E_RANGE, "at most 2^24 - 1 events per call");
  if (!event_offsets_out) return set_err(FCS_E_ARG, "event_offsets_out is required");
  if ((cell_ids == nullptr) != (cell_E == nullptr)) return set_err(FCS_E_ARG, "cell_ids and cell_E go together");
  if (prm->d.NL != geo->d.n_layers) return set_err(FCS_E_ARG, "parametrisation and geometry disagree on layers");
  int dev = 0;
  FCS_TRY(current_device(&dev));
  if (dev != geo->device || dev != prm->device)
    return set_err(FCS_E_ARG, "geometry and parametrisation must live on the current device");
  if (n_events == 0) {  // as fcs_simulate_events: an empty output, zeroed statistics
    k_empty_offsets<<<1, 32, 0, s>>>(event_offsets_out, 0);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    FCS_CUDA(cudaGetLastError());
    FCS_CUDA(cudaStreamSynchronize(s));
    return ok();
  }
  void* base = nullptr;
  int sms = 0;
  FCS_TRY(static_scratch(dev, &base, &sms));

  // Carve the workspace buffers for this call out of the array.
  const int NL = geo->d.n_layers;
  const int64_t P = std::max<int64_t>(n_particles, 1);
  const int64_t recheck_cap = 32768;
  fcs_workspace w;  // views only: pointers into the static array, nulled before return
  w.device = dev;
  w.num_sms = sms;
  Carve c{(unsigned char*)base, 0, (size_t)FCS_STATIC_SCRATCH_BYTES};
  w.d_sizes = c.take<Sizes>(1);
  w.pcount = c.take<int64_t>(P);
  w.poff = c.take<int64_t>(P);
  w.pinfo = c.take<uint4>(P);
  w.pcap = P;
  w.tasks = c.take<TaskRec>(P * NL);
  w.tehit = c.take<float>(P * NL);
  w.tn = c.take<int32_t>(P * NL);
  w.th = c.take<int64_t>(P * NL);
  w.pdefer = c.take<int32_t>(P * NL);
  w.pd_cap = P * NL;
  w.task_cap = P * NL;
  w.acc = c.take<double>((int64_t)n_events * geo->d.acc_stride);
  w.rows_cap = n_events;
  w.acc_stride = geo->d.acc_stride;
  const int64_t chunks = compact_chunks(geo->d.n_cells, n_events);
  w.ss_cap = std::max(scan_state_words(std::max({P * NL, (int64_t)n_events * geo->d.acc_stride, chunks})), chunks + 2);
  w.scan_state = c.take<uint64_t>(w.ss_cap);
  w.recheck = c.take<uint2>(recheck_cap);
  w.recheck_cap = recheck_cap;
  const bool fits = w.d_sizes && w.pcount && w.poff && w.pinfo && w.tasks && w.tehit && w.tn && w.th && w.pdefer &&
                    w.acc &&
                    w.scan_state && w.recheck && c.cap - c.off >= 4096;
  if (fits) {
    // the rest of the array maps tiles to tasks: it bounds the hits per call
    w.gmap_cap = (int64_t)((c.cap - c.off) / sizeof(int32_t));
    w.gmap = reinterpret_cast<int32_t*>((unsigned char*)base + c.off);
  }
  auto release = [&]() {  // the array is not the workspace's to free
    w.d_sizes = nullptr;
    w.pcount = nullptr;
    w.poff = nullptr;
    w.pinfo = nullptr;
    w.tasks = nullptr;
    w.tehit = nullptr;
    w.tn = nullptr;
    w.th = nullptr;
    w.pdefer = nullptr;
    w.acc = nullptr;
    w.scan_state = nullptr;
    w.recheck = nullptr;
    w.gmap = nullptr;
  };
  if (!fits) {
    release();
    return set_err(FCS_E_RANGE,
                   "static scratch of %d bytes is too small for %lld particles x %d layers and %d events of %d "
                   "cells; use fcs_simulate_events",
                   (int)FCS_STATIC_SCRATCH_BYTES, (long long)n_particles, NL, n_events, geo->d.n_cells);
  }
  fcs_config cfg{};
  cfg.mode = FCS_MODE_ATOMIC;
  cfg.batched = 1;
  cfg.sync = 1;
  // the array keeps the previous call's contents: the accumulation rows and
  // the scan state must start at zero
  int rc = FCS_OK;
  cudaError_t e = cudaMemsetAsync(w.acc, 0, (size_t)n_events * geo->d.acc_stride * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.scan_state, 0, (size_t)w.ss_cap * sizeof(uint64_t), s);
  if (e != cudaSuccess) rc = set_err(FCS_E_CUDA, "clearing the static scratch: %s", cudaGetErrorString(e));
  if (rc == FCS_OK) {
    CallArgs a{geo, prm, &w, *particles, n_particles, n_events, seed, first_event, cfg, nullptr,
               cell_ids, cell_E, event_offsets_out, capacity, nullptr, s};
    const HitCfg hc = hit_cfg(cfg);
    const int key_task_bits = bits_for(P * NL);
    rc = enqueue_call(a, false, hc, key_task_bits);
  }
  Sizes h{};
  if (rc == FCS_OK) {
    e = cudaMemcpyAsync(&h, w.d_sizes, sizeof(Sizes), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = set_err(FCS_E_CUDA, "reading the call status: %s", cudaGetErrorString(e));
  }
  release();
  if (rc != FCS_OK) return rc;
  if (h.flags & FCS_FLAG_HIT_CAPACITY) {
    if (stats) status_from(h, stats);
    return set_err(FCS_E_RANGE, "the call produced more hits than the static scratch maps (%lld > %lld)",
                   (long long)h.hit_base, (long long)(w.gmap_cap * kGranule));
  }
  return status_from(h, stats);
}
