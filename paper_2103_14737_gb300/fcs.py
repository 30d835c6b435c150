"""Python binding of the libfcs C ABI (include/fcs.h).

Thin ctypes marshalling: every ``fcs_*`` function below has the name of the C
entry point it calls and only converts arguments (torch tensors -> device
pointers, numpy arrays -> host pointers, the current torch stream -> its
cudaStream_t).  All work runs in the library's CUDA kernels; there is no CPU
fallback, and loading fails with an exception when the library is missing.

``Simulator`` bundles geometry, parametrisation and workspace for callers that
hold torch tensors.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

FCS_OK, FCS_E_ARG, FCS_E_RANGE, FCS_E_OOM, FCS_E_CUDA, FCS_E_DEVICE_CHECK, FCS_E_TIMEOUT, FCS_E_UNSUPPORTED = range(8)
FLAG_BAD_PARTICLE, FLAG_HIT_CAPACITY, FLAG_OUT_CAPACITY, FLAG_KEY_BITS, FLAG_RECHECK_SPILL, FLAG_BAD_OFFSETS = \
    (1 << i for i in range(6))
MODE_ATOMIC, MODE_DETERMINISTIC = 0, 1

EXPORTED = ("fcs_version", "fcs_last_error", "fcs_load_geometry", "fcs_geometry_info", "fcs_free_geometry",
            "fcs_load_params", "fcs_free_params", "fcs_workspace_create", "fcs_workspace_reserve",
            "fcs_workspace_status", "fcs_workspace_timings", "fcs_workspace_graph_kernels", "fcs_workspace_free",
            "fcs_selftest_wait_timeout",
            "fcs_simulate_events", "fcs_simulate_events_host",
            "fcs_simulate_events_static", "fcs_autotune", "fcs_microbench", "fcs_simulate_backward",
            "fcs_update_params", "fcs_poisson_audit")


class FcsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libfcs error {code}: {msg}")
        self.code = code


class fcs_particles(C.Structure):
    _fields_ = [("type", C.c_void_p), ("E", C.c_void_p), ("eta", C.c_void_p), ("phi", C.c_void_p),
                ("event_offsets", C.c_void_p)]


class fcs_config(C.Structure):
    _fields_ = [("mode", C.c_int32), ("batched", C.c_int32), ("hits_per_thread", C.c_int32),
                ("block", C.c_int32), ("sync", C.c_int32), ("use_graph", C.c_int32),
                ("timing", C.c_int32), ("wave_events", C.c_int32), ("energy_interp", C.c_int32),
                ("reserved", C.c_int32)]


class fcs_stats(C.Structure):
    _fields_ = [("n_tasks", C.c_int64), ("n_hits", C.c_int64), ("n_nonzero", C.c_int64),
                ("n_recheck", C.c_int64), ("device_flags", C.c_uint32), ("n_poisson_fp64", C.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class fcs_debug(C.Structure):
    _fields_ = [("task_capacity", C.c_int64), ("task_event", C.c_void_p), ("task_particle", C.c_void_p),
                ("task_layer", C.c_void_p), ("task_n", C.c_void_p), ("task_Ehit", C.c_void_p),
                ("hit_capacity", C.c_int64), ("hit_cell", C.c_void_p), ("hit_bin", C.c_void_p)]


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load libfcs.so; raises if it cannot be built or loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # FCS_LIBRARY selects another build of the same ABI (e.g. a tuned variant)
        path = os.environ.get("FCS_LIBRARY") or _build.LIB
        if build_if_missing and not os.environ.get("FCS_LIBRARY"):
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libfcs.so not found at {path}; run __graft_entry__.build()")
        L = C.CDLL(path)
        vp, i32, i64, u64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
        L.fcs_version.restype = C.c_char_p
        L.fcs_last_error.argtypes = [C.c_char_p, C.c_size_t]
        L.fcs_last_error.restype = C.c_int
        L.fcs_load_geometry.argtypes = [C.POINTER(vp), vp, i32, vp, i32, vp, vp]
        L.fcs_geometry_info.argtypes = [vp, vp, vp, vp]
        L.fcs_free_geometry.argtypes = [vp]
        L.fcs_free_geometry.restype = None
        L.fcs_load_params.argtypes = [C.POINTER(vp), vp, vp, vp, vp, vp, vp, i32, i32, i32, i32, i32, f64, i32, vp]
        L.fcs_free_params.argtypes = [vp]
        L.fcs_free_params.restype = None
        L.fcs_workspace_create.argtypes = [C.POINTER(vp)]
        L.fcs_workspace_reserve.argtypes = [vp, vp, i64, i32, i64, i32]
        L.fcs_workspace_status.argtypes = [vp, vp, vp]
        L.fcs_workspace_timings.argtypes = [vp, vp]
        L.fcs_workspace_graph_kernels.argtypes = [vp, vp]
        L.fcs_selftest_wait_timeout.argtypes = [vp, vp]
        L.fcs_workspace_free.argtypes = [vp]
        L.fcs_workspace_free.restype = None
        L.fcs_simulate_events.argtypes = [vp, vp, vp, vp, i64, i32, u64, i64, vp, vp, vp, vp, vp, i64, vp, vp, vp]
        L.fcs_simulate_events_host.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, i64, i32, u64, i64, vp, vp, vp, vp,
                                               i64, vp, vp]
        L.fcs_simulate_events_static.argtypes = [vp, vp, vp, i64, i32, u64, i64, vp, vp, vp, i64, vp, vp]
        L.fcs_autotune.argtypes = [vp, vp, vp, vp, i64, i32, u64, i64, i32, vp, vp, vp]
        L.fcs_microbench.argtypes = [i32, i64, i32, vp, vp]
        L.fcs_simulate_backward.argtypes = [vp, vp, vp, vp, i64, i32, u64, i64, vp, vp, vp, vp, vp, vp]
        L.fcs_update_params.argtypes = [vp, vp, vp, vp, vp]
        L.fcs_poisson_audit.argtypes = [vp, vp, i64, u64, vp, vp, vp]
        # every other entry point returns an int status (the ctypes default restype)
        _lib = L
        return L


def _check(rc):
    if rc != FCS_OK:
        buf = C.create_string_buffer(512)
        _lib.fcs_last_error(buf, 512)
        raise FcsError(rc, buf.value.decode(errors="replace"))


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _np(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def fcs_version() -> str:
    return load_library().fcs_version().decode()


def fcs_load_geometry(regions: np.ndarray, layer_region_begin: np.ndarray, layers: np.ndarray):
    L = load_library()
    reg, p_reg = _np(regions, regions.dtype)
    lrb, p_lrb = _np(layer_region_begin, np.int32)
    lay, p_lay = _np(layers, layers.dtype)
    assert reg.dtype.itemsize == 48 and lay.dtype.itemsize == 16
    out = C.c_void_p()
    _check(L.fcs_load_geometry(C.byref(out), p_reg, len(reg), p_lrb, len(lrb) - 1, p_lay, _stream()))
    return out


def fcs_geometry_info(geo):
    L = load_library()
    n = [C.c_int32(), C.c_int32(), C.c_int32()]
    _check(L.fcs_geometry_info(geo, C.byref(n[0]), C.byref(n[1]), C.byref(n[2])))
    return tuple(v.value for v in n)


def fcs_free_geometry(geo):
    load_library().fcs_free_geometry(geo)


def fcs_load_params(geo, frac, mean_hit_E, shape_w, r_edges, a_edges, eta_bin_scale=20.0, ebin_log2_min=6):
    L = load_library()
    NT, NE, NH, NL = frac.shape
    NR, NA = shape_w.shape[-2:]
    f, pf = _np(frac, np.float32)
    m, pm = _np(mean_hit_E, np.float32)
    w, pw = _np(shape_w, np.float32)
    re, pre = _np(r_edges, np.float32)
    ae, pae = _np(a_edges, np.float32)
    out = C.c_void_p()
    _check(L.fcs_load_params(C.byref(out), geo, pf, pm, pw, pre, pae, NT, NE, NH, NR, NA, float(eta_bin_scale),
                             int(ebin_log2_min), _stream()))
    return out


def fcs_free_params(prm):
    load_library().fcs_free_params(prm)


def fcs_workspace_create():
    L = load_library()
    out = C.c_void_p()
    _check(L.fcs_workspace_create(C.byref(out)))
    return out


def fcs_workspace_reserve(ws, geo, n_particles, n_events, n_hits, mode=MODE_ATOMIC):
    _check(load_library().fcs_workspace_reserve(ws, geo, n_particles, n_events, n_hits, mode))


def fcs_workspace_status(ws):
    st = fcs_stats()
    rc = load_library().fcs_workspace_status(ws, C.byref(st), _stream())
    return rc, st


STAGES = ("tasks", "hits", "recheck", "reduce", "total")


def fcs_workspace_timings(ws):
    """Stage times (ms) of the last timed call on ws."""
    ms = (C.c_float * len(STAGES))()
    _check(load_library().fcs_workspace_timings(ws, ms))
    return dict(zip(STAGES, [float(v) for v in ms]))


def fcs_workspace_graph_kernels(ws):
    """Kernel launches of one replay of the workspace's cached CUDA graph."""
    n = C.c_int64()
    _check(load_library().fcs_workspace_graph_kernels(ws, C.byref(n)))
    return n.value


def fcs_selftest_wait_timeout():
    """Runs the bounded-wait self-test; returns (status, kernel ms).  The
    expected status is FCS_E_TIMEOUT."""
    ms = C.c_float()
    rc = load_library().fcs_selftest_wait_timeout(C.byref(ms), _stream())
    return rc, ms.value


def fcs_workspace_free(ws):
    load_library().fcs_workspace_free(ws)


def make_config(mode=MODE_ATOMIC, batched=1, hits_per_thread=0, block=0, sync=1, use_graph=0, timing=0,
                wave_events=0, energy_interp=0):
    c = fcs_config()
    c.mode, c.batched, c.hits_per_thread, c.block, c.sync, c.use_graph, c.timing, c.wave_events = \
        mode, batched, hits_per_thread, block, sync, use_graph, timing, wave_events
    c.energy_interp = energy_interp
    return c


def fcs_simulate_events(geo, prm, ws, particles: fcs_particles, n_particles, n_events, seed, first_event, config,
                        cells_out=None, cell_ids=None, cell_E=None, event_offsets_out=None, capacity=0,
                        debug: fcs_debug | None = None, check=True):
    """Calls fcs_simulate_events on the current torch stream; tensors are device tensors.
    Returns (status, fcs_stats)."""
    L = load_library()
    st = fcs_stats()
    rc = L.fcs_simulate_events(geo, prm, ws, C.byref(particles), int(n_particles), int(n_events),
                               int(seed) & 0xFFFFFFFFFFFFFFFF, int(first_event), C.byref(config), _ptr(cells_out),
                               _ptr(cell_ids), _ptr(cell_E), _ptr(event_offsets_out), int(capacity), C.byref(st),
                               C.byref(debug) if debug is not None else None, _stream())
    if check and rc != FCS_OK:
        _check(rc)
    return rc, st


def fcs_simulate_events_host(geo, prm, ws, type_, E, eta, phi, event_offsets, seed, first_event, config,
                             cell_ids, cell_E, event_offsets_out, check=True):
    """Host-buffer end-to-end call: numpy arrays in, numpy arrays filled."""
    L = load_library()
    st = fcs_stats()
    n_events = len(event_offsets) - 1
    for a in (type_, E, eta, phi, event_offsets, cell_ids, cell_E, event_offsets_out):
        assert a.flags["C_CONTIGUOUS"]
    rc = L.fcs_simulate_events_host(geo, prm, ws, type_.ctypes.data_as(C.c_void_p), E.ctypes.data_as(C.c_void_p),
                                    eta.ctypes.data_as(C.c_void_p), phi.ctypes.data_as(C.c_void_p),
                                    event_offsets.ctypes.data_as(C.c_void_p), len(E), n_events,
                                    int(seed) & 0xFFFFFFFFFFFFFFFF, int(first_event), C.byref(config),
                                    cell_ids.ctypes.data_as(C.c_void_p), cell_E.ctypes.data_as(C.c_void_p),
                                    event_offsets_out.ctypes.data_as(C.c_void_p), len(cell_ids), C.byref(st),
                                    _stream())
    if check and rc != FCS_OK:
        _check(rc)
    return rc, st


MB_PHILOX, MB_MULWIDE, MB_LOP3, MB_FFMA, MB_RED, MB_MUFU, MB_LDS, MB_RED64 = range(8)


def fcs_microbench(kind, size=0, iters=256):
    """Operations per second of one unit microbenchmark (see include/fcs.h)."""
    rate = C.c_double()
    _check(load_library().fcs_microbench(int(kind), int(size), int(iters), C.byref(rate), _stream()))
    return rate.value


def fcs_poisson_audit(prm, mu, seed):
    """FP32-path and FP64-definition Poisson counts of draws i = 0..n-1 with
    means mu (a CUDA float32 tensor), as two CUDA int32 tensors (see
    include/fcs.h for the codes of uncertain FP32 draws)."""
    import torch
    n = mu.numel()
    n32 = torch.empty(n, dtype=torch.int32, device=mu.device)
    n64 = torch.empty(n, dtype=torch.int32, device=mu.device)
    _check(load_library().fcs_poisson_audit(prm, mu.data_ptr(), n, int(seed) & 0xFFFFFFFFFFFFFFFF, n32.data_ptr(),
                                            n64.data_ptr(), _stream()))
    return n32, n64


AUTOTUNE_BLOCKS = (128, 256, 512)
AUTOTUNE_HPT = (1, 2, 4, 8)


def fcs_autotune(geo, prm, ws, particles: fcs_particles, n_particles, n_events, seed, first_event, reps=3,
                 mode=MODE_ATOMIC, wave_events=0):
    """Times every (block, hits_per_thread) shape of the hit kernel on this
    workload; returns (block, hits_per_thread, {(block, hpt): median ms})."""
    L = load_library()
    cfg = make_config(mode=mode, wave_events=wave_events)
    ms = (C.c_float * 12)()
    _check(L.fcs_autotune(geo, prm, ws, C.byref(particles), int(n_particles), int(n_events),
                          int(seed) & 0xFFFFFFFFFFFFFFFF, int(first_event), int(reps), C.byref(cfg), ms, _stream()))
    table = {(b, h): float(ms[i * 4 + j]) for i, b in enumerate(AUTOTUNE_BLOCKS) for j, h in enumerate(AUTOTUNE_HPT)}
    return cfg.block, cfg.hits_per_thread, table


STATIC_SCRATCH_BYTES = 16 * 1024 * 1024


def fcs_simulate_events_static(geo, prm, particles: fcs_particles, n_particles, n_events, seed, first_event,
                               cell_ids, cell_E, event_offsets_out, check=True):
    """The allocation-free entry point (scratch in the library's static device
    array); device tensors in and out, synchronous.  Returns (status, fcs_stats)."""
    L = load_library()
    st = fcs_stats()
    rc = L.fcs_simulate_events_static(geo, prm, C.byref(particles), int(n_particles), int(n_events),
                                      int(seed) & 0xFFFFFFFFFFFFFFFF, int(first_event), _ptr(cell_ids), _ptr(cell_E),
                                      _ptr(event_offsets_out), int(cell_ids.numel()) if cell_ids is not None else 0,
                                      C.byref(st), _stream())
    if check and rc != FCS_OK:
        _check(rc)
    return rc, st


def fcs_simulate_backward(geo, prm, ws, particles: fcs_particles, n_particles, n_events, seed, first_event,
                          config, dL_dcells, d_frac, d_shape_w, check=True):
    """Adjoint of fcs_simulate_events: accumulates dL/dfrac and dL/dshape_w
    (device tensors or None) for dL/dE_cell given as dense device rows."""
    L = load_library()
    st = fcs_stats()
    rc = L.fcs_simulate_backward(geo, prm, ws, C.byref(particles), int(n_particles), int(n_events),
                                 int(seed) & 0xFFFFFFFFFFFFFFFF, int(first_event), C.byref(config), _ptr(dL_dcells),
                                 _ptr(d_frac), _ptr(d_shape_w), C.byref(st), _stream())
    if check and rc != FCS_OK:
        _check(rc)
    return rc, st


def fcs_update_params(prm, frac=None, mean_hit_E=None, shape_w=None):
    """Replaces tables of a loaded parametrisation from device tensors."""
    _check(load_library().fcs_update_params(prm, _ptr(frac), _ptr(mean_hit_E), _ptr(shape_w), _stream()))


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
class Simulator:
    """Geometry + parametrisation + workspace on the current CUDA device."""

    def __init__(self, geo, prm):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libfcs needs a CUDA device; there is no CPU path")
        load_library()
        self.n_layers = geo.n_layers
        self.geo = fcs_load_geometry(geo.regions, geo.layer_region_begin, geo.layers)
        self.n_cells = fcs_geometry_info(self.geo)[0]
        self.prm = fcs_load_params(self.geo, prm.frac, prm.mean_hit_E, prm.shape_w, prm.r_edges, prm.a_edges,
                                   prm.eta_bin_scale, prm.ebin_log2_min)
        self.n_entries = int(np.prod(np.shape(prm.frac)))
        self.ws = fcs_workspace_create()

    def close(self):
        if getattr(self, "ws", None):
            fcs_workspace_free(self.ws)
            self.ws = None
        if getattr(self, "prm", None):
            fcs_free_params(self.prm)
            self.prm = None
        if getattr(self, "geo", None):
            fcs_free_geometry(self.geo)
            self.geo = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, dparts, seed, first_event=0, reps=3, mode=MODE_ATOMIC, wave_events=0):
        parts = fcs_particles(dparts["type"].data_ptr(), dparts["E"].data_ptr(), dparts["eta"].data_ptr(),
                              dparts["phi"].data_ptr(), dparts["event_offsets"].data_ptr())
        return fcs_autotune(self.geo, self.prm, self.ws, parts, dparts["E"].numel(),
                            dparts["event_offsets"].numel() - 1, seed, first_event, reps, mode, wave_events)

    @staticmethod
    def to_device(parts, device="cuda"):
        """synth.Particles -> dict of device tensors."""
        import torch
        return dict(type=torch.as_tensor(parts.type, dtype=torch.int32, device=device),
                    E=torch.as_tensor(parts.E, dtype=torch.float32, device=device),
                    eta=torch.as_tensor(parts.eta, dtype=torch.float32, device=device),
                    phi=torch.as_tensor(parts.phi, dtype=torch.float32, device=device),
                    event_offsets=torch.as_tensor(parts.event_offsets, dtype=torch.int64, device=device))

    def simulate(self, dparts, seed, first_event=0, mode=MODE_ATOMIC, batched=1, hits_per_thread=0, block=0,
                 sync=1, use_graph=0, dense=False, capacity=None, debug_tasks=0, debug_hits=0, outputs=None,
                 check=True, timing=0, wave_events=0, energy_interp=0):
        """Runs one call.  dparts: dict of device tensors (see to_device).
        Returns a dict with cell_ids, cell_E, event_offsets (device tensors),
        cells (dense, if requested), stats, status and debug dumps."""
        import torch
        dev = dparts["E"].device
        n_events = dparts["event_offsets"].numel() - 1
        n_particles = dparts["E"].numel()
        if outputs is None:
            cap = capacity if capacity is not None else min(n_events * self.n_cells, 1 << 28)
            outputs = dict(cell_ids=torch.empty(cap, dtype=torch.int32, device=dev),
                           cell_E=torch.empty(cap, dtype=torch.float32, device=dev),
                           event_offsets=torch.empty(n_events + 1, dtype=torch.int64, device=dev),
                           cells=torch.empty((n_events, self.n_cells), dtype=torch.float32, device=dev)
                           if dense else None)
        parts = fcs_particles(dparts["type"].data_ptr(), dparts["E"].data_ptr(), dparts["eta"].data_ptr(),
                              dparts["phi"].data_ptr(), dparts["event_offsets"].data_ptr())
        dbg = None
        res = dict(outputs)
        if debug_tasks or debug_hits:
            dbg = fcs_debug()
            if debug_tasks:
                for k, dt in (("task_event", torch.int32), ("task_particle", torch.int32), ("task_layer", torch.int32),
                              ("task_n", torch.int32), ("task_Ehit", torch.float32)):
                    res[k] = torch.full((debug_tasks,), -1, dtype=dt, device=dev)
                    setattr(dbg, k, res[k].data_ptr())
                dbg.task_capacity = debug_tasks
            if debug_hits:
                res["hit_cell"] = torch.full((debug_hits,), -1, dtype=torch.int32, device=dev)
                res["hit_bin"] = torch.full((debug_hits,), -1, dtype=torch.int16, device=dev)
                dbg.hit_cell = res["hit_cell"].data_ptr()
                dbg.hit_bin = res["hit_bin"].data_ptr()
                dbg.hit_capacity = debug_hits
        cfg = make_config(mode, batched, hits_per_thread, block, sync, use_graph, timing, wave_events, energy_interp)
        rc, st = fcs_simulate_events(self.geo, self.prm, self.ws, parts, n_particles, n_events, seed, first_event,
                                     cfg, outputs.get("cells"), outputs.get("cell_ids"), outputs.get("cell_E"),
                                     outputs.get("event_offsets"),
                                     outputs["cell_ids"].numel() if outputs.get("cell_ids") is not None else 0, dbg,
                                     check=check)
        res["status"] = rc
        res["stats"] = st.as_dict()
        res["_keep"] = (parts, dbg, cfg)
        return res

    def update_params(self, frac=None, mean_hit_E=None, shape_w=None):
        """Loads new tables from contiguous float32 device tensors (None keeps one)."""
        for t in (frac, mean_hit_E, shape_w):
            if t is not None and (not t.is_cuda or t.dtype.itemsize != 4 or not t.is_contiguous()):
                raise ValueError("update_params wants contiguous float32 CUDA tensors")
        fcs_update_params(self.prm, frac, mean_hit_E, shape_w)

    def backward(self, dparts, seed, dL_dcells, first_event=0, d_frac=None, d_shape_w=None, batched=1,
                 hits_per_thread=0, block=0, sync=1, check=True, wave_events=0, energy_interp=0):
        """Gradients of a loss with dL/dE_cell = dL_dcells ([n_events][n_cells]
        float32 on the device) with respect to the layer fractions and shape
        weights; accumulated into d_frac / d_shape_w (flat float32 device
        tensors, allocated zeroed when None)."""
        import torch
        dev = dparts["E"].device
        n_events = dparts["event_offsets"].numel() - 1
        n_particles = dparts["E"].numel()
        if d_frac is None:
            d_frac = torch.zeros(self.n_entries, dtype=torch.float32, device=dev)
        if d_shape_w is None:
            d_shape_w = torch.zeros(self.n_entries * 128, dtype=torch.float32, device=dev)
        g = dL_dcells.contiguous()
        if g.dtype != torch.float32 or g.numel() != n_events * self.n_cells:
            raise ValueError("dL_dcells must be float32 [n_events][n_cells]")
        parts = fcs_particles(dparts["type"].data_ptr(), dparts["E"].data_ptr(), dparts["eta"].data_ptr(),
                              dparts["phi"].data_ptr(), dparts["event_offsets"].data_ptr())
        cfg = make_config(MODE_ATOMIC, batched, hits_per_thread, block, sync, 0, 0, wave_events, energy_interp)
        rc, st = fcs_simulate_backward(self.geo, self.prm, self.ws, parts, n_particles, n_events, seed, first_event,
                                       cfg, g, d_frac, d_shape_w, check=check)
        return dict(d_frac=d_frac, d_shape_w=d_shape_w, status=rc, stats=st.as_dict(), _keep=(parts, cfg, g))
