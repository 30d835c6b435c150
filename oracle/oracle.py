"""ctypes wrapper of the plain-C FP64 oracle (fcs_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke entry and by the
benchmark's CPU-baseline leg.  The CUDA library never imports it.

``build()`` compiles ``fcs_oracle.c`` with gcc (-O2 -ffp-contract=off) into
``oracle/_build/liboracle.so``; the functions below marshal numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fcs_oracle.c")
HDR = os.path.join(HERE, "fcs_oracle.h")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, single threaded) if it is missing or stale."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stale = force or not os.path.exists(LIB) or max(os.path.getmtime(SRC), os.path.getmtime(HDR)) > os.path.getmtime(LIB)
    if stale:
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


class _Region(C.Structure):
    _fields_ = [("eta_lo", C.c_double), ("deta", C.c_double), ("phi_lo", C.c_double),
                ("dphi", C.c_double), ("n_eta", C.c_int32), ("n_phi", C.c_int32),
                ("cell_offset", C.c_int32), ("layer", C.c_int32)]


class _Layer(C.Structure):
    _fields_ = [("rz", C.c_double), ("barrel", C.c_int32), ("pad", C.c_int32)]


class _Geometry(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("n_regions", C.c_int32), ("n_cells", C.c_int32),
                ("regions", C.c_void_p), ("layer_region_begin", C.c_void_p), ("layers", C.c_void_p)]


class _Params(C.Structure):
    _fields_ = [("NT", C.c_int32), ("NE", C.c_int32), ("NH", C.c_int32), ("NL", C.c_int32),
                ("NR", C.c_int32), ("NA", C.c_int32),
                ("frac", C.c_void_p), ("mean_hit_E", C.c_void_p), ("shape_w", C.c_void_p),
                ("r_edges", C.c_void_p), ("a_edges", C.c_void_p),
                ("eta_bin_scale", C.c_double), ("ebin_log2_min", C.c_int32), ("energy_interp", C.c_int32)]


class _Outputs(C.Structure):
    _fields_ = [("cells64", C.c_void_p), ("cells_canon", C.c_void_p),
                ("task_cap", C.c_int64),
                ("task_event", C.c_void_p), ("task_particle", C.c_void_p), ("task_layer", C.c_void_p),
                ("task_n", C.c_void_p), ("task_Ehit", C.c_void_p),
                ("hit_cap", C.c_int64),
                ("hit_cell", C.c_void_p), ("hit_bin", C.c_void_p), ("hit_eta", C.c_void_p),
                ("hit_phi", C.c_void_p), ("hit_r", C.c_void_p), ("hit_alpha", C.c_void_p),
                ("n_tasks", C.c_int64), ("n_hits", C.c_int64), ("E_layers", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # FCS_ORACLE_LIB lets a test load a deliberately altered oracle build
            # (mutation checks of the pins); default is the normal build.
            path = os.environ.get("FCS_ORACLE_LIB") or build()
            _lib = C.CDLL(path)
            L = _lib
            vp = C.c_void_p
            L.orc_version.restype = C.c_char_p
            L.orc_philox_n.argtypes = [C.c_int64, vp, vp, vp]
            L.orc_poisson_n.argtypes = [C.c_int64, vp, vp, vp, vp, vp, vp]
            L.orc_ptrs_iter_n.argtypes = [C.c_int64, C.c_double, vp, vp, vp]
            L.orc_param_entry.argtypes = [vp, C.c_int32, C.c_float, C.c_float]
            L.orc_param_entry.restype = C.c_int32
            L.orc_thresholds.argtypes = [vp, C.c_int32, vp, vp]
            L.orc_thresholds.restype = C.c_int32
            L.orc_sample_bin.argtypes = [vp, C.c_int32, C.c_uint32]
            L.orc_sample_bin.restype = C.c_int32
            L.orc_scales.argtypes = [vp, C.c_int32, C.c_double, vp, vp]
            L.orc_cell_n.argtypes = [vp, C.c_int64, vp, vp, vp, vp]
            L.orc_simulate.argtypes = [vp, vp, C.c_int64, vp, vp, vp, vp, C.c_int32, vp, C.c_uint64,
                                       C.c_int64, vp]
            L.orc_simulate.restype = C.c_int32
            L.orc_param_entry_rng.argtypes = [vp, C.c_int32, C.c_float, C.c_float, vp, C.c_uint32, C.c_uint32]
            L.orc_param_entry_rng.restype = C.c_int32
            L.orc_reweighted_cells.argtypes = [vp, vp, C.c_int64, vp, vp, vp, vp, C.c_int32, vp, C.c_uint64,
                                               C.c_int64, C.c_int64, C.c_double, C.c_int64, C.c_int32,
                                               C.c_double, vp]
            L.orc_reweighted_cells.restype = C.c_int32
            L.orc_backward.argtypes = [vp, vp, C.c_int64, vp, vp, vp, vp, C.c_int32, vp, C.c_uint64, C.c_int64,
                                       vp, vp, vp]
            L.orc_backward.restype = C.c_int32
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleGeometry:
    """Keeps the numpy arrays alive behind an ``orc_geometry`` struct."""

    def __init__(self, geo):
        self.regions = np.ascontiguousarray(geo.regions)
        self.lrb = np.ascontiguousarray(geo.layer_region_begin, dtype=np.int32)
        self.layers = np.ascontiguousarray(geo.layers)
        self.n_cells = int(geo.n_cells)
        self.n_layers = int(geo.n_layers)
        self.s = _Geometry(self.n_layers, len(self.regions), self.n_cells, self.regions.ctypes.data,
                           self.lrb.ctypes.data, self.layers.ctypes.data)

    @property
    def ptr(self):
        return C.byref(self.s)


class OracleParams:
    def __init__(self, prm, energy_interp: int = 0):
        self.frac = np.ascontiguousarray(prm.frac, dtype=np.float32)
        self.mhe = np.ascontiguousarray(prm.mean_hit_E, dtype=np.float32)
        self.w = np.ascontiguousarray(prm.shape_w, dtype=np.float32)
        self.re = np.ascontiguousarray(prm.r_edges, dtype=np.float32)
        self.ae = np.ascontiguousarray(prm.a_edges, dtype=np.float32)
        NT, NE, NH, NL = self.frac.shape
        NR, NA = self.w.shape[-2:]
        self.s = _Params(NT, NE, NH, NL, NR, NA, self.frac.ctypes.data, self.mhe.ctypes.data,
                         self.w.ctypes.data, self.re.ctypes.data, self.ae.ctypes.data,
                         float(prm.eta_bin_scale), int(prm.ebin_log2_min), int(energy_interp))

    @property
    def ptr(self):
        return C.byref(self.s)


# ----------------------------------------------------------------------------
# Element functions
# ----------------------------------------------------------------------------
def key_of(seed: int) -> np.ndarray:
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)


def philox(ctr: np.ndarray, seed: int) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    k = key_of(seed)
    lib().orc_philox_n(len(ctr), _p(ctr), _p(k), _p(out))
    return out


def poisson(mu, seed: int, layer, particle, event) -> np.ndarray:
    mu = np.ascontiguousarray(mu, dtype=np.float64).ravel()
    n = len(mu)
    lay = np.ascontiguousarray(np.broadcast_to(layer, n), dtype=np.uint32)
    par = np.ascontiguousarray(np.broadcast_to(particle, n), dtype=np.uint32)
    ev = np.ascontiguousarray(np.broadcast_to(event, n), dtype=np.uint32)
    out = np.empty(n, dtype=np.int64)
    k = key_of(seed)
    lib().orc_poisson_n(n, _p(mu), _p(k), _p(lay), _p(par), _p(ev), _p(out))
    return out


def ptrs_iter(mu: float, u, V) -> np.ndarray:
    """One PTRS iteration per (u, V) pair: the accepted count or -1."""
    u = np.ascontiguousarray(u, dtype=np.float64).ravel()
    V = np.ascontiguousarray(np.broadcast_to(V, u.shape), dtype=np.float64)
    out = np.empty(len(u), dtype=np.int64)
    lib().orc_ptrs_iter_n(len(u), float(mu), _p(u), _p(V), _p(out))
    return out


def param_entry(oprm: OracleParams, ptype: int, E: float, eta: float) -> int:
    return int(lib().orc_param_entry(oprm.ptr, ptype, E, eta))


def param_entry_rng(oprm: OracleParams, ptype: int, E: float, eta: float, seed: int, particle: int,
                    event: int) -> int:
    k = key_of(seed)
    return int(lib().orc_param_entry_rng(oprm.ptr, ptype, E, eta, _p(k), particle, event))


def thresholds(w: np.ndarray):
    w = np.ascontiguousarray(w, dtype=np.float32).ravel()
    T = np.empty(len(w), dtype=np.uint32)
    K = np.zeros(1, dtype=np.int32)
    rc = lib().orc_thresholds(_p(w), len(w), _p(T), _p(K))
    if rc != 0:
        return None, -1
    return T, int(K[0])


def sample_bin(T: np.ndarray, k_last: int, x0: int) -> int:
    T = np.ascontiguousarray(T, dtype=np.uint32)
    return int(lib().orc_sample_bin(_p(T), k_last, x0 & 0xFFFFFFFF))


def scales(ogeo: OracleGeometry, layer: int, eta_c: float):
    se = C.c_double()
    sp = C.c_double()
    lib().orc_scales(ogeo.ptr, layer, eta_c, C.byref(se), C.byref(sp))
    return se.value, sp.value


def cells(ogeo: OracleGeometry, layer, eta, phi) -> np.ndarray:
    eta = np.ascontiguousarray(eta, dtype=np.float64).ravel()
    n = len(eta)
    phi = np.ascontiguousarray(np.broadcast_to(phi, n), dtype=np.float64)
    lay = np.ascontiguousarray(np.broadcast_to(layer, n), dtype=np.int32)
    out = np.empty(n, dtype=np.int32)
    lib().orc_cell_n(ogeo.ptr, n, _p(lay), _p(eta), _p(phi), _p(out))
    return out


# ----------------------------------------------------------------------------
# Whole-batch simulation
# ----------------------------------------------------------------------------
class SimResult:
    pass


def simulate(ogeo: OracleGeometry, oprm: OracleParams, parts, seed: int, first_event: int = 0,
             cells64: bool = True, canon: bool = True, tasks: bool = True, hit_cap: int = 0,
             hit_positions: bool = False, task_cap: int | None = None) -> SimResult:
    """Run the oracle over a particle batch (a ``synth.Particles``)."""
    t = np.ascontiguousarray(parts.type, dtype=np.int32)
    E = np.ascontiguousarray(parts.E, dtype=np.float32)
    eta = np.ascontiguousarray(parts.eta, dtype=np.float32)
    phi = np.ascontiguousarray(parts.phi, dtype=np.float32)
    off = np.ascontiguousarray(parts.event_offsets, dtype=np.int64)
    ne = len(off) - 1
    nc = ogeo.n_cells
    res = SimResult()
    keep = []

    def arr(shape, dtype, on):
        if not on:
            return None, None
        a = np.zeros(shape, dtype=dtype)
        keep.append(a)
        return a, a.ctypes.data

    res.cells64, p_c64 = arr((ne, nc), np.float64, cells64)
    res.cells_canon, p_cc = arr((ne, nc), np.float32, canon)
    tcap = (len(E) * ogeo.n_layers if task_cap is None else task_cap) if tasks else 0
    res.task_event, p_te = arr(tcap, np.int32, tasks)
    res.task_particle, p_tp = arr(tcap, np.int32, tasks)
    res.task_layer, p_tl = arr(tcap, np.int32, tasks)
    res.task_n, p_tn = arr(tcap, np.int32, tasks)
    res.task_Ehit, p_th = arr(tcap, np.float32, tasks)
    hc = hit_cap
    res.hit_cell, p_hc = arr(hc, np.int32, hc > 0)
    res.hit_bin, p_hb = arr(hc, np.int16, hc > 0)
    res.hit_eta, p_he = arr(hc, np.float64, hc > 0 and hit_positions)
    res.hit_phi, p_hp = arr(hc, np.float64, hc > 0 and hit_positions)
    res.hit_r, p_hr = arr(hc, np.float64, hc > 0 and hit_positions)
    res.hit_alpha, p_ha = arr(hc, np.float64, hc > 0 and hit_positions)
    out = _Outputs(p_c64, p_cc, tcap, p_te, p_tp, p_tl, p_tn, p_th, hc, p_hc, p_hb, p_he, p_hp,
                   p_hr, p_ha, 0, 0, 0.0)
    rc = lib().orc_simulate(ogeo.ptr, oprm.ptr, len(E), _p(t), _p(E), _p(eta), _p(phi), ne, _p(off),
                            seed & 0xFFFFFFFFFFFFFFFF, first_event, C.byref(out))
    res.status = int(rc)
    res.n_tasks = int(out.n_tasks)
    res.n_hits = int(out.n_hits)
    res.E_layers = float(out.E_layers)
    if tasks:
        k = min(res.n_tasks, tcap)
        for name in ("task_event", "task_particle", "task_layer", "task_n", "task_Ehit"):
            setattr(res, name, getattr(res, name)[:k])
    if hc > 0:
        k = min(res.n_hits, hc)
        for name in ("hit_cell", "hit_bin", "hit_eta", "hit_phi", "hit_r", "hit_alpha"):
            a = getattr(res, name)
            if a is not None:
                setattr(res, name, a[:k])
    return res


# ----------------------------------------------------------------------------
# Gradients by reweighting
# ----------------------------------------------------------------------------
def _parts(parts):
    return (np.ascontiguousarray(parts.type, dtype=np.int32), np.ascontiguousarray(parts.E, dtype=np.float32),
            np.ascontiguousarray(parts.eta, dtype=np.float32), np.ascontiguousarray(parts.phi, dtype=np.float32),
            np.ascontiguousarray(parts.event_offsets, dtype=np.int64))


def reweighted_cells(ogeo: OracleGeometry, oprm: OracleParams, parts, seed: int, first_event: int = 0,
                     f_entry: int = -1, f_delta: float = 0.0, w_entry: int = -1, w_bin: int = 0,
                     w_delta: float = 0.0) -> np.ndarray:
    """FP64 cells of the base hits with one layer fraction and/or one shape
    weight moved (hit counts, bins and cells held fixed)."""
    t, E, eta, phi, off = _parts(parts)
    ne = len(off) - 1
    cells = np.zeros((ne, ogeo.n_cells), dtype=np.float64)
    rc = lib().orc_reweighted_cells(ogeo.ptr, oprm.ptr, len(E), _p(t), _p(E), _p(eta), _p(phi), ne, _p(off),
                                    seed & 0xFFFFFFFFFFFFFFFF, first_event, f_entry, f_delta, w_entry, w_bin,
                                    w_delta, _p(cells))
    assert rc == 0, rc
    return cells


def backward(ogeo: OracleGeometry, oprm: OracleParams, parts, seed: int, dL_dcells: np.ndarray,
             first_event: int = 0):
    """(dL/dfrac [entries], dL/dshape_w [entries][128]) in FP64."""
    t, E, eta, phi, off = _parts(parts)
    ne = len(off) - 1
    g = np.ascontiguousarray(dL_dcells, dtype=np.float64).reshape(ne, ogeo.n_cells)
    n_entries = oprm.frac.size
    d_frac = np.zeros(n_entries, dtype=np.float64)
    d_w = np.zeros((n_entries, oprm.w.shape[-2] * oprm.w.shape[-1]), dtype=np.float64)
    rc = lib().orc_backward(ogeo.ptr, oprm.ptr, len(E), _p(t), _p(E), _p(eta), _p(phi), ne, _p(off),
                            seed & 0xFFFFFFFFFFFFFFFF, first_event, _p(g), _p(d_frac), _p(d_w))
    assert rc == 0, rc
    return d_frac, d_w
