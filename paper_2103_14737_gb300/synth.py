"""Seeded synthetic inputs for the parameterised calorimeter hit path.

This module produces INPUT DATA only: a calorimeter geometry table, a
parametrisation table and particle lists.  It holds none of the simulation's
arithmetic (no random-stream, Poisson, inverse-CDF, (r, alpha)->(eta, phi),
cell lookup or accumulation step); both the CUDA library and the CPU oracle
receive the arrays built here and each applies the method on its own.

The paper's inputs (ATLAS particle tuples, parametrisation files and the
detector description, Sec. 2 and Sec. 4) are not available, so these tables
stand in for them at the paper's scales:

* geometry: 24 layers, 78 regions, 188,160 cells (the paper's description
  has 24 layers, 78 regions and 187,652 cells, Sec. 4);
* parametrisation: 3 particle types x 17 energy bins x 100 |eta| bins x 24
  layers, each entry with a layer energy fraction, a mean hit energy and a
  16 (r) x 8 (alpha) shape histogram (the paper loads such flattened tables
  to the GPU, Sec. 4);
* particles: single 65.536 GeV electrons at eta = 0.22 (the paper's
  benchmark sample, Sec. 4 and Table 1), a 400-particle ttbar-like event and
  pile-up events with a Poisson(200) number of minimum-bias collisions
  (Sec. 1 on HL-LHC pile-up).

Every generator is a pure function of its seed (numpy PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# ---------------------------------------------------------------------------
# Geometry table
# ---------------------------------------------------------------------------
# (name, barrel, radius (barrel) or |z| (end-cap) in mm,
#  per-side regions as (|eta| lo, |eta| hi, d_eta, n_phi))
# Granularities follow the ATLAS calorimeter layer structure at the level the
# paper describes (Sec. 4: 24 layers, 78 regions); radii and |z| are
# synthetic.
LAYER_TABLE = (
    ("PreSamplerB", True, 1450.0, ((0.0, 0.8, 0.025, 64), (0.8, 1.525, 0.025, 64))),
    ("EMB1", True, 1550.0, ((0.0, 1.4, 0.003125, 64), (1.4, 1.475, 0.025, 256))),
    ("EMB2", True, 1700.0, ((0.0, 1.4, 0.025, 256), (1.4, 1.475, 0.075, 256))),
    ("EMB3", True, 1900.0, ((0.0, 0.8, 0.05, 256), (0.8, 1.35, 0.05, 256))),
    ("PreSamplerE", False, 3650.0, ((1.5, 1.65, 0.025, 64), (1.65, 1.8, 0.025, 64))),
    ("EME1", False, 3750.0, ((1.375, 1.5, 0.025, 64), (1.5, 2.5, 0.00625, 64))),
    ("EME2", False, 3900.0, ((1.375, 2.5, 0.025, 256), (2.5, 3.2, 0.1, 64))),
    ("EME3", False, 4100.0, ((1.5, 2.0, 0.05, 256), (2.0, 2.5, 0.05, 256))),
    ("HEC0", False, 4350.0, ((1.5, 2.5, 0.1, 64), (2.5, 3.3, 0.1, 64))),
    ("HEC1", False, 4700.0, ((1.5, 2.5, 0.1, 64), (2.5, 3.1, 0.1, 64))),
    ("HEC2", False, 5200.0, ((1.6, 2.5, 0.1, 64), (2.5, 3.1, 0.1, 64))),
    ("HEC3", False, 5700.0, ((1.7, 2.5, 0.1, 64), (2.5, 3.3, 0.1, 64))),
    ("TileBar0", True, 2450.0, ((0.0, 0.5, 0.1, 64), (0.5, 1.0, 0.1, 64))),
    ("TileBar1", True, 2900.0, ((0.0, 1.0, 0.1, 64),)),
    ("TileBar2", True, 3500.0, ((0.0, 0.8, 0.1, 64),)),
    ("TileGap1", True, 3450.0, ((0.9, 1.0, 0.1, 64),)),
    ("TileGap2", True, 3550.0, ((1.0, 1.1, 0.1, 64),)),
    ("TileGap3", True, 3650.0, ((1.1, 1.6, 0.1, 64),)),
    ("TileExt0", True, 2450.0, ((1.1, 1.6, 0.1, 64),)),
    ("TileExt1", True, 2900.0, ((0.8, 1.7, 0.1, 64),)),
    ("TileExt2", True, 3500.0, ((0.9, 1.3, 0.1, 64),)),
    ("FCAL0", False, 4750.0, ((3.1, 4.0, 0.1, 64), (4.0, 4.9, 0.1, 64))),
    ("FCAL1", False, 5200.0, ((3.2, 4.0, 0.1, 64), (4.0, 4.9, 0.1, 64))),
    ("FCAL2", False, 5650.0, ((3.3, 4.9, 0.1, 64),)),
)

# numpy layout of one region record; identical field order and sizes to
# ``fcs_region`` in include/fcs.h (48 bytes, no padding).
REGION_DTYPE = np.dtype(
    [
        ("eta_lo", "<f8"),
        ("deta", "<f8"),
        ("phi_lo", "<f8"),
        ("dphi", "<f8"),
        ("n_eta", "<i4"),
        ("n_phi", "<i4"),
        ("cell_offset", "<i4"),
        ("layer", "<i4"),
    ]
)
# ``fcs_layer_geom``: radius (barrel) or |z| (end-cap) in mm, barrel flag.
LAYER_DTYPE = np.dtype([("rz", "<f8"), ("barrel", "<i4"), ("pad", "<i4")])


@dataclass
class Geometry:
    regions: np.ndarray  # REGION_DTYPE[n_regions], sorted by (layer, eta_lo)
    layer_region_begin: np.ndarray  # int32[n_layers + 1]
    layers: np.ndarray  # LAYER_DTYPE[n_layers]
    n_cells: int
    names: tuple

    @property
    def n_layers(self) -> int:
        return len(self.layers)

    @property
    def n_regions(self) -> int:
        return len(self.regions)


def geometry() -> Geometry:
    """The 24-layer, 78-region synthetic calorimeter (188,160 cells).

    Each per-side region (|eta| lo, |eta| hi) is mirrored to eta < 0; within a
    layer the regions are listed in ascending eta_lo.  phi runs from -pi with
    n_phi equal bins.  Cells are numbered layer-major, then region (ascending
    eta_lo), then i_eta, then i_phi.
    """
    recs = []
    lrb = [0]
    lay = np.zeros(len(LAYER_TABLE), dtype=LAYER_DTYPE)
    cell = 0
    for li, (name, barrel, rz, side) in enumerate(LAYER_TABLE):
        lay[li]["rz"] = rz
        lay[li]["barrel"] = 1 if barrel else 0
        regs = []
        for lo, hi, de, nphi in side:
            neta = int(round((hi - lo) / de))
            assert abs(neta * de - (hi - lo)) < 1e-9, (name, lo, hi, de)
            regs.append((-hi, de, neta, nphi))  # mirrored, eta < 0
            regs.append((lo, de, neta, nphi))  # eta >= 0
        regs.sort(key=lambda r: r[0])
        for eta_lo, de, neta, nphi in regs:
            recs.append((eta_lo, de, -math.pi, 2.0 * math.pi / nphi, neta, nphi, cell, li))
            cell += neta * nphi
        lrb.append(len(recs))
    regions = np.array(recs, dtype=REGION_DTYPE)
    return Geometry(
        regions=regions,
        layer_region_begin=np.array(lrb, dtype=np.int32),
        layers=lay,
        n_cells=cell,
        names=tuple(t[0] for t in LAYER_TABLE),
    )


def layer_covers(geo: Geometry, layer: int, abs_eta: float) -> bool:
    """True if a per-side region of ``layer`` spans |eta| = abs_eta."""
    for lo, hi, _de, _nphi in LAYER_TABLE[layer][3]:
        if lo <= abs_eta < hi:
            return True
    return False


# ---------------------------------------------------------------------------
# Parametrisation table
# ---------------------------------------------------------------------------
N_TYPES = 3  # 0 electron, 1 photon, 2 charged pion
N_EBINS = 17  # energy bins [2^(6+i), 2^(7+i)) MeV, i = 0..16
N_ETABINS = 100  # |eta| bins of width 0.05 on [0, 5)
N_RBINS = 16
N_ABINS = 8
PARAM_SEED = 20210326


@dataclass
class Params:
    frac: np.ndarray  # f32[NT][NE][NH][NL], per-entry layer energy fraction
    mean_hit_E: np.ndarray  # f32[NT][NE][NH][NL], MeV
    shape_w: np.ndarray  # f32[NT][NE][NH][NL][16][8], unnormalised weights
    r_edges: np.ndarray  # f32[17], mm
    a_edges: np.ndarray  # f32[9], rad
    eta_bin_scale: float = 20.0  # eta bins per unit |eta|
    ebin_log2_min: int = 6  # energy bin 0 starts at 2^6 MeV

    @property
    def dims(self):
        return self.frac.shape


def r_edges() -> np.ndarray:
    """Radial bin edges: 0, then 16 edges log-spaced from 1 mm to 500 mm."""
    e = np.empty(N_RBINS + 1, dtype=np.float64)
    e[0] = 0.0
    e[1:] = np.exp(np.linspace(0.0, math.log(500.0), N_RBINS))
    return e.astype(np.float32)


def a_edges() -> np.ndarray:
    """Angular bin edges: 8 equal bins on [0, 2 pi)."""
    return (np.arange(N_ABINS + 1, dtype=np.float64) * (2.0 * math.pi / N_ABINS)).astype(np.float32)


def params(geo: Geometry, seed: int = PARAM_SEED, mean_hit_range=(5.0, 200.0),
           n_types: int = N_TYPES, n_ebins: int = N_EBINS, n_etabins: int = N_ETABINS) -> Params:
    """Seeded parametrisation table.

    * layer fractions: Dirichlet(alpha = 2) over the layers whose regions
      span the |eta| bin centre, zero for the other layers (an |eta| bin with
      no covering layer deposits nothing);
    * mean hit energy: log-uniform on ``mean_hit_range`` MeV;
    * shape weights: w[ir][ia] = exp(-r_mid(ir) / lambda) * (1 + 0.2 xi) with
      lambda ~ U(10, 100) mm per entry and xi ~ U(-1, 1) per bin.
    """
    rng = np.random.default_rng(seed)
    nl = geo.n_layers
    frac = np.zeros((n_types, n_ebins, n_etabins, nl), dtype=np.float64)
    for h in range(n_etabins):
        centre = (h + 0.5) / 20.0
        cov = [l for l in range(nl) if layer_covers(geo, l, centre)]
        if not cov:
            continue
        d = rng.dirichlet(np.full(len(cov), 2.0), size=(n_types, n_ebins))
        frac[:, :, h, cov] = d
    lo, hi = mean_hit_range
    mhe = np.exp(rng.uniform(math.log(lo), math.log(hi), size=(n_types, n_ebins, n_etabins, nl)))
    re = r_edges().astype(np.float64)
    r_mid = 0.5 * (re[:-1] + re[1:])
    lam = rng.uniform(10.0, 100.0, size=(n_types, n_ebins, n_etabins, nl))
    xi = rng.uniform(-1.0, 1.0, size=(n_types, n_ebins, n_etabins, nl, N_RBINS, N_ABINS))
    w = np.exp(-r_mid[None, None, None, None, :, None] / lam[..., None, None]) * (1.0 + 0.2 * xi)
    return Params(
        frac=frac.astype(np.float32),
        mean_hit_E=mhe.astype(np.float32),
        shape_w=w.astype(np.float32),
        r_edges=r_edges(),
        a_edges=a_edges(),
    )


# ---------------------------------------------------------------------------
# Particles
# ---------------------------------------------------------------------------
@dataclass
class Particles:
    """Particles grouped by event: event e owns [event_offsets[e], event_offsets[e+1])."""

    type: np.ndarray  # int32[n]
    E: np.ndarray  # f32[n], MeV
    eta: np.ndarray  # f32[n]
    phi: np.ndarray  # f32[n]
    event_offsets: np.ndarray  # int64[n_events + 1]

    @property
    def n(self) -> int:
        return len(self.E)

    @property
    def n_events(self) -> int:
        return len(self.event_offsets) - 1

    def event(self, e: int) -> "Particles":
        a, b = int(self.event_offsets[e]), int(self.event_offsets[e + 1])
        return Particles(self.type[a:b].copy(), self.E[a:b].copy(), self.eta[a:b].copy(),
                         self.phi[a:b].copy(), np.array([0, b - a], dtype=np.int64))

    def events(self, e0: int, e1: int) -> "Particles":
        a, b = int(self.event_offsets[e0]), int(self.event_offsets[e1])
        off = self.event_offsets[e0:e1 + 1] - a
        return Particles(self.type[a:b].copy(), self.E[a:b].copy(), self.eta[a:b].copy(),
                         self.phi[a:b].copy(), off.astype(np.int64))


def _concat(parts) -> Particles:
    t = np.concatenate([p[0] for p in parts]).astype(np.int32)
    E = np.concatenate([p[1] for p in parts]).astype(np.float32)
    eta = np.concatenate([p[2] for p in parts]).astype(np.float32)
    phi = np.concatenate([p[3] for p in parts]).astype(np.float32)
    off = np.zeros(len(parts) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(p[1]) for p in parts])
    return Particles(t, E, eta, phi, off)


def single_particle(n_events: int, ptype: int = 0, E: float = 65536.0, eta: float = 0.22,
                    phi: float = 0.0) -> Particles:
    """One particle per event (the paper's 65.536 GeV electron sample)."""
    parts = [(np.array([ptype]), np.array([E]), np.array([eta]), np.array([phi]))] * n_events
    return _concat(parts)


def _hard_scatter(rng, n=400):
    # half photons/electrons, half charged pions; |eta| < 2.5; E ~ Exp(10 GeV)
    # clipped to [1 GeV, 1 TeV]
    t = np.empty(n, dtype=np.int32)
    h = n // 2
    t[:h] = rng.integers(0, 2, size=h)
    t[h:] = 2
    t = rng.permutation(t)
    E = np.clip(rng.exponential(10000.0, size=n), 1000.0, 1.0e6)
    eta = rng.uniform(-2.5, 2.5, size=n)
    phi = rng.uniform(-math.pi, math.pi, size=n)
    return t, E, eta, phi


def replicate(parts: Particles, n: int) -> Particles:
    """The events of ``parts`` repeated n times; each copy draws its own random
    numbers through its event number (n simulation seeds of the same event)."""
    return _concat([(parts.type, parts.E, parts.eta, parts.phi)] * n) if parts.n_events == 1 else \
        _concat([(parts.type[a:b], parts.E[a:b], parts.eta[a:b], parts.phi[a:b])
                 for _ in range(n) for a, b in zip(parts.event_offsets[:-1], parts.event_offsets[1:])])


def ttbar_like(seed: int = 1, n_events: int = 1, n: int = 400) -> Particles:
    """400-particle ttbar-like events without pile-up."""
    rng = np.random.default_rng(seed)
    return _concat([_hard_scatter(rng, n) for _ in range(n_events)])


def pileup(seed: int = 1, n_events: int = 64, mu_pu: float = 200.0, per_collision: float = 60.0,
           hs_particles: int = 400) -> Particles:
    """Hard scatter plus Poisson(mu_pu) minimum-bias collisions per event.

    Each collision has Poisson(per_collision) particles with E ~ Exp(1.5 GeV)
    clipped to [1 GeV, 1 TeV], |eta| < 3.2, 30 % photons, 10 % electrons and
    60 % charged pions.  Events therefore have uneven multiplicities around
    12,000 particles.
    """
    rng = np.random.default_rng(seed)
    parts = []
    for _ in range(n_events):
        t, E, eta, phi = _hard_scatter(rng, hs_particles)
        n_coll = rng.poisson(mu_pu)
        m = int(rng.poisson(per_collision, size=n_coll).sum())
        tp = rng.choice(np.array([1, 0, 2], dtype=np.int32), size=m, p=[0.3, 0.1, 0.6])
        Ep = np.clip(rng.exponential(1500.0, size=m), 1000.0, 1.0e6)
        etap = rng.uniform(-3.2, 3.2, size=m)
        phip = rng.uniform(-math.pi, math.pi, size=m)
        parts.append((np.concatenate([t, tp]), np.concatenate([E, Ep]),
                      np.concatenate([eta, etap]), np.concatenate([phi, phip])))
    return _concat(parts)


def bucket_by_multiplicity(p: Particles) -> np.ndarray:
    """Event order sorted by particle count (for multiplicity-bucketed batches)."""
    return np.argsort(np.diff(p.event_offsets), kind="stable")


# Named workloads (sizes as stated in the build's configuration list).
WORKLOADS = {
    "single_e65": dict(kind="single", n_events=16),
    "ttbar400": dict(kind="ttbar", n_events=1),
    "pileup64": dict(kind="pileup", n_events=64),
    "pileup1024": dict(kind="pileup", n_events=1024),
}


def workload(name: str, seed: int = 1, n_events: int | None = None) -> Particles:
    w = WORKLOADS[name]
    ne = n_events if n_events is not None else w["n_events"]
    if w["kind"] == "single":
        return single_particle(ne)
    if w["kind"] == "ttbar":
        return ttbar_like(seed, ne)
    return pileup(seed, ne)
