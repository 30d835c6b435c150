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


# ---------------------------------------------------------------------------
# Edge inputs: seeded geometries, parametrisations and particles that reach
# the corners of the method (the same loaders and the same rules as above;
# still input data only)
# ---------------------------------------------------------------------------
def random_geometry(seed: int, n_layers: int = 8, regions_per_layer=(1, 4), n_regions_total: int | None = None,
                    n_eta_range=(1, 40), n_phi_choices=(1, 2, 7, 32, 64, 100, 256)) -> Geometry:
    """A seeded geometry without the mirror symmetry of ``geometry()``.

    Per layer: barrel or end-cap at a random radius / |z|, 1 to 4 regions (or
    ``n_regions_total`` regions spread over the layers, up to 256) laid out
    from a random eta start in ascending eta_lo with unequal gaps between
    them: none (adjacent), 1e-4, a wide gap, or an overlap of 5e-10 (the
    loaders accept overlaps below 1e-9).  Granularities from a set that
    includes a non-dyadic 0.0371; phi grids start at -pi, 0 or a random angle,
    mostly with n_phi d_phi = 2 pi and sometimes covering less of the circle
    (the grid index wraps modulo n_phi either way).
    """
    rng = np.random.default_rng(seed)
    if n_regions_total is None:
        counts = rng.integers(regions_per_layer[0], regions_per_layer[1] + 1, size=n_layers)
    else:
        assert n_layers <= n_regions_total
        counts = np.ones(n_layers, dtype=np.int64)
        extra = rng.multinomial(n_regions_total - n_layers, rng.dirichlet(np.full(n_layers, 0.7)))
        counts += extra
    detas = (0.003125, 0.00625, 0.0125, 0.025, 0.05, 0.1, 0.0371, 0.2)
    recs, lrb = [], [0]
    n_gap = 0  # gap kinds cycle, so that every kind occurs
    lay = np.zeros(n_layers, dtype=LAYER_DTYPE)
    cell = 0
    for li in range(n_layers):
        barrel = bool(rng.random() < 0.5)
        lay[li]["rz"] = rng.uniform(1200.0, 6000.0)
        lay[li]["barrel"] = 1 if barrel else 0
        eta = rng.uniform(-2.2, 0.3) if barrel else rng.uniform(-4.6, 1.5)
        if counts[li] > 8:  # many regions: narrow ones, so that the layer stays within |eta| < 6
            eta = rng.uniform(-5.5, -3.0)
        for j in range(int(counts[li])):
            if j > 0:
                kind = n_gap % 4
                n_gap += 1
                eta += (0.0, 1e-4, rng.uniform(0.01, 0.5 if counts[li] <= 8 else 0.05), -5e-10)[kind]
            de = float(rng.choice(detas if counts[li] <= 8 else detas[:6]))
            ne = int(rng.integers(n_eta_range[0], n_eta_range[1] + 1))
            if counts[li] > 8:
                ne = max(1, min(ne, int(0.25 / de)))
            nphi = int(rng.choice(n_phi_choices))
            phi_lo = float(rng.choice([-math.pi, 0.0, rng.uniform(-math.pi, math.pi)]))
            dphi = 2.0 * math.pi / nphi
            if rng.random() < 0.15:
                dphi *= rng.uniform(0.5, 1.0)
            recs.append((eta, de, phi_lo, dphi, ne, nphi, cell, li))
            cell += ne * nphi
            eta = eta + ne * de
        lrb.append(len(recs))
    return Geometry(regions=np.array(recs, dtype=REGION_DTYPE), layer_region_begin=np.array(lrb, dtype=np.int32),
                    layers=lay, n_cells=cell, names=tuple(f"L{i}" for i in range(n_layers)))


# histogram kinds of edge_params
SHAPE_KINDS = ("falling", "interior_zeros", "trailing_zeros", "single_bin", "steep", "first_only", "last_only",
               "wide_range", "tiny_scale")


def edge_params(geo: Geometry, seed: int, n_types: int = 2, n_ebins: int = 7, n_etabins: int = 40,
                eta_bin_scale: float = 12.5, ebin_log2_min: int = 8, mean_hit_range=(1.0, 100.0),
                r_edge_kind: str = "random", a_edge_kind: str = "random", subnormal_frac: bool = True) -> Params:
    """A seeded parametrisation whose entries reach the edge cases of the method.

    * layer fractions: Dirichlet(1) over a random subset of the layers, a
      single layer, no layer at all, or (``subnormal_frac``) one subnormal
      fraction (a float layer energy that rounds to 0, no task, or to a
      subnormal value);
    * mean hit energy: log-uniform on ``mean_hit_range`` MeV, or 3e38 MeV for
      5 % of the entries (a Poisson mean near 0: every such task gets its one
      hit);
    * shape weights, one kind per entry (``SHAPE_KINDS``): falling with
      radius; the same with half the bins zero; the same with every bin after
      a random last bin K in [0, 126] zero; a single non-zero bin; one bin
      holding 99 % of the weight and the 127 others sharing 1 % (guide cells
      that span tens of bins); only bin 0; only bin 127; weights spread over
      24 decades; falling weights scaled by 1e-30;
    * radial edges: random increasing values from 0 or 0.5 mm; angular edges:
      random increasing values within [0, 2 pi] (or 8 equal bins).
    """
    rng = np.random.default_rng(seed)
    nl = geo.n_layers
    shape = (n_types, n_ebins, n_etabins, nl)
    frac = np.zeros(shape, dtype=np.float64)
    for t in range(n_types):
        for e in range(n_ebins):
            for h in range(n_etabins):
                kind = rng.integers(0, 10)
                if kind == 0:
                    continue  # no layer: the particle makes no task
                if kind == 1:
                    frac[t, e, h, rng.integers(0, nl)] = 1.0
                    continue
                k = int(rng.integers(1, nl + 1))
                lays = rng.choice(nl, size=k, replace=False)
                frac[t, e, h, lays] = rng.dirichlet(np.ones(k))
                if kind == 2 and subnormal_frac:
                    frac[t, e, h, lays[0]] = 1e-42  # subnormal in float32
    lo, hi = mean_hit_range
    mhe = np.exp(rng.uniform(math.log(lo), math.log(hi), size=shape))
    mhe[rng.random(size=shape) < 0.05] = 3.0e38
    if r_edge_kind == "random":
        r0 = float(rng.choice([0.0, 0.5]))
        re = np.concatenate([[r0], r0 + np.cumsum(rng.uniform(0.5, 60.0, size=N_RBINS))])
    else:
        re = r_edges().astype(np.float64)
    if a_edge_kind == "random":
        ae = np.sort(rng.uniform(0.0, 2.0 * math.pi, size=N_ABINS + 1))
        ae[0] = float(rng.choice([0.0, ae[0]]))
        ae[-1] = float(rng.choice([np.float32(2.0 * math.pi).astype(np.float64) - 1e-6, ae[-1]]))
    else:
        ae = a_edges().astype(np.float64)
    r_mid = 0.5 * (re[:-1] + re[1:])
    nb = N_RBINS * N_ABINS
    w = np.empty(shape + (nb,), dtype=np.float64)
    kinds = rng.integers(0, len(SHAPE_KINDS), size=shape)
    for idx in np.ndindex(*shape):
        lam = rng.uniform(10.0, 100.0)
        base = (np.exp(-r_mid[:, None] / lam) * (1.0 + 0.2 * rng.uniform(-1.0, 1.0, size=(N_RBINS, N_ABINS)))).ravel()
        name = SHAPE_KINDS[kinds[idx]]
        if name == "falling":
            v = base
        elif name == "interior_zeros":
            v = base * (rng.random(nb) < 0.5)
            if not v.any():
                v[rng.integers(0, nb)] = 1.0
        elif name == "trailing_zeros":
            K = int(rng.integers(0, nb - 1))
            v = base.copy()
            v[K + 1:] = 0.0
        elif name == "single_bin":
            v = np.zeros(nb)
            v[rng.integers(0, nb)] = rng.uniform(0.1, 10.0)
        elif name == "steep":
            v = rng.uniform(0.5, 1.5, size=nb)
            v *= 0.01 / v.sum()
            v[rng.integers(0, nb)] = 0.99
        elif name == "first_only":
            v = np.zeros(nb)
            v[0] = 1.0
        elif name == "last_only":
            v = np.zeros(nb)
            v[-1] = 2.0
        elif name == "wide_range":
            v = 10.0 ** rng.uniform(-12.0, 12.0, size=nb)
        else:  # tiny_scale
            v = base * 1e-30
        w[idx] = v
    return Params(frac=frac.astype(np.float32), mean_hit_E=mhe.astype(np.float32),
                  shape_w=w.reshape(shape + (N_RBINS, N_ABINS)).astype(np.float32),
                  r_edges=re.astype(np.float32), a_edges=ae.astype(np.float32),
                  eta_bin_scale=float(eta_bin_scale), ebin_log2_min=int(ebin_log2_min))


def _f32_neighbours(x: float) -> list:
    """x rounded to float32 and the float32 values one ulp below and above."""
    f = np.float32(x)
    return [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]


def edge_particles(seed: int, geo: Geometry, prm: Params, n_events: int = 4, n_random: int = 150,
                   extreme_eta=(7.5, -7.5, 6.0, -6.0)) -> Particles:
    """Particles at the edges of the parametrisation lookup and the geometry.

    Each event mixes: |eta| exactly on |eta|-bin edges k / scale and one float
    ulp either side, with both signs; energies exactly on the power-of-two
    energy-bin edges (below, inside and above the table's range) and one ulp
    either side; eta on region boundaries (eta_lo of each region and the
    midpoints between regions) and one ulp either side; phi at +-pi rounded
    to float, one ulp inside, and beyond the circle (7.5 and -40 rad); eta
    far outside every region (``extreme_eta``) and +-0; a subnormal and a
    tiny energy; plus ``n_random`` particles spread over the geometry.  Event
    1 (of 3 or more) is empty.  Types cycle over the table's types.
    """
    rng = np.random.default_rng(seed)
    NT, NE, NH = prm.frac.shape[:3]
    s = prm.eta_bin_scale
    etas = []
    for k in rng.choice(NH + 1, size=min(NH + 1, 12), replace=False):
        for v in _f32_neighbours(k / s):
            etas += [v, -v]
    reg = geo.regions
    for r in range(len(reg)):
        etas += _f32_neighbours(reg["eta_lo"][r])
        etas += _f32_neighbours(reg["eta_lo"][r] + reg["n_eta"][r] * reg["deta"][r])
    etas += [np.float32(v) for v in extreme_eta + (0.0, -0.0)]
    energies = []
    for j in range(-2, NE + 2):
        energies += _f32_neighbours(2.0 ** (prm.ebin_log2_min + j))
    energies += [np.float32(1e-40), np.float32(1e-3)]
    phis = _f32_neighbours(math.pi) + _f32_neighbours(-math.pi) + [np.float32(7.5), np.float32(-40.0), np.float32(0.0)]
    lo_eta = float(reg["eta_lo"].min()) - 0.3
    hi_eta = float((reg["eta_lo"] + reg["n_eta"] * reg["deta"]).max()) + 0.3
    parts = []
    for ev in range(n_events):
        if ev == 1 and n_events >= 3:
            z = np.zeros(0)
            parts.append((z.astype(np.int32), z, z, z))
            continue
        eta = np.array(etas + list(rng.uniform(lo_eta, hi_eta, size=n_random)), dtype=np.float32)
        n = len(eta)
        rng.shuffle(eta)
        E = np.array(energies, dtype=np.float32)[rng.integers(0, len(energies), size=n)]
        rand_E = rng.random(n) < 0.5
        E[rand_E] = (2.0 ** rng.uniform(prm.ebin_log2_min - 1, prm.ebin_log2_min + NE + 1, size=rand_E.sum()))
        phi = rng.uniform(-math.pi, math.pi, size=n).astype(np.float32)
        pick = rng.random(n) < 0.3
        phi[pick] = np.array(phis, dtype=np.float32)[rng.integers(0, len(phis), size=pick.sum())]
        t = (np.arange(n) % NT).astype(np.int32)
        parts.append((t, E.astype(np.float32), eta, phi))
    return _concat(parts)
