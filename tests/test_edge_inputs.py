"""The edge inputs of the GPU parity tests (tests/parity.py: EDGE_CASES) on
the CPU: they reach the corners of the method, and the oracle treats those
corners as the method's definition says.

* geometry: no mirror symmetry, gaps, adjacent and overlapping region
  boundaries, 1 to 4 regions per layer, and a case at the ABI's limits
  (32 layers, 256 regions, more than 2^19 cells);
* histograms: every kind of edge_params is present; zero-weight bins and bins
  after the last non-zero one are never drawn; a single-bin histogram always
  gives its bin; steep histograms draw their light tail bins too;
* hit counts: a mean hit energy of 3e38 MeV gives a Poisson mean below 1e-30,
  a draw of 0 and so exactly one hit (n = max(1, Poisson(mu)));
* parametrisation lookup: exact rational |eta| bins and frexp energy bins for
  particles on the bin edges (non-integer and integer scales);
* cells: every sampled hit's cell is one that a brute-force scan of the
  layer's cell boxes (nearest region by eta distance, phi index taken
  modulo n_phi) allows.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_14737_gb300 import synth
from parity import EDGE_CASES, edge_case

SEED, FIRST_EVENT = 5, 2


@pytest.fixture(scope="module", params=list(EDGE_CASES))
def case(request):
    geo, prm, parts = edge_case(request.param)
    og, op = O.OracleGeometry(geo), O.OracleParams(prm)
    ref = O.simulate(og, op, parts, seed=SEED, first_event=FIRST_EVENT, hit_cap=10**7, hit_positions=True)
    assert ref.status == 0 and ref.n_hits <= 10**7
    return dict(name=request.param, geo=geo, prm=prm, parts=parts, og=og, op=op, ref=ref)


def _entries(case):
    """Parametrisation entry (with layer) of every task and of every hit."""
    ref, parts, op = case["ref"], case["parts"], case["op"]
    NL = case["geo"].n_layers
    gp = parts.event_offsets[ref.task_event] + ref.task_particle
    base = np.array([O.param_entry(op, int(parts.type[i]), float(parts.E[i]), float(parts.eta[i])) for i in gp])
    task_entry = base * NL + ref.task_layer
    return task_entry, np.repeat(task_entry, ref.task_n)


def test_geometry_edges(case):
    geo = case["geo"]
    reg = geo.regions
    lrb = geo.layer_region_begin
    counts = np.diff(lrb)
    if case["name"] == "limits":
        assert geo.n_layers == 32 and geo.n_regions == 256 and geo.n_cells >= 1 << 19
    else:
        assert counts.min() == 1 and counts.max() >= 3
    gaps = []
    for l in range(geo.n_layers):
        for r in range(lrb[l] + 1, lrb[l + 1]):
            top = reg["eta_lo"][r - 1] + reg["n_eta"][r - 1] * reg["deta"][r - 1]
            gaps.append(reg["eta_lo"][r] - top)
    gaps = np.array(gaps)
    assert (gaps > 1e-3).any() and (np.abs(gaps) < 1e-9).any()
    if case["name"] != "limits":
        assert (gaps < 0).any()  # an overlap below the loaders' 1e-9 tolerance
    # not mirrored: some region has no partner at -eta
    lo, hi = reg["eta_lo"], reg["eta_lo"] + reg["n_eta"] * reg["deta"]
    mirrored = [np.any(np.isclose(-hi[r], lo[lrb[reg["layer"][r]]:lrb[reg["layer"][r] + 1]])) for r in range(len(reg))]
    assert not all(mirrored)


def test_histogram_kinds_present(case):
    w = case["prm"].shape_w.reshape(-1, 128).astype(np.float64)
    live = case["prm"].frac.reshape(-1) > 0
    w = w[live]
    nz = w > 0
    K = np.array([np.nonzero(r)[0].max() for r in nz])
    n_nz = nz.sum(1)
    assert (n_nz == 1).sum() > 10  # single bins (and first-only / last-only)
    assert (K == 0).any() and (K == 127).any()
    assert len(np.unique(K)) >= 40  # trailing zeros: many different last bins
    interior = np.array([not nz[i, :K[i]].all() for i in range(len(K))])
    assert interior.sum() > 10
    share = w.max(1) / w.sum(1)
    assert ((share > 0.98) & (n_nz == 128)).sum() > 10  # steep
    assert (w.sum(1) < 1e-25).any() and (w.max(1) > 1e9).any()  # tiny scale, 24 decades


def test_forced_single_hits(case):
    ref, prm = case["ref"], case["prm"]
    task_entry, _ = _entries(case)
    huge = prm.mean_hit_E.reshape(-1)[task_entry] >= 1e38
    assert huge.sum() > 20
    assert (ref.task_n[huge] == 1).all()
    # the same closed form through the Poisson function itself
    assert O.poisson(np.full(8, 1e-30), SEED, np.arange(8), 3, 4).tolist() == [0] * 8


def test_hits_respect_histograms(case):
    ref, prm = case["ref"], case["prm"]
    _, hit_entry = _entries(case)
    w = prm.shape_w.reshape(-1, 128)
    wb = w[hit_entry, ref.hit_bin]
    assert (wb > 0).all(), "a zero-weight bin was drawn"
    nz = w[hit_entry] > 0
    last = 127 - np.argmax(nz[:, ::-1], axis=1)
    assert (ref.hit_bin <= last).all()
    single = nz.sum(1) == 1
    assert single.sum() > 0 and (ref.hit_bin[single] == last[single]).all()
    steep = (w[hit_entry].max(1) / w[hit_entry].astype(np.float64).sum(1) > 0.98) & (nz.sum(1) == 128)
    dom = np.argmax(w[hit_entry], axis=1)
    assert (steep & (ref.hit_bin != dom)).sum() > 0, "no hit in a steep histogram's light bins"


def _exact_entry(prm, t, E, eta):
    NT, NE, NH, NL = prm.frac.shape
    _, ex = math.frexp(float(np.float32(E)))
    eb = min(max((ex - 1) - prm.ebin_log2_min, 0), NE - 1)
    hb = min(math.floor(Fraction(float(abs(np.float32(eta)))) * Fraction(prm.eta_bin_scale)), NH - 1)
    return (t * NE + eb) * NH + hb


def test_parametrisation_lookup_exact(case):
    parts, prm, op = case["parts"], case["prm"], case["op"]
    s = Fraction(prm.eta_bin_scale)
    on_edge = sum(1 for v in parts.eta if (Fraction(float(abs(v))) * s).denominator == 1 and v != 0)
    assert on_edge >= 4
    for i in range(parts.n):
        t, E, eta = int(parts.type[i]), float(parts.E[i]), float(parts.eta[i])
        assert O.param_entry(op, t, E, eta) == _exact_entry(prm, t, E, eta), (t, E, eta)


def _region_candidates(geo, layer, eta, tol=1e-9):
    rb, re = geo.layer_region_begin[layer], geo.layer_region_begin[layer + 1]
    reg = geo.regions[rb:re]
    lo, hi = reg["eta_lo"], reg["eta_lo"] + reg["n_eta"] * reg["deta"]
    d = np.maximum(np.maximum(lo - eta, eta - hi), 0.0)
    return [rb + j for j in np.nonzero(d <= d.min() + tol)[0]]


def _cell_candidates(geo, layer, eta, phi, tol=1e-9):
    out = set()
    for r in _region_candidates(geo, layer, eta):
        elo, de, plo, dp = (float(geo.regions[k][r]) for k in ("eta_lo", "deta", "phi_lo", "dphi"))
        ne, nphi, off = (int(geo.regions[k][r]) for k in ("n_eta", "n_phi", "cell_offset"))
        te = (min(max(eta, elo), elo + ne * de) - elo) / de
        ies = {min(max(int(math.floor(te + d)), 0), ne - 1) for d in (-tol, 0.0, tol)}
        tp = (phi - plo) / dp
        if abs(tp) > 2.0**52:
            tp = math.copysign(2.0**52, tp)
        ips = {int(math.floor(tp + d)) % nphi for d in (-tol * max(1.0, abs(tp)), 0.0, tol * max(1.0, abs(tp)))}
        out.update(off + ie * nphi + ip for ie in ies for ip in ips)
    return out


def test_hit_cells_bruteforce(case):
    ref, geo = case["ref"], case["geo"]
    lay = np.repeat(ref.task_layer, ref.task_n)
    rng = np.random.default_rng(3)
    idx = rng.choice(ref.n_hits, size=min(4000, ref.n_hits), replace=False)
    for i in idx:
        c = _cell_candidates(geo, int(lay[i]), float(ref.hit_eta[i]), float(ref.hit_phi[i]))
        assert int(ref.hit_cell[i]) in c, (i, lay[i], ref.hit_eta[i], ref.hit_phi[i], ref.hit_cell[i], c)


def test_conservation(case):
    ref = case["ref"]
    assert math.isclose(ref.cells64.sum(), float((ref.task_n.astype(np.float64) * ref.task_Ehit).sum()),
                        rel_tol=1e-12)
