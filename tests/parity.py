"""Comparison helpers shared by the GPU parity tests (CUDA path through the C
ABI against the CPU oracle on the same seeded inputs).

Bars (Sec. 6 of the paper validates CPU and GPU hit by hit on the same random
numbers and asks for identical cells):
  * task counts, hit counts and the hit -> cell and hit -> bin maps: bit-exact;
  * hit energies (float, Listing 1): bit-exact;
  * atomic mode cell energies: |dE| <= 1e-5 |E| + 1e-3 MeV against the FP64
    oracle (FP32 atomics in any order);
  * deterministic mode: bit-exact against the oracle's canonical FP32 fold;
  * gradients: within 1e-5 of the sum of the absolute values of their terms
    plus 1e-6 of their value (FP32 products summed over at most one warp
    before FP64 atomics).
"""
import numpy as np

from oracle import oracle as O

RTOL, ATOL = 1e-5, 1e-3
GRAD_TOL = 1e-5


def run_both(sim, ogeo, oprm, parts, seed, first_event=0, mode=0, batched=1, hpt=0, block=0, hits=True,
             energy_interp=0):
    import torch
    d = sim.to_device(parts)
    ref = O.simulate(ogeo, oprm, parts, seed=seed, first_event=first_event, hit_cap=(10**7 if hits else 0))
    got = sim.simulate(d, seed, first_event=first_event, mode=mode, batched=batched, hits_per_thread=hpt,
                       block=block, dense=True, debug_tasks=max(ref.n_tasks, 1),
                       debug_hits=(max(ref.n_hits, 1) if hits else 0), energy_interp=energy_interp)
    torch.cuda.synchronize()
    return ref, got


def check_tasks_hits(ref, got):
    st = got["stats"]
    assert st["n_tasks"] == ref.n_tasks
    assert st["n_hits"] == ref.n_hits
    for k in ("task_event", "task_particle", "task_layer", "task_n"):
        assert np.array_equal(got[k].cpu().numpy(), getattr(ref, k)), k
    assert np.array_equal(got["task_Ehit"].cpu().numpy().view(np.uint32), ref.task_Ehit.view(np.uint32))
    if "hit_cell" in got and ref.hit_cell is not None:
        hc = got["hit_cell"].cpu().numpy()
        mism = np.nonzero(hc != ref.hit_cell)[0]
        assert len(mism) == 0, f"{len(mism)} hit-cell mismatches, first {mism[:5]}"
        hb = got["hit_bin"].cpu().numpy()
        mism = np.nonzero(hb != ref.hit_bin)[0]
        assert len(mism) == 0, f"{len(mism)} hit-bin mismatches, first {mism[:5]}"


def check_compacted(got, dense, n_events):
    off = got["event_offsets"].cpu().numpy()
    ids = got["cell_ids"].cpu().numpy()
    E = got["cell_E"].cpu().numpy()
    assert off[0] == 0 and off[-1] == got["stats"]["n_nonzero"]
    for e in range(n_events):
        nz = np.nonzero(dense[e])[0]
        a, b = off[e], off[e + 1]
        assert np.array_equal(ids[a:b], nz)
        assert np.array_equal(E[a:b].astype(np.float64), dense[e][nz])


def check_cells_atomic(ref, got, n_events):
    cells = got["cells"].cpu().numpy().astype(np.float64)
    want = ref.cells64
    err = np.abs(cells - want)
    bad = err > RTOL * np.abs(want) + ATOL
    assert not bad.any(), f"{bad.sum()} cells out of tolerance, worst {err.max()}"
    assert np.array_equal(cells != 0, want != 0)
    check_compacted(got, cells, n_events)


def check_cells_det(ref, got, n_events):
    cells = got["cells"].cpu().numpy()
    assert np.array_equal(cells.view(np.uint32), ref.cells_canon.view(np.uint32))
    check_compacted(got, cells.astype(np.float64), n_events)


def grad_scales(ogeo, oprm, prm, parts, seed, g, first_event=0):
    """Per-component sums of absolute terms of the oracle's gradient."""
    fa, wa = O.backward(ogeo, oprm, parts, seed, np.abs(g), first_event=first_event)
    f = prm.frac.reshape(-1).astype(np.float64)
    w = prm.shape_w.reshape(-1, 128).astype(np.float64)
    S_abs = f * fa
    W = w.sum(axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        sw = np.where(W > 0, S_abs / W, 0.0)
    return fa, wa + 2 * sw[:, None]


def check_grad(got_f, got_w, ref_f, ref_w, sc_f, sc_w):
    gf = got_f.cpu().numpy().astype(np.float64)
    gw = got_w.cpu().numpy().astype(np.float64).reshape(ref_w.shape)
    ef = np.abs(gf - ref_f)
    bad = ef > GRAD_TOL * sc_f + 1e-6 * np.abs(ref_f) + 1e-30
    assert not bad.any(), f"{bad.sum()} d_frac out of tolerance, worst rel {(ef / (sc_f + 1e-300)).max()}"
    ew = np.abs(gw - ref_w)
    bad = ew > GRAD_TOL * sc_w + 1e-6 * np.abs(ref_w) + 1e-30
    assert not bad.any(), f"{bad.sum()} d_shape_w out of tolerance, worst rel {(ew / (sc_w + 1e-300)).max()}"
    # untouched entries stay exactly zero
    assert np.array_equal(gf == 0, ref_f == 0)


# ---------------------------------------------------------------------------
# Edge inputs (seeded): a geometry without mirror symmetry, with gaps, 1-4
# regions per layer, a non-integer |eta|-bin scale; a second one with 12
# layers and an integer scale; and one at the ABI's limits (32 layers, 256
# regions, more than 2^19 cells).  Parametrisations with zero-weight,
# trailing-zero, single-bin and steep histograms and mean hit energies that
# force one hit; particles on |eta|-bin, energy-bin and region edges.
# ---------------------------------------------------------------------------
EDGE_CASES = {
    "asym8": dict(geo=dict(seed=101), prm=dict(seed=11, eta_bin_scale=12.5, ebin_log2_min=8), parts=13),
    "asym12": dict(geo=dict(seed=102, n_layers=12),
                   prm=dict(seed=12, eta_bin_scale=7, ebin_log2_min=5, n_etabins=60), parts=14),
    "limits": dict(geo=dict(seed=7, n_layers=32, n_regions_total=256, n_eta_range=(1, 60),
                            n_phi_choices=(64, 128, 256, 512)),
                   prm=dict(seed=13, eta_bin_scale=20, ebin_log2_min=6, r_edge_kind="std", a_edge_kind="std"),
                   parts=15),
}


def edge_case(name, subnormal_frac=True):
    """(geometry, parametrisation, particles) of an edge case."""
    from paper_2103_14737_gb300 import synth
    c = EDGE_CASES[name]
    geo = synth.random_geometry(**c["geo"])
    prm = synth.edge_params(geo, subnormal_frac=subnormal_frac, **c["prm"])
    parts = synth.edge_particles(c["parts"], geo, prm)
    return geo, prm, parts
