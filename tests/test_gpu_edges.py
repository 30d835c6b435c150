"""GPU parity on the method's edge inputs (tests/parity.py: EDGE_CASES),
through the C ABI against the oracle on the same seeded inputs.

The inputs leave the default geometry and parametrisation: geometries
without mirror symmetry, with gaps, adjacent and overlapping region
boundaries, 1 to 4 regions per layer, non-dyadic granularities, partial phi
coverage, and one at the ABI's limits (32 layers, 256 regions, more than
2^19 cells, so 64-bit match keys); histograms with interior zero-weight
bins, trailing zero bins (every last bin from 0 to 126), single bins, steep
CDFs whose guide cells span tens of bins, weights over 24 decades and at a
1e-30 scale (the guide-table build and the binary search of the shape bin);
entries whose mean hit energy forces one hit; subnormal layer fractions;
particles exactly on |eta|-bin edges (integer and non-integer scales),
power-of-two energy edges and region boundaries, one float ulp either side,
phi at +-pi and beyond the circle, eta far outside the coverage.

Bars as in tests/parity.py: tasks, hits, hit bins and hit cells bit-exact;
deterministic cells bit-exact; atomic cells within 1e-5 |E| + 1e-3 MeV;
gradients within the adjoint's bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2103_14737_gb300 import fcs  # noqa: E402
from parity import (EDGE_CASES, check_cells_atomic, check_cells_det, check_grad, check_tasks_hits,  # noqa: E402
                    edge_case, grad_scales, run_both)

SEED, FIRST_EVENT = 5, 2


def _setup(name, subnormal_frac=True):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    geo, prm, parts = edge_case(name, subnormal_frac=subnormal_frac)
    sim = fcs.Simulator(geo, prm)
    return dict(name=name, geo=geo, prm=prm, parts=parts, sim=sim, og=O.OracleGeometry(geo),
                op=O.OracleParams(prm))


@pytest.fixture(scope="module", params=list(EDGE_CASES))
def case(request):
    c = _setup(request.param)
    yield c
    c["sim"].close()


def _run(c, **kw):
    return run_both(c["sim"], c["og"], c["op"], c["parts"], SEED, first_event=FIRST_EVENT, **kw)


def test_atomic(case):
    ref, got = _run(case)
    check_tasks_hits(ref, got)
    check_cells_atomic(ref, got, case["parts"].n_events)
    assert (ref.task_n == 1).sum() > 0


def test_deterministic(case):
    ref, got = _run(case, mode=fcs.MODE_DETERMINISTIC)
    check_tasks_hits(ref, got)
    check_cells_det(ref, got, case["parts"].n_events)


@pytest.mark.parametrize("block,hpt", [(512, 1), (256, 8)])
def test_launch_shapes(case, block, hpt):
    ref, got = _run(case, block=block, hpt=hpt)
    check_tasks_hits(ref, got)
    check_cells_atomic(ref, got, case["parts"].n_events)


def test_per_event_launches(case):
    ref, got = _run(case, batched=0, mode=fcs.MODE_DETERMINISTIC)
    check_tasks_hits(ref, got)
    check_cells_det(ref, got, case["parts"].n_events)


def test_per_task_launches(case):
    if case["name"] == "limits":
        pytest.skip("tens of thousands of tasks: one launch each takes minutes")
    ref, got = _run(case, batched=2, hits=False)
    check_tasks_hits(ref, got)
    check_cells_atomic(ref, got, case["parts"].n_events)


def test_energy_interpolation(case):
    op_i = O.OracleParams(case["prm"], energy_interp=1)
    ref, got = run_both(case["sim"], case["og"], op_i, case["parts"], SEED, first_event=FIRST_EVENT,
                        mode=fcs.MODE_DETERMINISTIC, energy_interp=1)
    check_tasks_hits(ref, got)
    check_cells_det(ref, got, case["parts"].n_events)


@pytest.mark.parametrize("name", list(EDGE_CASES))
def test_backward(name):
    """The adjoint on the edge inputs (no subnormal fractions: a subnormal
    float hit energy carries fewer significant bits than the adjoint's bound
    assumes)."""
    c = _setup(name, subnormal_frac=False)
    try:
        sim, parts = c["sim"], c["parts"]
        rng = np.random.default_rng(9)
        g = rng.normal(size=(parts.n_events, sim.n_cells)).astype(np.float32)
        r = sim.backward(sim.to_device(parts), SEED, torch.as_tensor(g, device="cuda"), first_event=FIRST_EVENT)
        torch.cuda.synchronize()
        g64 = g.astype(np.float64)
        ref_f, ref_w = O.backward(c["og"], c["op"], parts, SEED, g64, first_event=FIRST_EVENT)
        sc_f, sc_w = grad_scales(c["og"], c["op"], c["prm"], parts, SEED, g64, first_event=FIRST_EVENT)
        check_grad(r["d_frac"], r["d_shape_w"], ref_f, ref_w, sc_f, sc_w)
    finally:
        c["sim"].close()


def test_subnormal_energy_bins():
    """Energy bins of subnormal particle energies (floor(log2 E) below -126)
    with a table whose first bin starts at 2^-150: every particle's layer
    fraction is 1 on one layer, so even a subnormal energy makes a task, and
    the task lists, hit bins and deterministic cells show the bin chosen."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_14737_gb300 import synth
    geo = synth.random_geometry(101)
    prm = synth.edge_params(geo, 21, n_types=1, n_ebins=40, n_etabins=8, eta_bin_scale=2.0, ebin_log2_min=-150)
    frac = np.zeros_like(prm.frac)
    frac[..., 0] = 1.0
    prm.frac = frac
    prm.mean_hit_E = np.full_like(prm.mean_hit_E, 2.0**-136)
    w = prm.shape_w.reshape(-1, 128)
    w[w.sum(1) == 0] = 1.0
    rng = np.random.default_rng(4)
    E = np.concatenate([np.float32(2.0) ** -np.arange(126, 150, dtype=np.float32),
                        np.float32(2.0**-149) * rng.integers(1, 1 << 23, size=40).astype(np.float32),
                        np.float32(2.0) ** -np.arange(124, 127, dtype=np.float32)]).astype(np.float32)
    n = len(E)
    parts = synth.Particles(np.zeros(n, np.int32), E, rng.uniform(-2.0, 2.0, n).astype(np.float32),
                            rng.uniform(-3.0, 3.0, n).astype(np.float32), np.array([0, n], np.int64))
    sim = fcs.Simulator(geo, prm)
    try:
        og, op = O.OracleGeometry(geo), O.OracleParams(prm)
        ref, got = run_both(sim, og, op, parts, 3, mode=fcs.MODE_DETERMINISTIC)
        check_tasks_hits(ref, got)
        check_cells_det(ref, got, 1)
        assert ref.n_tasks == n
    finally:
        sim.close()


def test_extreme_eta_end_caps():
    """Particles at |eta| = 20, 40 and 95.  In an end-cap layer the map's
    scale sinh|eta| / |z| reaches 1e13 - 1e38, so a hit lands at |phi| up to
    1e15 (or beyond the float range, which the FP32 path hands to the FP64
    recheck): there the FP64 position moves by more than a cell when CUDA's
    and the C library's sinh, sin or cos differ in the last bit, and the cell
    is not a reproducible function of the inputs.  Compared: the task lists,
    counts, hit energies and hit bins bit-exact; the cells of every barrel
    hit and of end-cap hits of |eta| < 20 bit-exact; every other hit's cell a
    cell of its own layer; each event's energy equal to its tasks' energy."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_14737_gb300 import synth
    geo, prm, _ = edge_case("asym8")
    parts = synth.edge_particles(31, geo, prm, n_events=3, n_random=40, extreme_eta=(20.0, -20.0, 40.0, -40.0, 95.0))
    sim = fcs.Simulator(geo, prm)
    try:
        og, op = O.OracleGeometry(geo), O.OracleParams(prm)
        ref, got = run_both(sim, og, op, parts, SEED)
        assert got["status"] == 0 and got["stats"]["n_tasks"] == ref.n_tasks
        for k in ("task_event", "task_particle", "task_layer", "task_n"):
            assert np.array_equal(got[k].cpu().numpy(), getattr(ref, k)), k
        assert np.array_equal(got["task_Ehit"].cpu().numpy().view(np.uint32), ref.task_Ehit.view(np.uint32))
        assert np.array_equal(got["hit_bin"].cpu().numpy(), ref.hit_bin)
        gp = parts.event_offsets[ref.task_event] + ref.task_particle
        ill = (geo.layers["barrel"][ref.task_layer] == 0) & (np.abs(parts.eta[gp]) >= 20.0)
        assert ill.sum() > 0
        hit_ill = np.repeat(ill, ref.task_n)
        hc = got["hit_cell"].cpu().numpy()
        assert np.array_equal(hc[~hit_ill], ref.hit_cell[~hit_ill])
        lrb, reg = geo.layer_region_begin, geo.regions
        lay = np.repeat(ref.task_layer, ref.task_n)
        lo = reg["cell_offset"][lrb[lay]]
        last = lrb[lay + 1] - 1
        hi = reg["cell_offset"][last] + reg["n_eta"][last] * reg["n_phi"][last]
        assert ((hc >= lo) & (hc < hi)).all()
        cells = got["cells"].cpu().numpy().astype(np.float64)
        want = np.bincount(ref.task_event, weights=ref.task_n * ref.task_Ehit.astype(np.float64),
                           minlength=parts.n_events)
        assert np.allclose(cells.sum(1), want, rtol=1e-5)
    finally:
        sim.close()
