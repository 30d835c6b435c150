"""CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

Bars (Sec. 6 of the paper validates CPU and GPU hit by hit on the same random
numbers and asks for identical cells):
  * task counts, hit counts and the hit -> cell and hit -> bin maps: bit-exact;
  * hit energies (float, Listing 1): bit-exact;
  * atomic mode cell energies: |dE| <= 1e-5 |E| + 1e-3 MeV against the FP64
    oracle (FP32 atomics in any order);
  * deterministic mode: bit-exact against the oracle's canonical FP32 fold.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2103_14737_gb300 import fcs, synth  # noqa: E402
from parity import (ATOL, RTOL, check_cells_atomic, check_compacted, check_tasks_hits,  # noqa: E402
                    run_both)

# kernels of one event range in a replayed graph (begin and end of the call
# add two more)
KERNELS_PER_RANGE = 10


@pytest.fixture(scope="module")
def sim(geo, prm):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = fcs.Simulator(geo, prm)
    yield s
    s.close()


@pytest.mark.parametrize("batched", [1, 0])
def test_single_electron_parity(sim, ogeo, oprm, batched):
    parts = synth.single_particle(8)
    ref, got = run_both(sim, ogeo, oprm, parts, seed=1, batched=batched)
    check_tasks_hits(ref, got)
    check_cells_atomic(ref, got, 8)


def test_ttbar_parity_atomic(sim, ogeo, oprm):
    parts = synth.ttbar_like(seed=1)
    ref, got = run_both(sim, ogeo, oprm, parts, seed=7, first_event=3)
    check_tasks_hits(ref, got)
    check_cells_atomic(ref, got, 1)


def test_ttbar_high_hit_params(geo, ogeo):
    """The hard-scatter event with mean hit energies of 0.5-20 MeV instead of
    5-200 MeV (ten times the hits, about 2M): tasks, hits, per-hit cells and
    deterministic cells bit-exact, atomic cells within tolerance."""
    prm_hi = synth.params(geo, mean_hit_range=(0.5, 20.0))
    s = fcs.Simulator(geo, prm_hi)
    try:
        oprm_hi = O.OracleParams(prm_hi)
        parts = synth.ttbar_like(seed=3)
        ref, got = run_both(s, ogeo, oprm_hi, parts, seed=11, first_event=1)
        assert ref.n_hits > 1_000_000
        check_tasks_hits(ref, got)
        check_cells_atomic(ref, got, 1)
        det = s.simulate(s.to_device(parts), 11, first_event=1, mode=fcs.MODE_DETERMINISTIC, dense=True)
        torch.cuda.synchronize()
        assert np.array_equal(det["cells"].cpu().numpy().view(np.uint32), ref.cells_canon.view(np.uint32))
    finally:
        s.close()


@pytest.mark.parametrize("batched", [1, 0])
def test_deterministic_bit_exact(sim, ogeo, oprm, batched):
    parts = synth.pileup(seed=4, n_events=3, mu_pu=15)
    ref, got = run_both(sim, ogeo, oprm, parts, seed=11, mode=fcs.MODE_DETERMINISTIC, batched=batched)
    check_tasks_hits(ref, got)
    cells = got["cells"].cpu().numpy()
    assert np.array_equal(cells.view(np.uint32), ref.cells_canon.view(np.uint32))
    check_compacted(got, cells.astype(np.float64), 3)


def test_deterministic_hot_cells(sim, ogeo, oprm):
    """1 TeV electrons: tens of thousands of hits in a few tasks, so the core
    cells collect hundreds of records (the long-segment sort of the fold)."""
    parts = synth.single_particle(2, E=float(2 ** 20), eta=-1.1)
    ref, got = run_both(sim, ogeo, oprm, parts, seed=3, mode=fcs.MODE_DETERMINISTIC, hits=False)
    check_tasks_hits(ref, got)
    cells = got["cells"].cpu().numpy()
    assert np.array_equal(cells.view(np.uint32), ref.cells_canon.view(np.uint32))
    assert ref.n_hits > 20000


@pytest.mark.parametrize("block,hpt", [(128, 1), (128, 8), (256, 2), (256, 4), (512, 1), (512, 8)])
def test_launch_shapes(sim, ogeo, oprm, block, hpt):
    parts = synth.pileup(seed=6, n_events=2, mu_pu=10)
    ref, got = run_both(sim, ogeo, oprm, parts, seed=5, hpt=hpt, block=block)
    check_tasks_hits(ref, got)
    check_cells_atomic(ref, got, 2)
    got2 = sim.simulate(sim.to_device(parts), 5, mode=fcs.MODE_DETERMINISTIC, hits_per_thread=hpt, block=block,
                        dense=True)
    assert np.array_equal(got2["cells"].cpu().numpy().view(np.uint32), ref.cells_canon.view(np.uint32))


@pytest.mark.parametrize("mode", [fcs.MODE_ATOMIC, fcs.MODE_DETERMINISTIC])
@pytest.mark.parametrize("wave", [1, 2, 3])
def test_event_waves(sim, ogeo, oprm, mode, wave):
    """Launch sequences of `wave` events (a ragged last wave): the same tasks,
    cells and compacted output as the oracle."""
    parts = synth.pileup(seed=14, n_events=5, mu_pu=8)
    d = sim.to_device(parts)
    ref = O.simulate(ogeo, oprm, parts, seed=9, first_event=3)
    for timing in (0, 1):
        got = sim.simulate(d, 9, first_event=3, mode=mode, wave_events=wave, dense=True, debug_tasks=ref.n_tasks,
                           timing=timing)
        check_tasks_hits(ref, got)
        cells = got["cells"].cpu().numpy()
        if mode == fcs.MODE_DETERMINISTIC:
            assert np.array_equal(cells.view(np.uint32), ref.cells_canon.view(np.uint32))
            check_compacted(got, cells.astype(np.float64), 5)
        else:
            check_cells_atomic(ref, got, 5)
    t = fcs.fcs_workspace_timings(sim.ws)
    assert t["total"] > 0


@pytest.mark.parametrize("block,hpt", [(128, 1), (256, 4)])
def test_per_task_launches(sim, ogeo, oprm, block, hpt):
    """One hit-kernel launch per task (the paper's non-grouped GPU mode): every
    hit once, the same cells as the oracle."""
    parts = synth.replicate(synth.ttbar_like(2, 1, n=40), 2)
    ref, got = run_both(sim, ogeo, oprm, parts, seed=4, batched=2, hpt=hpt, block=block)
    check_tasks_hits(ref, got)
    check_cells_atomic(ref, got, 2)
    got = sim.simulate(sim.to_device(parts), 4, mode=fcs.MODE_DETERMINISTIC, batched=2, hits_per_thread=hpt,
                       block=block, dense=True)
    assert np.array_equal(got["cells"].cpu().numpy().view(np.uint32), ref.cells_canon.view(np.uint32))


@pytest.mark.parametrize("mode", [fcs.MODE_ATOMIC, fcs.MODE_DETERMINISTIC])
def test_energy_interpolation(sim, ogeo, prm, mode):
    """Probabilistic energy-bin interpolation: tasks, hits and cells as the
    oracle with the same option."""
    oprm_i = O.OracleParams(prm, energy_interp=1)
    parts = synth.pileup(seed=15, n_events=3, mu_pu=10)
    ref = O.simulate(ogeo, oprm_i, parts, seed=6, first_event=2, hit_cap=10**7)
    got = sim.simulate(sim.to_device(parts), 6, first_event=2, mode=mode, dense=True, energy_interp=1,
                       debug_tasks=ref.n_tasks, debug_hits=ref.n_hits)
    check_tasks_hits(ref, got)
    if mode == fcs.MODE_DETERMINISTIC:
        assert np.array_equal(got["cells"].cpu().numpy().view(np.uint32), ref.cells_canon.view(np.uint32))
    else:
        check_cells_atomic(ref, got, 3)
    plain = O.simulate(ogeo, O.OracleParams(prm), parts, seed=6, first_event=2)
    assert plain.n_tasks != ref.n_tasks or not np.array_equal(plain.task_n, ref.task_n)


def test_poisson_counts_wide_mu(sim, ogeo, oprm):
    """Hit counts over mu from ~1e-2 to ~1e5 (inversion, FP32-certified PTRS,
    the FP64-only large-mu path) equal the oracle's draw for draw."""
    rng = np.random.default_rng(12)
    n = 3000
    E = (2.0 ** rng.uniform(6.0, 22.0, n)).astype(np.float32)
    parts = synth.Particles(rng.integers(0, 3, n).astype(np.int32), E,
                            rng.uniform(-3.2, 3.2, n).astype(np.float32),
                            rng.uniform(-np.pi, np.pi, n).astype(np.float32),
                            np.array([0, 1000, 2000, 3000], dtype=np.int64))
    ref, got = run_both(sim, ogeo, oprm, parts, seed=77, first_event=9, hits=False)
    check_tasks_hits(ref, got)
    # tasks above mu = 4096 (about 15 % here) are drawn in FP64 on purpose
    assert got["stats"]["n_poisson_fp64"] < 0.25 * ref.n_tasks


def test_poisson_large_mu_draw_for_draw(sim, prm, oprm):
    """Hit counts of 6000 particles of 16 GeV to 1 TeV (means from tens to
    tens of thousands: PTRS draws that reject and continue at later
    iterations, uncertain FP32 decisions redone in FP64 from the iteration
    where they arose, and the FP64-only large-mu path) equal the oracle's
    Poisson function applied to each task's mean, draw for draw."""
    rng = np.random.default_rng(31)
    n = 6000
    E = (2.0 ** rng.uniform(14.0, 20.0, n)).astype(np.float32)
    ptype = rng.integers(0, 3, n).astype(np.int32)
    eta = rng.uniform(-2.4, 2.4, n).astype(np.float32)
    parts = synth.Particles(ptype, E, eta, rng.uniform(-np.pi, np.pi, n).astype(np.float32),
                            np.array([0, n], dtype=np.int64))
    got = sim.simulate(sim.to_device(parts), 5, first_event=3, debug_tasks=n * 24)
    torch.cuda.synchronize()
    k = got["stats"]["n_tasks"]
    lay = got["task_layer"].cpu().numpy()[:k]
    par = got["task_particle"].cpu().numpy()[:k]
    n_gpu = got["task_n"].cpu().numpy()[:k]
    NL = prm.frac.shape[-1]
    frac = prm.frac.reshape(-1, NL)
    mhe = prm.mean_hit_E.reshape(-1, NL)
    entry = np.array([O.param_entry(oprm, int(ptype[i]), float(E[i]), float(eta[i])) for i in range(n)])
    e = entry[par]
    El = (E[par] * frac[e, lay]).astype(np.float32)  # fl32(E f), then fl32(E_l / mean hit energy)
    mu = (El / mhe[e, lay]).astype(np.float32)
    ref = np.maximum(O.poisson(mu.astype(np.float64), 5, lay, par, 3), 1)
    assert (mu >= 10).sum() > 0.5 * k and (mu > 4096).sum() > 0
    assert np.array_equal(ref, n_gpu.astype(np.int64))
    assert got["stats"]["n_poisson_fp64"] > 0


def test_pileup_events_parity(sim, ogeo, oprm):
    parts = synth.pileup(seed=8, n_events=2)  # full mu = 200 pile-up events
    ref, got = run_both(sim, ogeo, oprm, parts, seed=1, hits=False)
    check_tasks_hits(ref, got)
    check_cells_atomic(ref, got, 2)
    assert got["stats"]["n_recheck"] < 0.01 * ref.n_hits
    assert got["stats"]["n_poisson_fp64"] < 0.01 * ref.n_tasks


def test_empty_events_and_zero_events(sim, ogeo, oprm):
    p = synth.ttbar_like(seed=2, n_events=3, n=50)
    # make event 1 empty
    keep = np.r_[0:50, 100:150]
    parts = synth.Particles(p.type[keep], p.E[keep], p.eta[keep], p.phi[keep], np.array([0, 50, 50, 100]))
    ref, got = run_both(sim, ogeo, oprm, parts, seed=3)
    check_tasks_hits(ref, got)
    check_cells_atomic(ref, got, 3)
    off = got["event_offsets"].cpu().numpy()
    assert off[1] == off[2]
    empty = synth.Particles(p.type[:0], p.E[:0], p.eta[:0], p.phi[:0], np.array([0]))
    r = sim.simulate(sim.to_device(empty), 1)
    assert r["status"] == 0 and r["event_offsets"].cpu().numpy().tolist() == [0]


def test_bad_particle_and_capacity(sim):
    p = synth.ttbar_like(seed=3, n=20)
    p.type[5] = 7
    p.E[6] = np.nan
    r = sim.simulate(sim.to_device(p), 1, check=False)
    assert r["status"] == fcs.FCS_E_DEVICE_CHECK
    assert r["stats"]["device_flags"] & fcs.FLAG_BAD_PARTICLE
    p = synth.ttbar_like(seed=3, n=20)
    full = sim.simulate(sim.to_device(p), 1)
    nnz = full["stats"]["n_nonzero"]
    small = sim.simulate(sim.to_device(p), 1, capacity=nnz - 5, check=False)
    assert small["status"] == fcs.FCS_E_RANGE
    assert small["event_offsets"][-1].item() == nnz
    assert np.array_equal(small["cell_ids"].cpu().numpy(), full["cell_ids"][:nnz - 5].cpu().numpy())


def test_async_graph_replay_matches(sim):
    parts = synth.pileup(seed=9, n_events=4, mu_pu=30)
    d = sim.to_device(parts)
    ref = sim.simulate(d, 21, dense=True)
    outs = dict(cell_ids=torch.empty_like(ref["cell_ids"]), cell_E=torch.empty_like(ref["cell_E"]),
                event_offsets=torch.empty_like(ref["event_offsets"]), cells=torch.empty_like(ref["cells"]))
    for _ in range(3):
        outs["cells"].fill_(-1)
        sim.simulate(d, 21, sync=0, use_graph=1, outputs=outs)
    torch.cuda.synchronize()
    rc, st = fcs.fcs_workspace_status(sim.ws)
    assert rc == 0 and st.n_nonzero == ref["stats"]["n_nonzero"]
    diff = (outs["cells"] - ref["cells"]).abs()
    assert (diff <= RTOL * ref["cells"].abs() + ATOL).all()
    # the launch sequence of one event range (10 kernels): range begin,
    # particle counts, the task-offset scan, task records with their FP32
    # Poisson draws, the FP64 draws, the hit-offset scan with the tile map,
    # hits, recheck, the one-pass compaction, range end; plus call begin and
    # end
    assert fcs.fcs_workspace_graph_kernels(sim.ws) == 2 + KERNELS_PER_RANGE
    sim.simulate(d, 21, sync=0, use_graph=1, outputs=outs, wave_events=2)
    torch.cuda.synchronize()
    assert fcs.fcs_workspace_graph_kernels(sim.ws) == 2 + 2 * KERNELS_PER_RANGE


def test_host_entry_point_matches(sim):
    parts = synth.pileup(seed=10, n_events=2, mu_pu=20)
    ref = sim.simulate(sim.to_device(parts), 4, mode=fcs.MODE_DETERMINISTIC)
    cap = ref["stats"]["n_nonzero"] + 10
    ids = np.empty(cap, np.int32)
    E = np.empty(cap, np.float32)
    off = np.empty(3, np.int64)
    cfg = fcs.make_config(mode=fcs.MODE_DETERMINISTIC)
    rc, st = fcs.fcs_simulate_events_host(sim.geo, sim.prm, sim.ws, parts.type, parts.E, parts.eta, parts.phi,
                                          parts.event_offsets, 4, 0, cfg, ids, E, off)
    n = st.n_nonzero
    assert np.array_equal(off, ref["event_offsets"].cpu().numpy())
    assert np.array_equal(ids[:n], ref["cell_ids"][:n].cpu().numpy())
    assert np.array_equal(E[:n].view(np.uint32), ref["cell_E"][:n].cpu().numpy().view(np.uint32))


def test_host_entry_point_pinned_outputs(sim):
    """Mapped pinned host outputs are written by the device directly."""
    parts = synth.pileup(seed=16, n_events=3, mu_pu=20)
    ref = sim.simulate(sim.to_device(parts), 4, mode=fcs.MODE_DETERMINISTIC)
    cap = ref["stats"]["n_nonzero"] + 10
    ids = torch.full((cap,), -1, dtype=torch.int32).pin_memory()
    E = torch.zeros(cap, dtype=torch.float32).pin_memory()
    off = torch.zeros(4, dtype=torch.int64).pin_memory()
    cfg = fcs.make_config(mode=fcs.MODE_DETERMINISTIC)
    rc, st = fcs.fcs_simulate_events_host(sim.geo, sim.prm, sim.ws, parts.type, parts.E, parts.eta, parts.phi,
                                          parts.event_offsets, 4, 0, cfg, ids.numpy(), E.numpy(), off.numpy())
    n = st.n_nonzero
    assert rc == 0 and n == ref["stats"]["n_nonzero"]
    assert np.array_equal(off.numpy(), ref["event_offsets"].cpu().numpy())
    assert np.array_equal(ids.numpy()[:n], ref["cell_ids"][:n].cpu().numpy())
    assert np.array_equal(E.numpy()[:n].view(np.uint32), ref["cell_E"][:n].cpu().numpy().view(np.uint32))
    assert (ids.numpy()[n:] == -1).all()


def test_host_entry_point_two_waves(sim):
    """Pinned inputs and outputs: after a sizing call the host entry runs as two
    waves on three streams (copies in, compute and results out overlapped),
    one graph of 2 + 2 x KERNELS_PER_RANGE kernels; its cells match the deterministic
    device call (atomic tolerance) and its ids and offsets match exactly, for
    an odd event count and over repeated calls."""
    parts = synth.pileup(seed=17, n_events=5, mu_pu=30)
    ref = sim.simulate(sim.to_device(parts), 6, first_event=2, mode=fcs.MODE_DETERMINISTIC)
    nnz = ref["stats"]["n_nonzero"]
    cap = nnz + 16
    pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(parts, k))).pin_memory()
           for k in ("type", "E", "eta", "phi", "event_offsets")}
    ids = torch.full((cap,), -1, dtype=torch.int32).pin_memory()
    E = torch.zeros(cap, dtype=torch.float32).pin_memory()
    off = torch.zeros(6, dtype=torch.int64).pin_memory()
    cfg = fcs.make_config()
    ref_ids = ref["cell_ids"][:nnz].cpu().numpy()
    ref_E = ref["cell_E"][:nnz].cpu().numpy().astype(np.float64)
    for call in range(3):
        ids.fill_(-1)
        E.zero_()
        rc, st = fcs.fcs_simulate_events_host(sim.geo, sim.prm, sim.ws, pin["type"].numpy(), pin["E"].numpy(),
                                              pin["eta"].numpy(), pin["phi"].numpy(), pin["event_offsets"].numpy(),
                                              6, 2, cfg, ids.numpy(), E.numpy(), off.numpy())
        assert rc == 0 and st.n_nonzero == nnz and st.n_hits == ref["stats"]["n_hits"]
        assert np.array_equal(off.numpy(), ref["event_offsets"].cpu().numpy())
        assert np.array_equal(ids.numpy()[:nnz], ref_ids)
        err = np.abs(E.numpy()[:nnz].astype(np.float64) - ref_E)
        assert (err <= RTOL * np.abs(ref_E) + ATOL).all()
        assert (ids.numpy()[nnz:] == -1).all()
        if call > 0:  # the first call may size the workspace synchronously
            assert fcs.fcs_workspace_graph_kernels(sim.ws) == 2 + 2 * KERNELS_PER_RANGE


def test_host_entry_point_four_waves(sim):
    """A host-buffer call of 512 events or more runs as four waves (2/8 of the
    events each): one graph of 2 + 4 x KERNELS_PER_RANGE kernels,
    whose ids and offsets equal the deterministic device call's and whose
    cells lie within the atomic tolerance, over repeated calls."""
    n_ev = 512
    parts = synth.pileup(seed=23, n_events=n_ev, mu_pu=1, per_collision=6, hs_particles=6)
    ref = sim.simulate(sim.to_device(parts), 8, first_event=5, mode=fcs.MODE_DETERMINISTIC)
    nnz = ref["stats"]["n_nonzero"]
    cap = nnz + 16
    pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(parts, k))).pin_memory()
           for k in ("type", "E", "eta", "phi", "event_offsets")}
    ids = torch.full((cap,), -1, dtype=torch.int32).pin_memory()
    E = torch.zeros(cap, dtype=torch.float32).pin_memory()
    off = torch.zeros(n_ev + 1, dtype=torch.int64).pin_memory()
    cfg = fcs.make_config()
    ref_ids = ref["cell_ids"][:nnz].cpu().numpy()
    ref_E = ref["cell_E"][:nnz].cpu().numpy().astype(np.float64)
    for call in range(3):
        ids.fill_(-1)
        E.zero_()
        rc, st = fcs.fcs_simulate_events_host(sim.geo, sim.prm, sim.ws, pin["type"].numpy(), pin["E"].numpy(),
                                              pin["eta"].numpy(), pin["phi"].numpy(), pin["event_offsets"].numpy(),
                                              8, 5, cfg, ids.numpy(), E.numpy(), off.numpy())
        assert rc == 0 and st.n_nonzero == nnz and st.n_hits == ref["stats"]["n_hits"]
        assert np.array_equal(off.numpy(), ref["event_offsets"].cpu().numpy())
        assert np.array_equal(ids.numpy()[:nnz], ref_ids)
        err = np.abs(E.numpy()[:nnz].astype(np.float64) - ref_E)
        assert (err <= RTOL * np.abs(ref_E) + ATOL).all()
        if call > 0:  # the first call may size the workspace synchronously
            assert fcs.fcs_workspace_graph_kernels(sim.ws) == 2 + 4 * KERNELS_PER_RANGE


@pytest.mark.parametrize("layout", ["two_events", "empty_first_wave"])
def test_host_entry_point_two_waves_edges(sim, layout):
    """Two-wave host calls at their edges: two events (a wave each), and a first
    wave whose events have no particles (all particles in the last quarter)."""
    src = synth.pileup(seed=18, n_events=2, mu_pu=10)
    if layout == "two_events":
        parts = src
    else:
        # eight events: six empty, then the two events above
        parts = synth.Particles(src.type, src.E, src.eta, src.phi,
                                np.concatenate([np.zeros(6, np.int64), src.event_offsets]).astype(np.int64))
    ne = len(parts.event_offsets) - 1
    ref = sim.simulate(sim.to_device(parts), 8, mode=fcs.MODE_DETERMINISTIC)
    nnz = ref["stats"]["n_nonzero"]
    pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(parts, k))).pin_memory()
           for k in ("type", "E", "eta", "phi", "event_offsets")}
    ids = torch.full((nnz + 8,), -1, dtype=torch.int32).pin_memory()
    E = torch.zeros(nnz + 8, dtype=torch.float32).pin_memory()
    off = torch.zeros(ne + 1, dtype=torch.int64).pin_memory()
    for _ in range(2):
        rc, st = fcs.fcs_simulate_events_host(sim.geo, sim.prm, sim.ws, pin["type"].numpy(), pin["E"].numpy(),
                                              pin["eta"].numpy(), pin["phi"].numpy(), pin["event_offsets"].numpy(),
                                              8, 0, fcs.make_config(), ids.numpy(), E.numpy(), off.numpy())
        assert rc == 0 and st.n_nonzero == nnz and st.n_hits == ref["stats"]["n_hits"]
        assert np.array_equal(off.numpy(), ref["event_offsets"].cpu().numpy())
        assert np.array_equal(ids.numpy()[:nnz], ref["cell_ids"][:nnz].cpu().numpy())
        want = ref["cell_E"][:nnz].cpu().numpy().astype(np.float64)
        assert (np.abs(E.numpy()[:nnz] - want) <= RTOL * np.abs(want) + ATOL).all()
    assert fcs.fcs_workspace_graph_kernels(sim.ws) == 2 + 2 * KERNELS_PER_RANGE


def test_host_entry_point_async_two_workspaces(sim):
    """config sync = 0: host calls on two fresh workspaces and two streams,
    enqueued without waiting and interleaved, return the synchronous call's
    cells (ids and offsets exactly, energies to the atomic tolerance); each
    status comes from fcs_workspace_status.  A fresh workspace's first call
    sizes it synchronously."""
    parts = synth.pileup(seed=21, n_events=6, mu_pu=30)
    pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(parts, k))).pin_memory().numpy()
           for k in ("type", "E", "eta", "phi", "event_offsets")}
    cap = 6 * sim.n_cells

    def bufs():
        return (torch.full((cap,), -1, dtype=torch.int32).pin_memory().numpy(),
                torch.zeros(cap, dtype=torch.float32).pin_memory().numpy(),
                torch.zeros(7, dtype=torch.int64).pin_memory().numpy())

    ref = bufs()
    rc, st = fcs.fcs_simulate_events_host(sim.geo, sim.prm, sim.ws, pin["type"], pin["E"], pin["eta"], pin["phi"],
                                          pin["event_offsets"], 4, 1, fcs.make_config(), *ref)
    assert rc == 0
    nnz = st.n_nonzero
    acfg = fcs.make_config(sync=0)
    slots = [(fcs.fcs_workspace_create(), torch.cuda.Stream(), bufs()) for _ in range(2)]
    try:
        for rep in range(3):
            for ws, stream, out in slots:
                out[0].fill(-1)
                with torch.cuda.stream(stream):
                    rc, _ = fcs.fcs_simulate_events_host(sim.geo, sim.prm, ws, pin["type"], pin["E"], pin["eta"],
                                                         pin["phi"], pin["event_offsets"], 4, 1, acfg, *out)
                assert rc == 0
            for ws, stream, out in slots:
                with torch.cuda.stream(stream):
                    rc, st = fcs.fcs_workspace_status(ws)
                assert rc == 0 and st.n_nonzero == nnz
                assert np.array_equal(out[2], ref[2]) and np.array_equal(out[0][:nnz], ref[0][:nnz])
                want = ref[1][:nnz].astype(np.float64)
                assert (np.abs(out[1][:nnz] - want) <= RTOL * np.abs(want) + ATOL).all()
                assert (out[0][nnz:] == -1).all()
        assert fcs.fcs_workspace_graph_kernels(slots[0][0]) == 2 + 2 * KERNELS_PER_RANGE
    finally:
        torch.cuda.synchronize()
        for ws, _, _ in slots:
            fcs.fcs_workspace_free(ws)


def test_bounded_wait_gives_up(sim):
    """A device wait that nothing ends (a scan tile that never publishes its
    status) gives up after its poll limit; the call reports FCS_E_TIMEOUT and the
    device stays usable: a simulation call right after it succeeds."""
    rc, ms = fcs.fcs_selftest_wait_timeout()
    assert rc == fcs.FCS_E_TIMEOUT, rc
    assert 0.0 < ms < 20000.0, ms
    parts = synth.pileup(seed=19, n_events=1, mu_pu=5)
    r = sim.simulate(sim.to_device(parts), 3)
    assert r["status"] == 0 and r["stats"]["n_hits"] > 0


def test_allocation_failure_is_reported(geo, prm, sim):
    """A workspace request larger than the device (2^46 hits: a tile map of
    2 TiB) is refused by cudaMalloc and reported as FCS_E_OOM; the workspace
    stays usable and its next call gives the same deterministic cells as a
    workspace that never failed."""
    s = fcs.Simulator(geo, prm)
    try:
        with pytest.raises(fcs.FcsError) as ei:
            fcs.fcs_workspace_reserve(s.ws, s.geo, 0, 1, 1 << 46)
        assert ei.value.code == fcs.FCS_E_OOM
        parts = synth.pileup(seed=23, n_events=2, mu_pu=5)
        a = s.simulate(s.to_device(parts), 5, mode=fcs.MODE_DETERMINISTIC, dense=True)
        b = sim.simulate(sim.to_device(parts), 5, mode=fcs.MODE_DETERMINISTIC, dense=True)
        assert a["status"] == 0 and b["status"] == 0
        assert torch.equal(a["cells"].view(torch.int32), b["cells"].view(torch.int32))
    finally:
        s.close()


def test_sync_call_outgrows_workspace(geo, prm, ogeo, oprm):
    """A fresh workspace is sized by its first call; a larger later call
    overflows it, grows it and runs again with the same results."""
    s = fcs.Simulator(geo, prm)
    try:
        small = synth.single_particle(1)
        s.simulate(s.to_device(small), 2, mode=fcs.MODE_DETERMINISTIC)
        big = synth.pileup(seed=17, n_events=2, mu_pu=30)
        got = s.simulate(s.to_device(big), 5, mode=fcs.MODE_DETERMINISTIC, dense=True)
        ref = O.simulate(ogeo, oprm, big, seed=5)
        assert got["stats"]["n_hits"] == ref.n_hits
        assert np.array_equal(got["cells"].cpu().numpy().view(np.uint32), ref.cells_canon.view(np.uint32))
        got2 = s.simulate(s.to_device(big), 5, dense=True)
        check_cells_atomic(ref, got2, 2)
    finally:
        s.close()


def test_autotune_picks_a_valid_shape(sim, ogeo, oprm):
    parts = synth.pileup(seed=13, n_events=2, mu_pu=20)
    d = sim.to_device(parts)
    b, h, table = sim.autotune(d, 3, reps=1)
    assert (b, h) in table and len(table) == 12
    assert all(v > 0 for v in table.values()) and table[(b, h)] == min(table.values())
    ref = O.simulate(ogeo, oprm, parts, seed=3)
    got = sim.simulate(d, 3, block=b, hits_per_thread=h, mode=fcs.MODE_DETERMINISTIC, dense=True)
    assert np.array_equal(got["cells"].cpu().numpy().view(np.uint32), ref.cells_canon.view(np.uint32))


def test_unit_microbenchmarks(sim):
    """Every unit microbenchmark returns a positive rate within the pipe's
    plausible range (lanes per SM per clock at up to 2.1 GHz, 152 SMs)."""
    per_clk = 152 * 2.1e9
    limits = {fcs.MB_PHILOX: 8, fcs.MB_MULWIDE: 64, fcs.MB_LOP3: 128, fcs.MB_FFMA: 256, fcs.MB_MUFU: 32,
              fcs.MB_LDS: 64}
    for kind, lim in limits.items():
        r = fcs.fcs_microbench(kind, 0, 64)
        assert 0 < r < lim * per_clk, (kind, r)
    assert fcs.fcs_microbench(fcs.MB_RED, 1 << 20, 16) > 0
    assert fcs.fcs_microbench(fcs.MB_RED64, 1 << 20, 16) > 0
    with pytest.raises(fcs.FcsError):
        fcs.fcs_microbench(99, 0, 1)
