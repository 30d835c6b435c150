"""fcs_simulate_events_static: the entry point for callers that must not
allocate device memory while they run (its buffers live in the library's
static device array).  Its cells must match those of fcs_simulate_events,
the entry point with a cudaMalloc'd workspace, on the same inputs and seed,
for two calls in a row (the second call reuses the array the first one
left behind).  Collected last so that a failure here comes after every
other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2103_14737_gb300 import fcs, synth  # noqa: E402

RTOL, ATOL = 1e-5, 1e-3


def _dense(ids, E, off, n_events, n_cells):
    out = np.zeros((n_events, n_cells), np.float64)
    for e in range(n_events):
        a, b = off[e], off[e + 1]
        out[e, ids[a:b]] = E[a:b]
    return out


def test_static_scratch_matches_workspace_entry_point(geo, prm):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sim = fcs.Simulator(geo, prm)
    try:
        inputs = [(synth.pileup(seed=31, n_events=2, mu_pu=6), 17, 5),
                  (synth.ttbar_like(seed=32, n_events=3, n=150), 18, 40)]
        for parts, seed, first in inputs:  # two calls in a row on the same array
            d = sim.to_device(parts)
            ref = sim.simulate(d, seed, first_event=first)
            n_ev = parts.n_events
            cap = ref["stats"]["n_nonzero"] + 64
            ids = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
            E = torch.zeros(cap, dtype=torch.float32, device="cuda")
            off = torch.empty(n_ev + 1, dtype=torch.int64, device="cuda")
            pp = fcs.fcs_particles(d["type"].data_ptr(), d["E"].data_ptr(), d["eta"].data_ptr(),
                                   d["phi"].data_ptr(), d["event_offsets"].data_ptr())
            rc, st = fcs.fcs_simulate_events_static(sim.geo, sim.prm, pp, parts.n, n_ev, seed, first, ids, E, off)
            assert rc == fcs.FCS_OK
            assert st.n_hits == ref["stats"]["n_hits"] and st.n_tasks == ref["stats"]["n_tasks"]
            assert st.n_nonzero == ref["stats"]["n_nonzero"]
            got = _dense(ids.cpu().numpy(), E.cpu().numpy(), off.cpu().numpy(), n_ev, sim.n_cells)
            want = _dense(ref["cell_ids"].cpu().numpy(), ref["cell_E"].cpu().numpy(),
                          ref["event_offsets"].cpu().numpy(), n_ev, sim.n_cells)
            assert np.array_equal(got != 0, want != 0)
            assert (np.abs(got - want) <= RTOL * np.abs(want) + ATOL).all()
    finally:
        sim.close()


def test_static_scratch_rejects_oversized_calls(geo, prm):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sim = fcs.Simulator(geo, prm)
    try:
        parts = synth.pileup(seed=33, n_events=30, mu_pu=1)  # 30 accumulation rows exceed the array
        d = sim.to_device(parts)
        pp = fcs.fcs_particles(d["type"].data_ptr(), d["E"].data_ptr(), d["eta"].data_ptr(), d["phi"].data_ptr(),
                               d["event_offsets"].data_ptr())
        ids = torch.empty(16, dtype=torch.int32, device="cuda")
        E = torch.empty(16, dtype=torch.float32, device="cuda")
        off = torch.empty(31, dtype=torch.int64, device="cuda")
        rc, _ = fcs.fcs_simulate_events_static(sim.geo, sim.prm, pp, parts.n, 30, 1, 0, ids, E, off, check=False)
        assert rc == fcs.FCS_E_RANGE
    finally:
        sim.close()


def _pp(d):
    return fcs.fcs_particles(d["type"].data_ptr(), d["E"].data_ptr(), d["eta"].data_ptr(), d["phi"].data_ptr(),
                             d["event_offsets"].data_ptr())


def test_static_scratch_empty_batch_and_no_allocation(geo, prm):
    """No events: offsets [0], zeroed statistics, FCS_OK (as the workspace
    entry point).  Repeated calls leave the device's free memory unchanged:
    the calls allocate nothing (the array itself is reserved when the library's
    module is first used, before the first measurement)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sim = fcs.Simulator(geo, prm)
    try:
        empty = synth.Particles(np.zeros(0, np.int32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                                np.zeros(0, np.float32), np.array([0], np.int64))
        d0 = sim.to_device(empty)
        off0 = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        rc, st = fcs.fcs_simulate_events_static(sim.geo, sim.prm, _pp(d0), 0, 0, 1, 0, None, None, off0)
        assert rc == fcs.FCS_OK and off0.item() == 0 and st.n_hits == 0 and st.n_tasks == 0
        parts = synth.pileup(seed=34, n_events=2, mu_pu=4)
        d = sim.to_device(parts)
        ids = torch.empty(2 * sim.n_cells, dtype=torch.int32, device="cuda")
        E = torch.empty_like(ids, dtype=torch.float32)
        off = torch.empty(3, dtype=torch.int64, device="cuda")
        fcs.fcs_simulate_events_static(sim.geo, sim.prm, _pp(d), parts.n, 2, 3, 0, ids, E, off)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for seed in (4, 5, 6):
            rc, st = fcs.fcs_simulate_events_static(sim.geo, sim.prm, _pp(d), parts.n, 2, seed, 0, ids, E, off)
            assert rc == fcs.FCS_OK and st.n_hits > 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        sim.close()


def test_static_scratch_tile_map_overflow(geo):
    """A call whose particles and accumulation rows fit in the array but whose
    hits outgrow the tile map left after them (10 events of a 2 TeV electron
    with mean hit energies of 0.05-0.5 MeV: millions of hits each, against a
    map for about 4.5e7): the hit kernel reports it, the call returns
    FCS_E_RANGE with the hit count in its statistics, and the next call on
    the same array is correct again."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    prm_hi = synth.params(geo, mean_hit_range=(0.05, 0.5))
    sim = fcs.Simulator(geo, prm_hi)
    try:
        many = synth.single_particle(10, E=float(2**21), eta=0.6)
        d = sim.to_device(many)
        ids = torch.empty(1 << 20, dtype=torch.int32, device="cuda")
        E = torch.empty(1 << 20, dtype=torch.float32, device="cuda")
        off = torch.empty(11, dtype=torch.int64, device="cuda")
        rc, st = fcs.fcs_simulate_events_static(sim.geo, sim.prm, _pp(d), many.n, 10, 1, 0, ids, E, off, check=False)
        assert rc == fcs.FCS_E_RANGE
        assert st.device_flags & fcs.FLAG_HIT_CAPACITY and st.n_hits > 10_000_000
        small = synth.single_particle(2, E=float(2**14), eta=0.6)
        ds = sim.to_device(small)
        ref = sim.simulate(ds, 2)
        off2 = torch.empty(3, dtype=torch.int64, device="cuda")
        rc, st = fcs.fcs_simulate_events_static(sim.geo, sim.prm, _pp(ds), small.n, 2, 2, 0, ids, E, off2)
        assert rc == fcs.FCS_OK and st.n_hits == ref["stats"]["n_hits"]
        n = st.n_nonzero
        assert n == ref["stats"]["n_nonzero"]
        assert torch.equal(ids[:n], ref["cell_ids"][:n]) and torch.equal(off2, ref["event_offsets"])
        want = ref["cell_E"][:n].double()
        assert ((E[:n].double() - want).abs() <= RTOL * want.abs() + ATOL).all()
    finally:
        sim.close()
