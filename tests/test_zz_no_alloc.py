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
