"""The benchmark batches against the oracle, in the launch configuration the
bench times: one batched call of 128 threads x 8 hits per thread, replayed as
a CUDA graph.

* 64 pile-up events: every event, cell by cell, in atomic mode and (bit-exact
  against the canonical fold) in deterministic mode.
* 1024 pile-up events (the bench step): sampled events cell by cell, and every
  event's energy total against the oracle's.

The oracle runs one event per host thread (plain C through ctypes, which
releases the GIL)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2103_14737_gb300 import fcs, synth  # noqa: E402
from parity import ATOL, RTOL  # noqa: E402

SEED = 1
SHAPE = dict(block=128, hits_per_thread=8)
THREADS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def sim(geo, prm):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = fcs.Simulator(geo, prm)
    yield s
    s.close()


def _bench_call(sim, parts):
    """A sizing call, then the graph-replayed call the bench times; returns the
    replay's compacted output on the host."""
    d = sim.to_device(parts)
    first = sim.simulate(d, SEED, **SHAPE)
    nnz = first["stats"]["n_nonzero"]
    outs = dict(cell_ids=torch.empty(nnz + 64, dtype=torch.int32, device="cuda"),
                cell_E=torch.empty(nnz + 64, dtype=torch.float32, device="cuda"),
                event_offsets=torch.empty(parts.n_events + 1, dtype=torch.int64, device="cuda"))
    sim.simulate(d, SEED, sync=0, use_graph=1, outputs=outs, **SHAPE)
    torch.cuda.synchronize()
    rc, st = fcs.fcs_workspace_status(sim.ws)
    assert rc == fcs.FCS_OK and st.n_nonzero == nnz and st.n_hits == first["stats"]["n_hits"]
    off = outs["event_offsets"].cpu().numpy()
    assert off[-1] == nnz
    return (outs["cell_ids"][:nnz].cpu().numpy(), outs["cell_E"][:nnz].cpu().numpy().astype(np.float64), off,
            st.n_hits)


def _oracle(ogeo, oprm, parts, events, keep):
    """Oracle cells of `events`: the FP64 row for those in `keep`, the row's
    total for the others."""
    def one(e):
        c = O.simulate(ogeo, oprm, parts.event(e), seed=SEED, first_event=e, tasks=False, canon=False).cells64[0]
        return e, (c if e in keep else None), float(c.sum())
    with ThreadPoolExecutor(THREADS) as ex:
        res = list(ex.map(one, events))
    return {e: c for e, c, _ in res if c is not None}, {e: s for e, _, s in res}


def _check_event(ids, E, off, e, ref, n_cells):
    a, b = off[e], off[e + 1]
    assert (np.diff(ids[a:b]) > 0).all()  # ascending cell ids within the event
    row = np.zeros(n_cells)
    row[ids[a:b]] = E[a:b]
    assert np.array_equal(row != 0, ref != 0), f"event {e}: hit cells differ"
    err = np.abs(row - ref)
    assert (err <= RTOL * np.abs(ref) + ATOL).all(), f"event {e}: max error {err.max()}"


def test_pileup64_every_event(sim, ogeo, oprm):
    parts = synth.workload("pileup64", seed=SEED)
    ids, E, off, _ = _bench_call(sim, parts)
    events = list(range(parts.n_events))
    rows, _ = _oracle(ogeo, oprm, parts, events, set(events))
    for e in events:
        _check_event(ids, E, off, e, rows[e], sim.n_cells)


def test_pileup64_deterministic_every_event(sim, ogeo, oprm):
    """Deterministic mode on the 64-event batch, replayed as a graph: every
    event's compacted cells bit-equal to the oracle's canonical fold (segments
    of every size class, the per-event task bases, the one-pass compaction)."""
    parts = synth.workload("pileup64", seed=SEED)
    d = sim.to_device(parts)
    first = sim.simulate(d, SEED, mode=fcs.MODE_DETERMINISTIC, **SHAPE)
    nnz = first["stats"]["n_nonzero"]
    outs = dict(cell_ids=torch.empty(nnz + 64, dtype=torch.int32, device="cuda"),
                cell_E=torch.empty(nnz + 64, dtype=torch.float32, device="cuda"),
                event_offsets=torch.empty(parts.n_events + 1, dtype=torch.int64, device="cuda"))
    sim.simulate(d, SEED, mode=fcs.MODE_DETERMINISTIC, sync=0, use_graph=1, outputs=outs, **SHAPE)
    torch.cuda.synchronize()
    rc, st = fcs.fcs_workspace_status(sim.ws)
    assert rc == fcs.FCS_OK and st.n_nonzero == nnz
    ids = outs["cell_ids"][:nnz].cpu().numpy()
    E = outs["cell_E"][:nnz].cpu().numpy()
    off = outs["event_offsets"].cpu().numpy()

    def one(e):
        r = O.simulate(ogeo, oprm, parts.event(e), seed=SEED, first_event=e, tasks=False, cells64=False)
        return e, r.cells_canon[0]

    with ThreadPoolExecutor(THREADS) as ex:
        ref = dict(ex.map(one, range(parts.n_events)))
    for e in range(parts.n_events):
        a, b = off[e], off[e + 1]
        row = np.zeros(sim.n_cells, dtype=np.float32)
        row[ids[a:b]] = E[a:b]
        assert np.array_equal(row.view(np.uint32), ref[e].view(np.uint32)), f"event {e}: cells differ"


def test_pileup1024_bench_step(sim, ogeo, oprm):
    """The 1024-event step: events 0, 1, 2, 255, 256, 511, 512, 767, 1022 and
    1023 and four random ones cell by cell; every event's total within 1e-6 of
    the oracle's FP64 total (each cell is one FP32 rounding off)."""
    parts = synth.pileup(seed=SEED, n_events=1024)
    ids, E, off, n_hits = _bench_call(sim, parts)
    assert n_hits > 1_000_000_000
    rng = np.random.default_rng(7)
    keep = {0, 1, 2, 255, 256, 511, 512, 767, 1022, 1023} | set(int(x) for x in rng.integers(3, 1022, 4))
    rows, totals = _oracle(ogeo, oprm, parts, range(parts.n_events), keep)
    for e in sorted(keep):
        _check_event(ids, E, off, e, rows[e], sim.n_cells)
    got_tot = np.bincount(np.repeat(np.arange(parts.n_events), np.diff(off)), weights=E, minlength=parts.n_events)
    want_tot = np.array([totals[e] for e in range(parts.n_events)])
    assert np.allclose(got_tot, want_tot, rtol=1e-6, atol=1e-3)
