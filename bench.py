#!/usr/bin/env python
"""Benchmark of the calorimeter hit path on GB300.

One step = one fcs_simulate_events call over a batch of 1024 pile-up events
(hard scatter + Poisson(200) minimum-bias collisions of Poisson(60) particles,
about 12.7M particles and 1.37e9 hits), i.e. every step of the hot path:
parametrisation lookup and Poisson hit counts, task records, the hit kernel
(Philox, inverse-CDF shape sampling, (r, alpha) -> (eta, phi), cell lookup,
warp-aggregated deposit), the FP64 recheck and the compaction of non-zero
cells.  Inputs are resident in HBM; the call is replayed as a CUDA graph; L2
is flushed (256 MB write) between timed steps.  The same JSON line carries
the paper's comparison (Sec. 4, GPU vs GPU_g): the same events as one launch
sequence per event (graph-replayed and eagerly launched) and, on a two-event
subset, one hit-kernel launch per task.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "simulated hits/s at 1 GB300 (batched; events/s and per-event launches alongside)"
UNIT = "hits/s"
WORKLOAD = "pileup1024"
N_EVENTS = 1024
PER_TASK_EVENTS = 2  # events 0 .. 1 of the batch: the per-task launch comparison (one launch per task)
SEED = 1
# ALU roofline of the hit kernel (the hit path's bound, per pipe):
#   time per hit = sum over pipes of (algorithmic ops per hit / pipe peak),
# with the algorithmic operation counts of one hit taken from the algorithm
# (not from compiled code) and each pipe's peak derived from its lanes per SM
# per clock x 152 SMs x 2070 MHz.  The lane counts are those the unit
# microbenchmarks show (fcs_microbench; bench.py reports them as measured).
OPS_PER_HIT = {
    # Philox4x32-10: 10 rounds x 2 (32 x 32 -> 64-bit) multiplies
    "mulwide": 20,
    # Philox 20 3-input XORs; bin 6; uniforms 4; region search 6; grid index 10;
    # deposit 4; task lookup 4
    "int": 54,
    # uniforms 2; (r, alpha) 2; sincos range 1; (eta, phi) 4; bounds 8;
    # scaled indices 4; certification compares 8
    "fp32": 29,
    # sin, cos
    "mufu": 2,
    # 32-bit shared-memory words read from the staged tables: the hit's region
    # (eta_lo, 1/deta, phi_lo, 1/dphi, n_eta, n_phi, cell offset), its r bin
    # (lo, width, hi) and alpha bin (lo, width); the per-task parameters are
    # per task, not per hit
    "lds": 12,
}
SMS, SM_MAX_MHZ = 152, 2070.0
# DRAM bytes per hit of the hit kernel, from the committed ncu summary of its
# 16-event capture (94.18 MB read + 4.50 MB written for 21,805,787 hits;
# traffic grows with the hits): valid for the kernel version captured there,
# None after a kernel change.
K_HITS_DRAM_BYTES_PER_HIT = 4.53
LANES_PER_SM_CLK = {"mulwide": 32, "int": 64, "fp32": 128, "mufu": 16, "lds": 32}


def alu_bound_hits_per_s():
    t = 0.0
    for k, n in OPS_PER_HIT.items():
        t += n / (LANES_PER_SM_CLK[k] * SMS * SM_MAX_MHZ * 1e6)
    return 1.0 / t


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _oracle_events(og, op, parts, events, threads):
    """Runs the oracle on whole events (event-parallel over host threads; the
    oracle is plain C called through ctypes, which releases the GIL).
    Returns the hits simulated."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle as O

    def one(e):
        return O.simulate(og, op, parts.event(e), seed=SEED, first_event=e, tasks=False, canon=False).n_hits

    if threads <= 1:
        return sum(one(e) for e in events)
    with ThreadPoolExecutor(threads) as ex:
        return sum(ex.map(one, events))


def cpu_baseline(geo, prm, parts, seconds=10.0):
    """The oracle as it stands on whole events of the same workload: one
    thread for about seconds / 3, then event-parallel on every host core for
    the rest (events taken round-robin from the batch)."""
    from oracle import oracle as O
    og, op = O.OracleGeometry(geo), O.OracleParams(prm)
    cores = os.cpu_count() or 1
    hits1, ev1, t0 = 0, 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds / 3:
        hits1 += _oracle_events(og, op, parts, [ev1 % parts.n_events], 1)
        ev1 += 1
    dt1 = time.perf_counter() - t0
    hitsN, evN, t0 = 0, 0, time.perf_counter()
    while time.perf_counter() - t0 < 2 * seconds / 3:
        batch = [(evN + k) % parts.n_events for k in range(cores)]
        hitsN += _oracle_events(og, op, parts, batch, cores)
        evN += cores
    dtN = time.perf_counter() - t0
    return {"value": hitsN / dtN, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{evN} whole events of pileup{parts.n_events} ({hitsN} hits, {dtN:.1f} s) event-parallel on {cores} "
                      f"threads",
            "events_per_s": evN / dtN,
            "single_thread": {"value": hits1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"{ev1} whole events ({hits1} hits, {dt1:.1f} s)"}}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle; each step simulates one whole pile-up
    event per host core, event-parallel."""
    from paper_2103_14737_gb300 import synth
    from oracle import oracle as O
    if rank != 0:
        return
    geo = synth.geometry()
    prm = synth.params(geo)
    cores = os.cpu_count() or 1
    # the batch's leading events (event k of a pile-up batch does not depend on the batch size)
    parts = synth.pileup(seed=SEED, n_events=min(args.events, (args.warmup + args.steps) * cores))
    og, op = O.OracleGeometry(geo), O.OracleParams(prm)
    hits = 0
    times = []
    for k in range(args.warmup + args.steps):
        batch = [(k * cores + j) % parts.n_events for j in range(cores)]
        t0 = time.perf_counter()
        h = _oracle_events(og, op, parts, batch, cores)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            hits += h
    tot = sum(times)
    v = hits / tot
    workload = f"pileup{args.events}"
    sample = f"{cores} whole events of {workload} per step, event-parallel on {cores} threads"
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """--sweep: the 1024-event pile-up batch (about 1.5e9 hits) swept over event
    waves, hit-kernel launch shapes, atomic vs deterministic accumulation and
    multiplicity bucketing; plus the launch latency of a one-particle call
    eagerly and as a graph, and per-event vs batched launches.  One JSON line."""
    import torch
    from paper_2103_14737_gb300 import fcs, synth
    n_ev = args.sweep_events
    geo = synth.geometry()
    prm = synth.params(geo)
    parts = synth.pileup(seed=SEED, n_events=n_ev)
    sim = fcs.Simulator(geo, prm)
    d = sim.to_device(parts)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {"mode": "sweep", "workload": f"pileup{n_ev}", "events": n_ev, "particles": parts.n,
           "l2": "flushed between steps (256 MB write)", "timing": "CUDA events, graph replay, mean of K steps"}

    def t_call(dd, K=5, W=3, **kw):
        r = sim.simulate(dd, SEED, outputs=dict(cells=None), **kw)  # sizes the workspace (not timed)
        for _ in range(W):
            sim.simulate(dd, SEED, sync=0, use_graph=1, outputs=dict(cells=None), **kw)
        st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        for k in range(K):
            flush.zero_()
            st[k].record()
            sim.simulate(dd, SEED, sync=0, use_graph=1, outputs=dict(cells=None), **kw)
            en[k].record()
        torch.cuda.synchronize()
        rc, stt = fcs.fcs_workspace_status(sim.ws)
        assert rc == 0, (rc, stt.as_dict())
        ms = float(np.mean([a.elapsed_time(b) for a, b in zip(st, en)]))
        return ms, r["stats"]["n_hits"]

    clk = ClockSampler(0)
    clk.start()
    # event waves (atomic mode, default launch shape)
    waves = {}
    for w in (16, 32, 64, 128, 256, 512, 0):
        ms, H = t_call(d, wave_events=w)
        waves[str(w or n_ev)] = {"ms": ms, "hits_per_s": H / (ms * 1e-3)}
    out["hits"] = H
    best_w = int(max(waves, key=lambda k: waves[k]["hits_per_s"]))
    out["waves_atomic"] = waves
    out["best_wave"] = best_w
    # launch shapes at the best wave
    b, h, table = sim.autotune(d, SEED, reps=3, wave_events=best_w)
    out["shapes_hits_ms_at_best_wave"] = {f"{k[0]}x{k[1]}": v for k, v in table.items()}
    out["best_shape"] = f"{b}x{h}"
    ms, _ = t_call(d, wave_events=best_w, block=b, hits_per_thread=h)
    out["atomic"] = {"ms": ms, "hits_per_s": H / (ms * 1e-3), "events_per_s": n_ev / (ms * 1e-3)}
    det = {}
    for w in (64, 256):
        ms, _ = t_call(d, K=3, wave_events=w, block=b, hits_per_thread=h, mode=fcs.MODE_DETERMINISTIC)
        det[str(w)] = {"ms": ms, "hits_per_s": H / (ms * 1e-3)}
    out["deterministic"] = det
    # multiplicity bucketing: events in ascending particle count, so that a
    # wave holds events of similar size
    order = np.argsort(np.diff(parts.event_offsets), kind="stable")
    sp = synth.Particles(*[np.concatenate([getattr(parts.event(int(e)), k) for e in order])
                           for k in ("type", "E", "eta", "phi")],
                         np.concatenate([[0], np.cumsum(np.diff(parts.event_offsets)[order])]).astype(np.int64))
    ms, H2 = t_call(sim.to_device(sp), wave_events=best_w, block=b, hits_per_thread=h)
    out["bucketed"] = {"ms": ms, "hits_per_s": H2 / (ms * 1e-3), "hits": H2,
                       "note": "the same events sorted by multiplicity (different random streams per event number)"}
    out["clocks"] = clk.stop()
    # launch latency: one 65.5 GeV electron (about 20 tasks, 1.5k hits)
    one = sim.to_device(synth.single_particle(1))
    lat = {}
    for name, kw in (("eager", dict(sync=0, use_graph=0)), ("graph", dict(sync=0, use_graph=1)),
                     ("sync_call", dict(sync=1, use_graph=0))):
        sim.simulate(one, SEED, outputs=dict(cells=None))
        for _ in range(20):
            sim.simulate(one, SEED, outputs=dict(cells=None), **kw)
        torch.cuda.synchronize()
        host, dev = [], []
        for _ in range(200):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record()
            sim.simulate(one, SEED, outputs=dict(cells=None), check=False, **kw)
            e1.record()
            t1 = time.perf_counter()
            torch.cuda.synchronize()
            host.append((t1 - t0) * 1e6)
            dev.append(e0.elapsed_time(e1) * 1e3)
        lat[name] = {"host_us_median": float(np.median(host)), "device_us_median": float(np.median(dev))}
    n_launch = fcs.fcs_workspace_graph_kernels(sim.ws)
    lat["launches_per_call"] = n_launch
    lat["per_launch_us_eager_minus_graph"] = (lat["eager"]["device_us_median"] -
                                              lat["graph"]["device_us_median"]) / (n_launch - 1)
    out["latency_one_electron"] = lat
    # per-event vs batched launch sequences for 64 single-electron events
    many = sim.to_device(synth.single_particle(64))
    ms_b, Hm = t_call(many, K=10)
    ms_e, _ = t_call(many, K=10, batched=0)
    # per-task launches (the paper's non-grouped GPU mode): the call reads each
    # event's task list back and launches the hit kernel once per task, so it
    # is timed as a whole synchronous call
    for b_, h_ in ((128, 1), (256, 4)):
        sim.simulate(many, SEED, outputs=dict(cells=None), batched=2, block=b_, hits_per_thread=h_)
    torch.cuda.synchronize()
    tt = []
    for _ in range(5):
        t0 = time.perf_counter()
        sim.simulate(many, SEED, outputs=dict(cells=None), batched=2, block=128, hits_per_thread=1)
        torch.cuda.synchronize()
        tt.append(time.perf_counter() - t0)
    ms_t = 1e3 * float(np.median(tt))
    out["single_e65_x64"] = {"hits": Hm, "batched_ms": ms_b, "per_event_ms": ms_e, "per_task_ms": ms_t,
                             "tasks": int(sim.simulate(many, SEED, outputs=dict(cells=None))["stats"]["n_tasks"]),
                             "per_event_over_batched": ms_e / ms_b, "per_task_over_batched": ms_t / ms_b,
                             "per_task_shape": "128x1"}
    # one training step on 256 events: the forward call (graph replay) and the
    # adjoint for a fixed dL/dE_cell (dense float32 rows, 193 MB)
    n256 = min(256, n_ev)
    d256 = sim.to_device(synth.pileup(seed=SEED, n_events=n256))
    g256 = torch.randn((n256, geo.n_cells), generator=torch.Generator("cuda").manual_seed(5), device="cuda")
    gf = torch.zeros(sim.n_entries, dtype=torch.float32, device="cuda")
    gw = torch.zeros(sim.n_entries * 128, dtype=torch.float32, device="cuda")
    shape = dict(block=b, hits_per_thread=h)
    r256 = sim.simulate(d256, SEED, outputs=dict(cells=None), **shape)
    sim.backward(d256, SEED, g256, d_frac=gf, d_shape_w=gw, **shape)
    for _ in range(2):
        sim.simulate(d256, SEED, sync=0, use_graph=1, outputs=dict(cells=None), **shape)
        sim.backward(d256, SEED, g256, sync=0, d_frac=gf, d_shape_w=gw, **shape)
    torch.cuda.synchronize()
    tf, tb = [], []
    for _ in range(3):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        sim.simulate(d256, SEED, sync=0, use_graph=1, outputs=dict(cells=None), **shape)
        e1.record()
        sim.backward(d256, SEED, g256, sync=0, d_frac=gf, d_shape_w=gw, **shape)
        e2.record()
        torch.cuda.synchronize()
        tf.append(e0.elapsed_time(e1))
        tb.append(e1.elapsed_time(e2))
    rc, stt = fcs.fcs_workspace_status(sim.ws)
    assert rc == 0, (rc, stt.as_dict())
    H256 = r256["stats"]["n_hits"]
    out["forward_backward_256"] = {"events": n256, "hits": H256, "forward_ms": float(np.mean(tf)),
                                   "backward_ms": float(np.mean(tb)),
                                   "step_hits_per_s": H256 / ((np.mean(tf) + np.mean(tb)) * 1e-3)}
    print(json.dumps(out), flush=True)
    sim.close()


def per_event_and_per_task(sim, d, parts, first_event, H, ms_batched, shape, flush, steps):
    """The paper's comparison on GB300 (Sec. 4: the GPU path launched per
    particle and layer, GPU_g grouping many tasks per launch), timed like the
    headline: the same events as one launch sequence per event, replayed as
    a CUDA graph and launched eagerly from the host; and one hit-kernel launch
    per task on the first PER_TASK_EVENTS events, against the batched call on
    the same events.  Each mode gives the same cells (parity tests)."""
    import torch
    from paper_2103_14737_gb300 import fcs
    out = {}
    n_ev = parts.n_events
    K = max(3, min(10, steps // 10))
    kw = dict(first_event=first_event, outputs=dict(cells=None), **shape)

    def device_time(W, **extra):
        sizing = {k: v for k, v in extra.items() if k != "use_graph"}
        r = sim.simulate(d, SEED, **kw, **sizing)  # sizes the workspace (not timed)
        assert r["status"] == 0 and r["stats"]["n_hits"] == H
        for _ in range(W):
            sim.simulate(d, SEED, sync=0, **kw, **extra)
        st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        for k in range(K):
            flush.zero_()
            st[k].record()
            sim.simulate(d, SEED, sync=0, **kw, **extra)
            en[k].record()
        torch.cuda.synchronize()
        rc, stt = fcs.fcs_workspace_status(sim.ws)
        assert rc == 0, (rc, stt.as_dict())
        return float(np.mean([a.elapsed_time(b) for a, b in zip(st, en)]))

    ms_g = device_time(2, batched=0, use_graph=1)
    launches = fcs.fcs_workspace_graph_kernels(sim.ws)
    out["per_event_graph"] = {"events": n_ev, "ms_per_step": ms_g, "hits_per_s": H / (ms_g * 1e-3),
                              "launches_per_step": launches, "batched_speedup": ms_g / ms_batched,
                              "mode": "one launch sequence per event (batched = 0), the call replayed as a CUDA graph"}
    ms_e = device_time(1, batched=0, use_graph=0)
    out["per_event_eager"] = {"events": n_ev, "ms_per_step": ms_e, "hits_per_s": H / (ms_e * 1e-3),
                              "batched_speedup": ms_e / ms_batched,
                              "mode": "one launch sequence per event (batched = 0), kernels launched from the host "
                                      "as the paper's per-event GPU path"}
    # one hit-kernel launch per task: synchronous calls (the call reads each event's
    # task list back), timed on the host like the batched call on the same events
    sub = sim.to_device(parts.events(0, PER_TASK_EVENTS))

    def host_time(reps, **extra):
        kw2 = {**shape, **extra}
        r = sim.simulate(sub, SEED, first_event=first_event, outputs=dict(cells=None), **kw2)
        assert r["status"] == 0
        torch.cuda.synchronize()
        tt = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.simulate(sub, SEED, first_event=first_event, outputs=dict(cells=None), **kw2)
            torch.cuda.synchronize()
            tt.append(time.perf_counter() - t0)
        return 1e3 * float(np.median(tt)), r["stats"]

    ms_b, st_b = host_time(max(5, K))
    ms_t, st_t = host_time(3, batched=2, block=128, hits_per_thread=1)
    assert st_t["n_hits"] == st_b["n_hits"] and st_t["n_nonzero"] == st_b["n_nonzero"]
    out["per_task"] = {"events": PER_TASK_EVENTS, "subset": f"events 0-{PER_TASK_EVENTS - 1} of the batch",
                       "tasks": st_t["n_tasks"], "hits": st_t["n_hits"], "ms_per_call": ms_t,
                       "hits_per_s": st_t["n_hits"] / (ms_t * 1e-3), "batched_ms_per_call": ms_b,
                       "batched_hits_per_s": st_b["n_hits"] / (ms_b * 1e-3), "batched_speedup": ms_t / ms_b,
                       "mode": "one hit-kernel launch per task (batched = 2, 128 x 1), the paper's non-grouped GPU "
                               "mode; both calls synchronous, host wall time, median"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--hpt", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--extra", action="store_true", help="also time deterministic mode and per-event launches")
    ap.add_argument("--events", type=int, default=N_EVENTS, help="events per step (smaller cases for profiling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ab", action="store_true", help="skip the per-event and per-task launch comparison")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner")
    ap.add_argument("--sweep", action="store_true", help="the 1024-event sweep and launch latency table instead")
    ap.add_argument("--sweep-events", type=int, default=1024)
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.sweep:
        if rank == 0:
            run_sweep(args)
        return

    import torch
    import torch.distributed as dist
    from paper_2103_14737_gb300 import fcs, synth
    from paper_2103_14737_gb300.shard import max_over_ranks, shard_events

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    geo = synth.geometry()
    prm = synth.params(geo)
    # weak scaling: the job is world x n_ev events; rank r simulates its contiguous
    # share (random-stream events first_event ...), with no data-path collective
    n_ev = args.events
    first_event, n_mine = shard_events(n_ev * world, rank, world)
    assert n_mine == n_ev
    parts = synth.pileup(seed=SEED + rank, n_events=n_ev)
    sim = fcs.Simulator(geo, prm)
    d = sim.to_device(parts)
    # autotune the hit kernel's launch shape on this workload (not timed)
    tune = None
    if not args.hpt and not args.block and not args.no_tune:
        b, h, table = sim.autotune(d, SEED, first_event=first_event, reps=3)
        args.block, args.hpt = b, h
        tune = {"block": b, "hits_per_thread": h, "hits_ms": {f"{k[0]}x{k[1]}": v for k, v in table.items()}}
    # size the workspace and the outputs with one synchronous call
    ref = sim.simulate(d, SEED, first_event=first_event, hits_per_thread=args.hpt, block=args.block)
    H = ref["stats"]["n_hits"]
    nnz_ref = ref["stats"]["n_nonzero"]
    cap = nnz_ref + nnz_ref // 20 + 4096  # room for the other simulation seeds of --extra
    outs = dict(cell_ids=torch.empty(cap, dtype=torch.int32, device="cuda"),
                cell_E=torch.empty(cap, dtype=torch.float32, device="cuda"),
                event_offsets=torch.empty(n_ev + 1, dtype=torch.int64, device="cuda"), cells=None)
    ref_stats = ref["stats"]
    del ref
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(K, W, seed=SEED, **kw):
        # one synchronous call sizes the workspace for this mode (not timed)
        r = sim.simulate(d, seed, first_event=first_event, outputs=outs, **kw)
        timed.n_hits = r["stats"]["n_hits"]
        for _ in range(W):
            sim.simulate(d, seed, first_event=first_event, sync=0, use_graph=1, outputs=outs, timing=1, **kw)
        torch.cuda.synchronize()
        t_step, t_hit = [], []
        st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        for k in range(K):
            flush.zero_()
            st[k].record()
            sim.simulate(d, seed, first_event=first_event, sync=0, use_graph=1, outputs=outs, timing=1, **kw)
            en[k].record()
            t_hit.append(fcs.fcs_workspace_timings(sim.ws))  # waits for this step's stage events
        torch.cuda.synchronize()
        t_step = [s.elapsed_time(e) for s, e in zip(st, en)]
        rc, stt = fcs.fcs_workspace_status(sim.ws)
        assert rc == 0, (rc, stt.as_dict())
        return t_step, t_hit

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    wall0 = time.perf_counter()
    t_step, t_stage = timed(args.steps, args.warmup, hits_per_thread=args.hpt, block=args.block)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    # kernels of one step: the kernel nodes of the timed call's CUDA graph
    launches_per_step = fcs.fcs_workspace_graph_kernels(sim.ws)
    clocks = clk.stop()
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(float(np.mean(t_step)))
    value = H * world / (ms * 1e-3)

    hit_ms = float(np.mean([s["hits"] for s in t_stage]))
    stage_ms = {k: float(np.mean([s[k] for s in t_stage])) for k in fcs.STAGES}
    achieved = H / (hit_ms * 1e-3) / 1e9
    peak = alu_bound_hits_per_s() / 1e9
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G hits/s",
                "frac": achieved / peak,
                "traffic": (K_HITS_DRAM_BYTES_PER_HIT * H if K_HITS_DRAM_BYTES_PER_HIT else None),
                "traffic_note": "dram bytes per launch scaled by hits from the 16-event ncu capture",
                "kernel": "k_hits", "hits_per_launch": H,
                "kernel_ms": hit_ms, "ops_per_hit": OPS_PER_HIT, "lanes_per_sm_clk": LANES_PER_SM_CLK,
                "peak_note": "derived: sum over pipes of ops/hit / (lanes x 152 SMs x 2070 MHz)"}

    # the paper's comparison: per-event and per-task launches of the same events
    ab = None
    if rank == 0 and not args.no_ab:
        ab = per_event_and_per_task(sim, d, parts, first_event, H, ms, dict(hits_per_thread=args.hpt,
                                                                            block=args.block), flush, args.steps)

    extra = {}
    if args.extra and rank == 0:
        ts, tst = timed(max(5, args.steps // 2), 2, mode=fcs.MODE_DETERMINISTIC, hits_per_thread=args.hpt,
                        block=args.block)
        extra["deterministic"] = {"hits_per_s": H / (np.mean(ts) * 1e-3), "ms_per_step": float(np.mean(ts)),
                                  "stages_ms": {k: float(np.mean([s[k] for s in tst])) for k in fcs.STAGES}}
        # the adjoint (gradients of the layer fractions and shape weights) over the
        # same events, for a fixed dL/dE_cell (dense float32 rows, 48 MB)
        gcell = torch.randn((n_ev, geo.n_cells), generator=torch.Generator("cuda").manual_seed(3), device="cuda")
        gf = torch.zeros(sim.n_entries, dtype=torch.float32, device="cuda")
        gw = torch.zeros(sim.n_entries * 128, dtype=torch.float32, device="cuda")
        kw = dict(first_event=first_event, d_frac=gf, d_shape_w=gw, hits_per_thread=args.hpt, block=args.block)
        sim.backward(d, SEED, gcell, **kw)  # sizes the workspace (not timed)
        for _ in range(2):
            sim.backward(d, SEED, gcell, sync=0, **kw)
        Kb = max(5, args.steps // 2)
        st = [torch.cuda.Event(enable_timing=True) for _ in range(Kb)]
        en = [torch.cuda.Event(enable_timing=True) for _ in range(Kb)]
        for k in range(Kb):
            flush.zero_()
            st[k].record()
            sim.backward(d, SEED, gcell, sync=0, **kw)
            en[k].record()
        torch.cuda.synchronize()
        rc, stt = fcs.fcs_workspace_status(sim.ws)
        assert rc == 0, (rc, stt.as_dict())
        tb = float(np.mean([a.elapsed_time(b) for a, b in zip(st, en)]))
        extra["backward"] = {"hits_per_s": H / (tb * 1e-3), "ms_per_step": tb, "forward_ms_per_step": ms,
                             "outputs": "dL/dfrac and dL/dshape_w of all entries, FP32, accumulated"}
        # three more simulation seeds of the same events (the parametrisation keeps its seed)
        seeds = {}
        for sd in (2, 3, 4):
            ts, _ = timed(max(5, args.steps // 4), 2, seed=sd, hits_per_thread=args.hpt, block=args.block)
            seeds[str(sd)] = {"hits": timed.n_hits, "hits_per_s": timed.n_hits / (np.mean(ts) * 1e-3),
                              "ms_per_step": float(np.mean(ts))}
        extra["seeds"] = seeds
        # the 400-particle hard-scatter event alone, with the standard mean hit
        # energies (5-200 MeV) and with 0.5-20 MeV ("hi": ten times the hits)
        one = {}
        p1 = synth.ttbar_like(SEED, 1)
        for name, rng_mhe in (("ttbar400", (5.0, 200.0)), ("ttbar400_hi", (0.5, 20.0))):
            s1 = sim if name == "ttbar400" else fcs.Simulator(geo, synth.params(geo, mean_hit_range=rng_mhe))
            d1 = s1.to_device(p1)
            r1 = s1.simulate(d1, SEED, outputs=dict(cells=None), hits_per_thread=args.hpt, block=args.block)
            for _ in range(3):
                s1.simulate(d1, SEED, sync=0, use_graph=1, outputs=dict(cells=None), hits_per_thread=args.hpt,
                            block=args.block)
            Ko = 20
            st = [torch.cuda.Event(enable_timing=True) for _ in range(Ko)]
            en = [torch.cuda.Event(enable_timing=True) for _ in range(Ko)]
            for k in range(Ko):
                st[k].record()
                s1.simulate(d1, SEED, sync=0, use_graph=1, outputs=dict(cells=None), hits_per_thread=args.hpt,
                            block=args.block)
                en[k].record()
            torch.cuda.synchronize()
            t1 = float(np.median([a.elapsed_time(b) for a, b in zip(st, en)]))
            one[name] = {"hits": r1["stats"]["n_hits"], "ms_per_event": t1,
                         "hits_per_s": r1["stats"]["n_hits"] / (t1 * 1e-3), "mean_hit_E_MeV": list(rng_mhe)}
            if s1 is not sim:
                s1.close()
        extra["single_event"] = one

    # end to end through the host-buffer entry point (copies inside the timed region)
    e2e = None
    if rank == 0 and not args.no_e2e:
        pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(parts, k))).pin_memory().numpy()
               for k in ("type", "E", "eta", "phi", "event_offsets")}
        ids = torch.empty(cap, dtype=torch.int32).pin_memory().numpy()
        cE = torch.empty(cap, dtype=torch.float32).pin_memory().numpy()
        off = torch.empty(n_ev + 1, dtype=torch.int64).pin_memory().numpy()
        cfg = fcs.make_config(hits_per_thread=args.hpt, block=args.block)
        for _ in range(2):
            fcs.fcs_simulate_events_host(sim.geo, sim.prm, sim.ws, pin["type"], pin["E"], pin["eta"], pin["phi"],
                                         pin["event_offsets"], SEED, first_event, cfg, ids, cE, off)
        K = max(3, args.steps // 2)
        tt = []
        nnz = 0
        for _ in range(K):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, st = fcs.fcs_simulate_events_host(sim.geo, sim.prm, sim.ws, pin["type"], pin["E"], pin["eta"],
                                                  pin["phi"], pin["event_offsets"], SEED, first_event, cfg, ids, cE,
                                                  off)
            tt.append(time.perf_counter() - t0)
            nnz = st.n_nonzero
        h2d = parts.n * 16 + (n_ev + 1) * 8
        d2h = nnz * 8 + (n_ev + 1) * 8
        single = {"value": H / float(np.mean(tt)), "ms_per_step": 1e3 * float(np.mean(tt))}

        # A serving loop: two workspaces on two streams, each call enqueued without
        # waiting (config sync = 0).  Before a workspace is used again, its previous
        # call is waited for and its status and counts are read.  Every step still
        # copies its inputs in and writes its results into mapped host buffers inside
        # the timed region; one call's copies and results overlap the other's compute.
        ws2 = fcs.fcs_workspace_create()
        slots = []
        for ws_k in (sim.ws, ws2):
            slots.append((ws_k, torch.cuda.Stream(), torch.empty(cap, dtype=torch.int32).pin_memory().numpy(),
                          torch.empty(cap, dtype=torch.float32).pin_memory().numpy(),
                          torch.empty(n_ev + 1, dtype=torch.int64).pin_memory().numpy()))
        acfg = fcs.make_config(hits_per_thread=args.hpt, block=args.block, sync=0)

        def enqueue(sl):
            with torch.cuda.stream(sl[1]):
                fcs.fcs_simulate_events_host(sim.geo, sim.prm, sl[0], pin["type"], pin["E"], pin["eta"], pin["phi"],
                                             pin["event_offsets"], SEED, first_event, acfg, sl[2], sl[3], sl[4])

        def wait(sl):
            with torch.cuda.stream(sl[1]):
                rc, st = fcs.fcs_workspace_status(sl[0])
            if rc != fcs.FCS_OK or st.n_nonzero != nnz:
                raise RuntimeError(f"pipelined host call: status {rc}, {st.n_nonzero} cells (expected {nnz})")

        for _ in range(2):  # sizes the second workspace, captures both graphs
            for sl in slots:
                enqueue(sl)
                wait(sl)
        torch.cuda.synchronize()
        Kp = max(4, args.steps)
        t0 = time.perf_counter()
        for i in range(Kp):
            if i >= 2:
                wait(slots[i % 2])
            enqueue(slots[i % 2])
        for i in range(max(0, Kp - 2), Kp):
            wait(slots[i % 2])
        tp = (time.perf_counter() - t0) / Kp
        if not np.array_equal(slots[0][4], off) or not np.array_equal(slots[1][2][:nnz], ids[:nnz]):
            raise RuntimeError("pipelined host calls returned other cells than the synchronous call")
        fcs.fcs_workspace_free(ws2)
        e2e = {"value": H / tp, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1e3 * tp, "steps": Kp,
               "mode": "serving loop: two workspaces on two streams, asynchronous host-buffer calls, "
                       "a workspace's previous call waited for and its status read before reuse; "
                       "no L2 flush (the other workspace's step streams over 300 MB through L2)",
               "single_call": single}

    # unit throughputs on this GPU (roofline denominators), measured after the timed region
    pipes = None
    if rank == 0:
        acc_cells = n_ev * geo.n_cells
        pipes = {"philox_blocks_per_s": fcs.fcs_microbench(fcs.MB_PHILOX, 0, 256),
                 "mulwide_per_s": fcs.fcs_microbench(fcs.MB_MULWIDE, 0, 1024),
                 "lop3_steps_per_s": fcs.fcs_microbench(fcs.MB_LOP3, 0, 1024),
                 "ffma_per_s": fcs.fcs_microbench(fcs.MB_FFMA, 0, 1024),
                 "mufu_sin_per_s": fcs.fcs_microbench(fcs.MB_MUFU, 0, 1024),
                 "lds_words_per_s": fcs.fcs_microbench(fcs.MB_LDS, 0, 1024),
                 "red_f32_random_per_s": fcs.fcs_microbench(fcs.MB_RED, acc_cells, 64),
                 "red_f64_random_per_s": fcs.fcs_microbench(fcs.MB_RED64, acc_cells, 64),
                 "red_array_floats": acc_cells}
        # lanes per SM per clock the microbenchmarks reach at the sampled clock
        mhz = (clocks or {}).get("sm_mhz") or SM_MAX_MHZ
        per_clk = SMS * mhz * 1e6
        pipes["lanes_per_sm_clk_measured"] = {
            "mulwide": pipes["mulwide_per_s"] / per_clk, "int": 3 * pipes["lop3_steps_per_s"] / per_clk,
            "fp32": pipes["ffma_per_s"] / per_clk, "mufu": pipes["mufu_sin_per_s"] / per_clk,
            "lds": pipes["lds_words_per_s"] / per_clk}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(geo, prm, parts, args.cpu_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"pileup{n_ev}",
                           "events_per_step": n_ev, "particles_per_step": parts.n,
                           "hits_per_step": H, "tasks_per_step": ref_stats["n_tasks"],
                           "nonzero_cells_per_step": ref_stats["n_nonzero"],
                           "recheck_hits_per_step": ref_stats["n_recheck"],
                           "poisson_fp64_per_step": ref_stats["n_poisson_fp64"], "mode": "atomic",
                           "hit_kernel_shape": f"{args.block or 128}x{args.hpt or 8}",
                           "launch": "batched, CUDA graph", "l2": "flushed between steps (256 MB write)",
                           "parallelism": f"replicas x{world} (events sharded, no collective)"},
                "events_per_s": n_ev * world / (ms * 1e-3),
                "autotune": tune,
                "stages_ms": stage_ms,
                "batched_vs_per_event": ab,
                "roofline": roofline, "pipes": pipes, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches_per_step * args.steps, "wall_s": wall}
        line.update(extra)
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
