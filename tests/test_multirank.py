"""The N > 1 path on CPU with gloo, world_size 2: ranks simulate contiguous
event ranges of one batch (the oracle stands in for each rank's GPU) and the
gathered cells equal the unsplit run; timing is the maximum over ranks; the
adjoint's gradients, summed over ranks that each took an event range or a
seed, equal the gradient of the whole batch."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2103_14737_gb300.shard import allreduce_gradients, max_over_ranks, shard_events  # noqa: E402


def test_shard_events_partition():
    for n in (0, 1, 5, 64, 1023):
        for world in (1, 2, 3, 8):
            ranges = [shard_events(n, r, world) for r in range(world)]
            assert sum(c for _, c in ranges) == n
            assert ranges[0][0] == 0
            for (f0, c0), (f1, _) in zip(ranges, ranges[1:]):
                assert f0 + c0 == f1
            assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1
    with pytest.raises(ValueError):
        shard_events(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_2103_14737_gb300 import synth

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        geo = synth.geometry()
        prm = synth.params(geo)
        parts = synth.pileup(seed=5, n_events=5, mu_pu=4)
        first, count = shard_events(parts.n_events, rank, world)
        res = O.simulate(O.OracleGeometry(geo), O.OracleParams(prm), parts.events(first, first + count), seed=21,
                         first_event=first, tasks=False)
        cells = torch.from_numpy(np.ascontiguousarray(res.cells_canon))
        sizes = [None] * world
        dist.all_gather_object(sizes, cells.shape[0])
        # gloo all_gather needs equal shapes: pad to the largest shard
        m = max(sizes)
        padded = torch.zeros((m, cells.shape[1]), dtype=cells.dtype)
        padded[: cells.shape[0]] = cells
        gathered = [torch.zeros_like(padded) for _ in range(world)]
        dist.all_gather(gathered, padded)
        t = max_over_ranks(float(rank + 1) * 0.5)
        if rank == 0:
            full = torch.cat([g[:n] for g, n in zip(gathered, sizes)]).numpy()
            np.save(os.path.join(out_dir, "gathered.npy"), full)
            np.save(os.path.join(out_dir, "tmax.npy"), np.array([t]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_equal_single_run(tmp_path):
    import torch.multiprocessing as mp

    from oracle import oracle as O
    from paper_2103_14737_gb300 import synth

    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    geo = synth.geometry()
    prm = synth.params(geo)
    parts = synth.pileup(seed=5, n_events=5, mu_pu=4)
    single = O.simulate(O.OracleGeometry(geo), O.OracleParams(prm), parts, seed=21, tasks=False)
    gathered = np.load(tmp_path / "gathered.npy")
    assert np.array_equal(gathered.view(np.uint32), single.cells_canon.view(np.uint32))
    assert float(np.load(tmp_path / "tmax.npy")[0]) == 1.0


GRAD_SEEDS = (31, 32)


def _grad_worker(rank, world, port, out_dir):
    import torch.distributed as dist

    from oracle import oracle as O
    from paper_2103_14737_gb300 import synth

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        geo = synth.geometry()
        prm = synth.params(geo)
        og, op = O.OracleGeometry(geo), O.OracleParams(prm)
        parts = synth.ttbar_like(seed=4, n_events=5, n=60)
        g = np.random.default_rng(7).normal(size=(parts.n_events, geo.n_cells))
        # event shards: each rank the gradient of its event range
        first, count = shard_events(parts.n_events, rank, world)
        f, w = O.backward(og, op, parts.events(first, first + count), GRAD_SEEDS[0], g[first:first + count],
                          first_event=first)
        tf, tw = torch.from_numpy(f), torch.from_numpy(w)
        allreduce_gradients(tf, None, tw)
        # seed shards: each rank every event with its own seed
        f2, w2 = O.backward(og, op, parts, GRAD_SEEDS[rank], g)
        sf, sw = torch.from_numpy(f2), torch.from_numpy(w2)
        allreduce_gradients(sf, sw)
        np.savez(os.path.join(out_dir, f"grad{rank}.npz"), f=tf.numpy(), w=tw.numpy(), sf=sf.numpy(), sw=sw.numpy())
    finally:
        dist.destroy_process_group()


def test_two_ranks_gradient_allreduce(tmp_path):
    import torch.multiprocessing as mp

    from oracle import oracle as O
    from paper_2103_14737_gb300 import synth

    world = 2
    mp.spawn(_grad_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    geo = synth.geometry()
    prm = synth.params(geo)
    og, op = O.OracleGeometry(geo), O.OracleParams(prm)
    parts = synth.ttbar_like(seed=4, n_events=5, n=60)
    g = np.random.default_rng(7).normal(size=(parts.n_events, geo.n_cells))
    full_f, full_w = O.backward(og, op, parts, GRAD_SEEDS[0], g)
    seeds = [O.backward(og, op, parts, s, g) for s in GRAD_SEEDS]
    for r in range(world):
        d = np.load(tmp_path / f"grad{r}.npz")
        assert np.count_nonzero(full_f) > 100
        # event shards: the sum over ranks is the whole batch's gradient (FP64 sums in another order)
        np.testing.assert_allclose(d["f"], full_f, rtol=1e-12, atol=1e-12 * np.abs(full_f).max())
        np.testing.assert_allclose(d["w"], full_w, rtol=1e-12, atol=1e-12 * np.abs(full_w).max())
        assert np.array_equal(d["f"] != 0, full_f != 0)
        # seed shards: the sum of the two seeds' gradients
        np.testing.assert_allclose(d["sf"], seeds[0][0] + seeds[1][0], rtol=1e-12)
        np.testing.assert_allclose(d["sw"], seeds[0][1] + seeds[1][1], rtol=1e-12,
                                   atol=1e-12 * np.abs(seeds[0][1]).max())


def test_allreduce_without_group_is_identity():
    t = torch.arange(4.0)
    assert allreduce_gradients(t, None)[0] is t and torch.equal(t, torch.arange(4.0))
