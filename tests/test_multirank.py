"""The N > 1 path on CPU with gloo, world_size 2: ranks simulate contiguous
event ranges of one batch (the oracle stands in for each rank's GPU) and the
gathered cells equal the unsplit run; timing is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2103_14737_gb300.shard import max_over_ranks, shard_events  # noqa: E402


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
