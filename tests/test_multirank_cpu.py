"""Multi-rank path on CPU: subcarriers split across ranks with no data-path
collective (Section IV: subcarriers are independent), checked with two gloo
ranks; plus the partition itself."""
import os
import socket

import numpy as np
import pytest

from paper_1611_08779_gb300.shard import shard_range


@pytest.mark.parametrize("n", [0, 1, 7, 1200, 24001])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_ranges_partition_exactly(n, world):
    ranges = [shard_range(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_shard_range_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)
    with pytest.raises(ValueError):
        shard_range(-1, 0, 1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import oracle as orc
    from paper_1611_08779_gb300 import synth

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = synth.make_uplink(10, 16, 3, 4, 16, 10.0, seed=5)  # same batch on every rank
    a, b = shard_range(10, rank, world)
    z, L = orc.ocd_detect(d["H"][a:b], d["Y"][a:b], d["N0"], 1.0, 3, orc.BOX, 16)
    # results are gathered only to check them here; the detector itself
    # exchanges nothing between ranks
    zs = [None] * world
    dist.all_gather_object(zs, (a, b, z, L))
    # max-over-ranks timing as the benchmark reduces it
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((zs, float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_rank_result():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    import oracle as orc
    from paper_1611_08779_gb300 import synth

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    zs, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert tmax == 2.0
    d = synth.make_uplink(10, 16, 3, 4, 16, 10.0, seed=5)
    z_all, L_all = orc.ocd_detect(d["H"], d["Y"], d["N0"], 1.0, 3, orc.BOX, 16)
    z = np.concatenate([r[2] for r in sorted(zs, key=lambda r: r[0])])
    L = np.concatenate([r[3] for r in sorted(zs, key=lambda r: r[0])])
    assert np.array_equal(z, z_all) and np.array_equal(L, L_all)
