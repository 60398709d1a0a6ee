"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1) each build their own
seeded batch (parts are independent, so the work shards with no data-path collective) and
the step time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_setup()
    specs = bench.rank_specs(16, seed=3, rank=r)
    ms = bench.max_over_ranks(10.0 + 5.0 * r, dist, torch.device("cpu"))
    total = torch.tensor([float(sum(sp.n_target for sp in specs))], dtype=torch.float64)
    dist.all_reduce(total)
    q.put((r, w, ms, [sp.seed for sp in specs], float(total.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_parts_and_take_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (r0, w0, ms0, seeds0, tot0), (r1, w1, ms1, seeds1, tot1) = out
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert ms0 == ms1 == 15.0                    # both ranks see the slowest rank's time
    assert not set(seeds0) & set(seeds1)         # disjoint parts per rank
    assert tot0 == tot1 > 0
