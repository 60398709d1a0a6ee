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


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import oracle
    from paper_1904_08225_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    keys = _seeded_parts()

    def oracle_fn(ks, ids):
        return [oracle.greedy(k, oracle.start_index(len(k), seed=5, part_id=i), nthreads=1) for k, i in zip(ks, ids)]

    got = shard.order_sharded(keys, oracle_fn, world=world, rank=rank, dist=dist)
    mine = shard.shard([len(k) for k in keys], world, rank)
    q.put((rank, mine, None if got is None else [(p.tobytes(), r.tobytes()) for p, r in got]))
    dist.barrier()
    dist.destroy_process_group()


def _seeded_parts():
    import oracle
    g = np.random.default_rng(11)
    out = []
    for n in g.integers(50, 2500, size=23):
        pts = np.unique(g.integers(0, 1 << 16, size=(int(n) + 20, 3)), axis=0)[:int(n)]
        out.append(oracle.pack(pts))
    return out


def test_lpt_assignment():
    from paper_1904_08225_gb300 import shard
    sizes = [1000, 50, 50, 999, 400, 400, 10, 2000]
    a = shard.lpt_assign(sizes, 3)
    assert sorted(i for r in a for i in r) == list(range(len(sizes)))
    loads = [sum(shard.part_cost(sizes[i]) for i in r) for r in a]
    # LPT: the largest part alone first; every rank within the largest part's cost of the others
    assert a[0][0] == 7 or 7 in a[0]
    assert max(loads) - min(loads) <= shard.part_cost(2000)
    assert shard.lpt_assign(sizes, 1) == [list(range(len(sizes)))]
    assert shard.lpt_assign([], 4) == [[], [], [], []]
    with pytest.raises(ValueError):
        shard.shard(sizes, 2, 2)


def test_two_gloo_ranks_order_lpt_shards_and_gather():
    """Two gloo ranks each order their LPT shard of one seeded part set (the oracle as the
    ordering function, on CPU); rank 0's gathered results equal a single-rank run."""
    import oracle
    from paper_1904_08225_gb300 import shard
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, mine0, got0), (r1, mine1, got1) = out
    assert got1 is None and got0 is not None
    assert mine0 and mine1 and not set(mine0) & set(mine1)
    keys = _seeded_parts()
    assert sorted(mine0 + mine1) == list(range(len(keys)))
    single = shard.order_sharded(keys, lambda ks, ids: [oracle.greedy(k, oracle.start_index(len(k), seed=5, part_id=i),
                                                                       nthreads=1) for k, i in zip(ks, ids)])
    assert [(p.tobytes(), r.tobytes()) for p, r in single] == got0
