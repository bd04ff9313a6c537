"""Multi-process (world size 2, gloo, CPU) check of the beam sharding: each rank
marches its share of a beam batch (with the CPU oracle: no GPU here) and the
gathered results equal the unsplit run; throughput aggregation takes the sum of
work over the slowest rank's time."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2306_15678_gb300 import shard


def test_partition_is_balanced_and_complete():
    sizes = [512, 1024, 2048, 512, 1024, 2048, 2048, 512]
    parts = shard.partition(sizes, 3)
    flat = sorted(b for p in parts for b in p)
    assert flat == list(range(len(sizes)))
    loads = [sum(sizes[b] ** 2 for b in p) for p in parts]
    assert max(loads) - min(loads) <= max(s ** 2 for s in sizes)
    assert shard.partition(sizes, 3) == parts  # deterministic
    assert shard.partition(sizes, 1) == [list(range(len(sizes)))]
    with pytest.raises(ValueError):
        shard.partition(sizes, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _cfgs():
    from paper_2306_15678_gb300 import configs
    out = []
    for b, n in enumerate([16, 32, 16, 32, 16]):
        cfg = configs.physics(n, 0.08 * n, 0.5, configs.ALL_TERMS)
        cfg["beam"] = dict(w0=0.01 * n, P=50 * configs.critical_power(), amp=0.05, ell_cells=2.0,
                           seed=50 + b, phase=0.1, phase_seed=60 + b)
        out.append(cfg)
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    from paper_2306_15678_gb300 import beams
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfgs = _cfgs()
    mine = shard.my_beams([c["n"] for c in cfgs], world, rank)
    res = {b: oracle.march(beams.make_field(cfgs[b]), cfgs[b], 6, record=False)[0] for b in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    work = float(sum(cfgs[b]["n"] ** 2 * 6 for b in mine))
    value, tmax = shard.aggregate(work, 10.0 * (rank + 1), dist)
    if rank == 0:
        allres = {}
        for g in gathered:
            allres.update(g)
        q.put((allres, value, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_unsplit_batch():
    import oracle
    from paper_2306_15678_gb300 import beams
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    allres, value, tmax = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    cfgs = _cfgs()
    assert sorted(allres) == list(range(len(cfgs)))
    for b, c in enumerate(cfgs):
        ref, _, _ = oracle.march(beams.make_field(c), c, 6, record=False)
        assert np.array_equal(allres[b], ref)
    total = sum(c["n"] ** 2 * 6 for c in cfgs)
    assert tmax == 20.0
    assert value == pytest.approx(total / 0.020)
