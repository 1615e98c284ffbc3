"""Population sharding across ranks (gloo, world size 2, CPU): the merged fitness of the shards equals
the fitness of the whole population, for even, ragged and empty slices. The oracle stands in for the
per-rank evaluation, so this checks the split and the merge, not the kernels."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1909_11474_gb300 import inputs as I
from paper_1909_11474_gb300.shard import broadcast_population, gather_population_values, population_shard


def test_population_shard_partitions():
    for P in (0, 1, 2, 7, 200, 201):
        for ws in (1, 2, 3, 8):
            sl = [population_shard(P, ws, r) for r in range(ws)]
            assert sl[0][0] == 0 and sl[-1][1] == P
            assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
            sizes = [b - a for a, b in sl]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        population_shard(5, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, P, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import oracle
        w = I.workload_ga_batch(P=P, C=2)
        cs = w["configs"]
        Eh, Wh, Fh = oracle.evaluate_batch(cs, w["hidden"][None, :])
        t = I.with_targets(w, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0])
        # rank 0 breeds the population; the others receive it
        pop = torch.tensor(w["params"]) if rank == 0 else torch.zeros((P, 6), dtype=torch.float64)
        broadcast_population(pop, src=0)
        s0, s1 = population_shard(P, ws, rank)
        if s1 > s0:
            E, W, F = oracle.evaluate_batch(cs, pop[s0:s1].numpy())
            r = oracle.fitness_from_predictions(cs, t, E, W, F)
            local = torch.tensor(np.concatenate([r["Z"][:, None], r["Zq"]], axis=1))
        else:
            local = torch.zeros((0, 4), dtype=torch.float64)
        full = gather_population_values(local, P)
        q.put((rank, full.numpy(), pop.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("P", [4, 5, 1])
def test_sharded_fitness_equals_whole_population(P):
    import oracle
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, P, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = I.workload_ga_batch(P=P, C=2)
    cs = w["configs"]
    Eh, Wh, Fh = oracle.evaluate_batch(cs, w["hidden"][None, :])
    t = I.with_targets(w, Eh[0] / cs.natoms, Wh[0] / cs.natoms[:, None], Fh[0])
    E, W, F = oracle.evaluate_batch(cs, w["params"])
    r = oracle.fitness_from_predictions(cs, t, E, W, F)
    ref = np.concatenate([r["Z"][:, None], r["Zq"]], axis=1)
    for rank, full, pop in got:
        assert np.array_equal(pop, w["params"])
        assert full.shape == (P, 4)
        np.testing.assert_allclose(full, ref, rtol=1e-12, atol=0)
