"""The multi-rank path of bench.py on CPU with gloo, world size 2: every rank runs its own
replica (seed 42 + rank) of a small oracle step, ranks meet at barriers, and the reported
time is the max over ranks while the value counts every rank's steps.  No data-path
collective exists: the only collective is the timing reduction."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    import oracle as O
    from paper_1311_2481_gb300 import inputs as I
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prm = O.Params(12, 2, 3, 1, 0.5, 50.0, 0.0, 2 * math.pi / 3.16, 1e-3)
    ops = O.Operators(prm)
    u0 = I.initial_state(ops.r, prm.M, prm.K, 1, prm.L_z, 0.5, 50.0, 0.0, kind="box", amp=1e-2,
                         seed=bench.replica_seed(rank), mbox=2, kbox=3)
    dist.barrier()
    st = O.run(ops, O.cold_state(u0), 3)
    my_ms = 10.0 * (rank + 1)                   # a per-rank timing to reduce
    mx = bench.max_over_ranks(dist, my_ms, "cpu")
    dist.barrier()
    q.put((rank, mx, bench.aggregate_value(world, 5, mx), float(np.abs(st.u).sum())))
    dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [20.0, 20.0]               # max over ranks
    assert out[0][2] == pytest.approx(2 * 5 / 0.020)         # all ranks' steps / slowest time
    assert out[0][3] != out[1][3]                            # different seeds: independent replicas
