"""The multi-GPU path is replicas with no data-path collective: two gloo
ranks on CPU own different cells and the whole-job rate is the sum of their
cells over the slowest rank's time."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import time

    import torch.distributed as dist

    import oracle
    from paper_2111_07436_gb300 import replicas, workloads as w
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = w.workload(2)
    wl.cell_seed = replicas.cell_seed(wl.cell_seed, rank)
    y0, env = wl.inputs(16 + 8 * rank)
    om = oracle.Mechanism(wl.json())
    t = time.perf_counter()
    y, st, _ = om.solve(y0, env, wl.dt, wl.rtol, wl.atol, threads=1)
    secs = time.perf_counter() - t + 0.05 * rank
    cells, tmax, rate = replicas.aggregate(len(y0), secs, dist)
    out[rank] = (y0[0].copy(), int((st == 0).sum()), cells, tmax, rate, secs, len(y0))
    dist.destroy_process_group()


def test_two_replicas_on_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    r0, r1 = out[0], out[1]
    assert not np.array_equal(r0[0], r1[0])  # different cells per rank
    assert r0[1] == r0[6] and r1[1] == r1[6]  # every cell solved
    assert r0[2] == r1[2] == r0[6] + r1[6]
    assert r0[3] == r1[3] == max(r0[5], r1[5])
    assert abs(r0[4] - (r0[6] + r1[6]) / max(r0[5], r1[5])) < 1e-9
