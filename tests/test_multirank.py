"""The N > 1 path on CPU ranks (gloo, world size 2): every rank builds its own
seeded workload (weak scaling: per-rank work fixed), steps it with no
collective, and only the whole-job totals cross ranks (max time, summed
body-steps), as bench.py does under torchrun."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    import oracle
    import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)

    class A:
        episodes, tol, cap, fixed_iters = 3, 1e-5, 2000, 0
    scene, prot, prm = bench.workload(A, rank)
    s64 = synth.Scene(scene.body_off, *[getattr(scene, k).astype(np.float64) for k in
                                        ("half", "mass", "mu", "x", "q", "v", "w", "ground_mu")])
    w = oracle.World(s64, dict(prm, residual_tol=0.0, pgs_iters=5))
    w.set_protocol(prot)
    w.run_protocol(max_steps=4, threads=1)
    st = w.stats()
    body_steps = float(st["body_steps"].sum())
    fake_ms = 10.0 * (rank + 1)
    ms, wall, tot = bench.reduce_ranks(fake_ms, 0.5 + rank, body_steps, "cpu", dist)
    out.put((rank, float(scene.mass.sum()), body_steps, ms, wall, tot))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_collectives():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, b0, ms0, w0, t0), (r1, m1, b1, ms1, w1, t1) = res
    assert m0 != m1                      # different seeds per rank
    assert ms0 == ms1 == 20.0            # slowest rank's time
    assert w0 == w1 == 1.5
    assert t0 == t1 == b0 + b1           # body-steps of all ranks
