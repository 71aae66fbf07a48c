"""The multi-rank path on CPU: two gloo ranks, each with its own system (the benchmark's
weak-scaling layout), computed by the oracle; the ranks exchange only the step time (max) and
their unit counts (sum) through bench.aggregate."""
import multiprocessing as mp
import os
import socket
import time

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    import npf_synth as S
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sysm = S.config_small(seed=rank, orders=(2, 3))
        t0 = time.perf_counter()
        res = oracle.npf_orders(sysm, 3, p1_block=10)
        t = time.perf_counter() - t0 + 0.01 * rank   # ranks differ in time on purpose
        units = bench.entries_per_step(10, (2, 3))
        tmax, total = bench.aggregate(dist, t, units)
        q.put((rank, res, t, tmax, total, units))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        r, res, t, tmax, total, units = q.get(timeout=120)
        out[r] = (res, t, tmax, total, units)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import npf_synth as S
    import oracle
    ts = [out[r][1] for r in range(2)]
    for r in range(2):
        res, t, tmax, total, units = out[r]
        assert tmax == max(ts)                   # both ranks see the slowest rank's time
        assert total == 2 * units                # whole-job units
        ref = oracle.npf_orders(S.config_small(seed=r, orders=(2, 3)), 3, p1_block=10)
        np.testing.assert_array_equal(res, ref)  # each rank solved its own system
    assert not np.allclose(out[0][0], out[1][0])


def test_aggregate_single_process():
    import bench
    assert bench.aggregate(None, 1.5, 7) == (1.5, 7)
