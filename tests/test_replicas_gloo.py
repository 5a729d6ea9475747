"""The multi-process path (replicas, one process per GPU) exercised with
two gloo ranks on the CPU: distinct instances per rank, the max-over-ranks
timing every rank agrees on, the whole-job throughput, and that two ranks
solving their own instances (with the oracle, on the CPU) need no exchange
of problem data."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1912_04263_gb300 import replicas  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import numpy as np
        import qpgen
        from oracle import admm
        seed = replicas.replica_seed(7, rank)
        qp = qpgen.random_qp(20, 60, seed)
        r = admm.solve(qp)
        elapsed = 1.0 + rank  # rank 1 is the slow one
        m = replicas.max_over_ranks(elapsed, dist)
        dist.barrier()
        out[rank] = (seed, r.status, float(r.obj), m,
                     replicas.job_throughput(1, world, m), float(np.sum(qp.q)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_timing_and_solve_distinct_instances():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] != res[1][0]                  # distinct seeds
    assert res[0][1] == res[1][1] == "solved"
    assert res[0][5] != res[1][5]                  # distinct problem data
    assert res[0][3] == res[1][3] == 2.0           # max over ranks
    assert res[0][4] == res[1][4] == pytest.approx(1.0)  # 2 solves / 2 s


def test_single_process_helpers():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(5, 4, 2.0) == 10.0
    with pytest.raises(ValueError):
        replicas.job_throughput(1, 1, 0.0)
