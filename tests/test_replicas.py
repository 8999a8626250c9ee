"""The multi-process (replica) path of bench.py on CPU with the gloo backend,
world size 2: every rank gets its own seeded workload, the job time is the
slowest rank's, the rate counts all ranks' cell-steps, and the reference arm
runs on rank 0 only."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    import bench
    ws_, rank_, _ = bench.dist_env()
    # each rank's own timing; the job's is the slowest
    mine = 10.0 + 5.0 * rank
    job_ms = bench.max_over_ranks(mine, ws_, "cpu")
    prob = bench.workload("kh512", rank_)
    rate = bench.job_rate(ws_, prob.ncells, 4, job_ms)

    class Args:
        steps, warmup = 1, 0

    ref = bench.run_reference(Args()) if rank_ != 0 else "skipped"
    digest = float(np.abs(prob.U).sum())
    out.put((rank_, ws_, job_ms, rate, digest, ref))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, t0, v0, d0, _), (r1, w1, t1, v1, d1, ref1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert t0 == t1 == 15.0                       # the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 512 * 512 * 4 / 0.015)
    assert d0 != d1                               # replicas run different seeds
    assert ref1 is None                           # the reference arm: rank 0 only
