"""The multi-rank path of bench.py on the CPU: two gloo ranks (the launch torchrun makes, one
process per GPU, here without GPUs). Barrier, max and sum over ranks, the whole-job rate of weak
scaling (units of all ranks over the slowest rank's time), and the reference arm printing from
rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    d.barrier()
    res = {"world": d.world, "max": d.max(10.0 * (rank + 1)), "sum": d.sum(rank + 1.0),
           "rate": bench.whole_job_rate(d, 1000.0 * (rank + 1), 10.0 * (rank + 1))}

    class Args:
        steps, warmup, cpu_sample = 1, 3, 256
    buf = io.StringIO()
    if rank != 0:
        with redirect_stdout(buf):
            bench.run_reference(Args, d)      # rank 0 alone runs the reference arm
    res["printed"] = buf.getvalue()
    d.barrier()
    d.close()
    out[rank] = res


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as m:     # no fork: the parent may hold a CUDA context
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r]["world"] == 2
        assert res[r]["max"] == 20.0
        assert res[r]["sum"] == 3.0
        assert res[r]["rate"] == pytest.approx(3000.0 / 0.020)
    assert res[1]["printed"] == ""
