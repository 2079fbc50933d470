"""The replica plumbing of bench.py at world size 2 over gloo on the host:
process group from the launcher's environment, barrier, the slowest rank's
time, the whole-job aggregate over ranks, and the reference arm, which runs
and prints on rank 0 alone."""
import argparse
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    os.environ["CUDA_VISIBLE_DEVICES"] = ""   # host plumbing only: gloo
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(WORLD), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_init(None)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    slowest = bench.max_over_ranks(1.0 + 0.5 * rank, w)   # rank 1 is the slower one
    value = bench.job_value(1000, 10, w, slowest)
    ref = bench.run_reference(argparse.Namespace(steps=1, warmup=0), r, w) if r != 0 else "rank 0"
    out[rank] = (r, w, local, slowest, value, ref)
    bench.barrier(w)
    dist.destroy_process_group()


def test_replicas_world_size_two_gloo():
    import torch.multiprocessing as mp
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(_free_port(), out), nprocs=WORLD, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, w, local, slowest, value, ref) in res.items():
        assert (r, w, local) == (rank, WORLD, rank)
        assert slowest == 1.5                              # max over ranks
        assert value == pytest.approx(1000 * 10 * WORLD / 1.5 / 1e6)   # all ranks' cells / slowest time
    assert res[1][5] is None                               # only rank 0 runs the reference arm
