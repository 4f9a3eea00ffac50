"""bench.py's multi-process path on CPU: N replicas under a gloo process
group (world size 2) agree on the slowest replica's time, and the reference
arm's non-zero ranks exit without work."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks(10.0 + 3.5 * rank)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_gloo_world_2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        assert dict(out) == {0: 13.5, 1: 13.5}


def test_max_over_ranks_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(7.25) == 7.25


def test_reference_arm_other_ranks_do_no_work():
    import bench
    sys_argv = sys.argv
    try:
        sys.argv = ["bench.py", "--impl", "reference"]
        args = bench.parse()
    finally:
        sys.argv = sys_argv
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, rank=1, world=2)
    assert buf.getvalue() == ""
