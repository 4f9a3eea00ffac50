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


def test_generator_pair_count_and_precision_choice():
    """Host-side helpers: distinct qubit pairs carrying a weight-2 generator,
    and the training loop's choice of the low-order form."""
    import numpy as np
    import bench
    from paper_2501_04776_gb300 import inputs as I
    from paper_2501_04776_gb300 import train
    assert bench.generator_pairs(12, I.local_gates_packed(12)) == 66
    G = I.random_k_body(I.Rng(1), 3000, 130, [1, 2], 1)
    bits = I.unpack_bits(G, 130)
    pairs = {tuple(np.nonzero(r)[0]) for r in bits if r.sum() == 2}
    assert bench.generator_pairs(130, G) == len(pairs)
    assert train.choose_precision(I.local_gates_packed(20)) == "loworder_fp32"
    assert train.choose_precision(I.random_k_body(I.Rng(2), 50, 30, [1, 2, 3], 1)) == "split_bf16"


def test_parity_roofline_bytes():
    import bench
    kt = {"parity": {"total_ms": 2.0, "launches": 8, "avg_ms": 0.25}}
    r = bench.parity_roofline(kt, {"hbm_gbs": 6000.0}, 1000, 100_000, 10_000, 10_000, 2)
    # per call: P and P^T for A and Z (2 x 1e4 x 1563 words each) + the rows of A and Z
    assert r["bytes_per_step"] == 2 * 8 * (2 * 10_000 * 1563 * 2 + 20_000 * 16)
    assert abs(r["frac"] - r["achieved"] / 6000.0) < 1e-3
