"""The multi-process parts of bench.py on CPU (gloo, two ranks on 127.0.0.1): the step time a
replicated run reports is the slowest rank's, and only rank 0 of the reference arm prints."""
import argparse
import contextlib
import io
import os
import socket

import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, values, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out.put((rank, bench.max_over_ranks_of(values[rank], world, "cpu")))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    values = [12.5, 30.25]
    mp.start_processes(_rank_main, args=(2, _free_port(), values, out), nprocs=2, start_method="spawn")
    got = dict(out.get() for _ in range(2))
    assert got == {0: 30.25, 1: 30.25}


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks_of(7.0, 1, "cpu") == 7.0


def test_reference_arm_prints_on_rank_0_only():
    args = argparse.Namespace(kappa=4, steps=1, warmup=0)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args, 1, 2)
    assert buf.getvalue() == ""
