"""bench.py's multi-rank host logic on CPU (gloo, world size 2): the max over ranks of a per-rank time, the
per-rank problem seeds of the replicas, and the reference arm printing on rank 0 only."""
import contextlib
import io
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r reports 10 + r ms: every rank must see the largest
        v = bench.max_over_ranks(10.0 + rank, dist, torch.device("cpu"))
        with open(f"{out_dir}/{rank}.txt", "w") as f:
            f.write(repr(v))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [float((tmp_path / f"{r}.txt").read_text()) for r in range(world)]
    assert got == [11.0, 11.0]


def test_max_over_ranks_single_process():
    assert bench.max_over_ranks(7.5, None, torch.device("cpu")) == 7.5


def test_replicas_solve_their_own_problems():
    seeds = [bench.replica_seed(r) for r in range(8)]
    assert len(set(seeds)) == 8 and seeds[0] == 3


def test_reference_arm_prints_on_rank_0_only():
    args = bench.parse(["--impl", "reference", "--gpus", "2"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args, 1, 2)
    assert buf.getvalue() == ""
