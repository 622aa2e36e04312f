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


def test_reference_arm_line_has_the_contract_keys():
    """The reference arm (the oracle on the host cores) prints one JSON line with the contract's keys, on a
    tiny sample so that the test stays short."""
    import json
    args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0", "--sample-N", "16"])
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args, 0, 1)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is False
    assert line["config"]["workload"].startswith("force step")
    assert set(line["cpu_baseline"]) >= {"value", "unit", "cores", "kind", "sample"}
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
