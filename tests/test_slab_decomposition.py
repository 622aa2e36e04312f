"""The partitioned solve equals the single-rank solve (CPU, gloo, world size 2).  tests/slab_fas.py runs the
oracle's FAS V-cycle on z-slabs with one ghost-plane exchange per colour pass, a residual sum over ranks and the
coarse levels gathered; the serial-vs-parallel agreement is the one Sect. 5.1 reports for eight MPI processes.
The same driver on one rank is first pinned to oracle.solve at a fixed cycle count."""
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import slab_fas
from paper_1307_6748_gb300 import synth

N, BOX, NCYC = 32, 64.0, 3
CASES = {"symmetron": (oracle.SYMMETRON, 0.8), "poisson": (oracle.POISSON, 1.0)}


def _problem(name):
    model, a = CASES[name]
    return oracle.Problem(model, N, BOX, a=a, a_ssb=0.5, lambda0=1.0)


def _inputs(name):
    eta = synth.lognormal_eta(N, BOX, 1.0, 4).numpy()
    model, a = CASES[name]
    g0 = oracle.background_field(model, a, a_ssb=0.5) if model == oracle.SYMMETRON else 0.0
    return eta, np.full((N,) * 3, g0)


def _run(name, comm):
    eta, phi0 = _inputs(name)
    s = slab_fas.SlabFAS(_problem(name), eta, phi0, comm)
    hist = [s.cycle() for _ in range(NCYC)]
    return s.field(), hist


@pytest.mark.parametrize("name", sorted(CASES))
def test_single_rank_driver_matches_the_oracle(name):
    """World size 1: the slab driver is the oracle's algorithm (same cycles, same residual history)."""
    phi, hist = _run(name, slab_fas.Comm())
    eta, phi0 = _inputs(name)
    ref = oracle.solve(_problem(name), eta, phi0, tol=0.0, max_cycles=NCYC)
    scale = max(1.0, float(np.abs(ref.phi).max())) if name == "symmetron" else float(np.abs(ref.phi).max())
    assert np.abs(phi - ref.phi).max() <= 1e-12 * scale
    np.testing.assert_allclose(hist, ref.hist, rtol=1e-9)


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, out_dir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        for name in sorted(CASES):
            phi, hist = _run(name, slab_fas.Comm())
            if rank == 0:
                np.save(f"{out_dir}/{name}_phi.npy", phi)
                np.save(f"{out_dir}/{name}_hist.npy", np.array(hist))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_slabs_equal_one(tmp_path):
    """Two ranks, each with half of the planes of the 32^3 and 16^3 levels (8^3 and 4^3 gathered): the field
    after three V(2,2) cycles equals the single-rank field to rounding (the sums over ranks change the order of
    the Poisson mean and of the residual norm only), and so does the residual history."""
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for name in sorted(CASES):
        one, hist1 = _run(name, slab_fas.Comm())
        two = np.load(tmp_path / f"{name}_phi.npy")
        hist2 = np.load(tmp_path / f"{name}_hist.npy")
        scale = float(np.abs(one).max())
        assert np.abs(two - one).max() <= 1e-14 * scale, (name, np.abs(two - one).max() / scale)
        np.testing.assert_allclose(hist2, hist1, rtol=1e-12)
