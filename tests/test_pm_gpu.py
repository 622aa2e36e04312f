"""Particle time stepping on the GPU (leapfrog of Sect. 4.1, Eqs. (leap_frog_1)-(leap_frog_3)) against the
FP64 oracle's leapfrog (oracle.pm_run) from the same seeded Zel'dovich particles, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_1307_6748_gb300 import synth

pytestmark = pytest.mark.gpu

A_STEPS = [0.9, 0.93, 0.96, 1.0]


def _ic(N, box, seed):
    x, y, z, vx, vy, vz = synth.zeldovich_ic(N, box, A_STEPS[0], seed=seed)
    return (x, y, z, vx, vy, vz)


def _periodic_dist(a, b, N):
    d = np.abs(a - b) % N
    return np.minimum(d, N - d)


@pytest.mark.parametrize("model,prec", [(None, "f64"), ("sym", "f64"), ("fofr", "f64"), ("sym", "refine"),
                                        ("fofr", "refine")])
def test_pm_matches_oracle(cuda_lib, model, prec):
    isis = cuda_lib
    from paper_1307_6748_gb300 import pm
    N, box = 32, 32.0
    ic = _ic(N, box, seed=11)
    om = {None: None, "sym": oracle.SYMMETRON, "fofr": oracle.FOFR}[model]
    gm = {None: None, "sym": isis.ISIS_SYMMETRON, "fofr": isis.ISIS_FOFR_HS}[model]
    pos = [t.double().numpy().copy() for t in ic[:3]]
    vel = [t.double().numpy().copy() for t in ic[3:]]
    pos, vel = oracle.pm_run(om, N, box, pos, vel, A_STEPS, tol=1e-11)
    x, y, z, vx, vy, vz = (t.cuda() for t in ic)
    p = isis.ISIS_F64 if prec == "f64" else isis.ISIS_F32_REFINE64
    run = pm.PM(isis.Grid(N, box), gm, isis.Params(), x, y, z, vx, vy, vz, prec=p,
                tol=1e-11 if prec == "f64" else 1e-9, ncoarse=4).run(A_STEPS)
    torch.cuda.synchronize()
    for info in run.infos:
        for v in info.values():
            assert v.res_final <= (1e-11 if prec == "f64" else 1e-9) * v.res_ref
    for d, (gx, ov) in enumerate(zip((run.x, run.y, run.z), pos)):
        assert _periodic_dist(gx.cpu().double().numpy(), ov, N).max() <= 2e-4, d
    for gv, ov in zip((run.vx, run.vy, run.vz), vel):
        g = gv.cpu().double().numpy()
        assert np.linalg.norm(g - ov) <= 1e-4 * np.linalg.norm(ov)
    # the particles did move: the check is not between two copies of the initial conditions
    moved = _periodic_dist(run.x.cpu().double().numpy(), ic[0].double().numpy(), N)
    assert moved.max() > 1e-2


def test_kick_drift_formula(cuda_lib):
    """The fused kernel against its formula: v += kick g / h; x += drift v; x wrapped into [0, N)."""
    isis = cuda_lib
    N, box, n = 16, 48.0, 100_003
    g = torch.Generator().manual_seed(2)
    x = (torch.rand(n, generator=g) * N).float()
    v = (torch.randn(n, generator=g) * 3.0).float()
    f = torch.randn(n, generator=g).float()
    xs = [x.clone().cuda() for _ in range(3)]
    vs = [v.clone().cuda() for _ in range(3)]
    fs = [f.clone().cuda() for _ in range(3)]
    kick, drift = 0.7, 1.9
    isis.isis_kick_drift(isis.Grid(N, box), *xs, *vs, fs, kick, drift)
    torch.cuda.synchronize()
    h = box / N
    vv = v.double() + kick * f.double() / h
    xx = (x.double() + drift * vv) % N
    np.testing.assert_allclose(vs[0].cpu().double().numpy(), vv.numpy(), rtol=2e-7, atol=1e-6)
    assert _periodic_dist(xs[0].cpu().double().numpy(), xx.numpy(), N).max() <= 1e-5
    assert float(xs[0].min()) >= 0.0 and float(xs[0].max()) < N
