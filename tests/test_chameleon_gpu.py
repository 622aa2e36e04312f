"""The chameleon (the chameleon equation of Sect. 6 as a free source, Sect. 2) on the GPU against the oracle,
through the C ABI: FP64 at fixed cycles and converged, the mixed path, the fifth force and a refinement patch.
The model runs on the f(R) kernels with its own constants, so these tests check the constants and the
dispatch; n = -1/2 is the Hu-Sawicki-equivalent exponent of Sect. 6's mapping."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1307_6748_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = [(1.0, 2.0), (-0.5, 7.5)]  # (n, lambda0 [Mpc/h])


def _setup(isis, n, lam, N, box, a=1.0, beta=0.8):
    eta = synth.lognormal_eta(N, box, 1.0, 1)
    p = oracle.Problem(oracle.CHAMELEON, N, box, a=a, lambda0=lam, beta=beta, cham_n=n)
    par = isis.Params(lambda0=lam, beta=beta, cham_n=n)
    g0 = oracle.background_field(oracle.CHAMELEON, a, cham_n=n)
    return eta, p, par, g0


@pytest.mark.parametrize("n,lam", CASES)
def test_chameleon_f64_fixed_and_converged(cuda_lib, n, lam):
    isis = cuda_lib
    N, box, a = 32, 64.0, 0.9
    eta, p, par, g0 = _setup(isis, n, lam, N, box, a)
    for tol, ncyc in ((0.0, 3), (1e-10, 100)):
        phi = torch.full((N,) * 3, g0, dtype=torch.float64, device="cuda")
        info = isis.isis_scalar_solve(isis.ISIS_CHAMELEON, par, isis.Grid(N, box), a, eta.cuda(), phi, tol=tol,
                                      opts=isis.Opts(max_cycles=ncyc), allow_noconv=True)
        ref = oracle.solve(p, eta.numpy(), np.full((N,) * 3, g0), tol=tol, max_cycles=ncyc)
        assert info.cycles == ref.cycles
        assert (info.status == isis.ISIS_OK) == (ref.status == oracle.OK)
        assert np.abs(phi.cpu().numpy() - ref.phi).max() <= 1e-10
        assert abs(info.res_ref - ref.ref) <= 1e-12 * ref.ref
    assert ref.status == oracle.OK


@pytest.mark.parametrize("n,lam", CASES)
def test_chameleon_mixed_precision(cuda_lib, n, lam):
    isis = cuda_lib
    N, box = 64, 128.0
    eta, p, par, g0 = _setup(isis, n, lam, N, box)
    phi = torch.full((N,) * 3, g0, dtype=torch.float64, device="cuda")
    info = isis.isis_scalar_solve(isis.ISIS_CHAMELEON, par, isis.Grid(N, box), 1.0, eta.cuda(), phi, tol=1e-10,
                                  opts=isis.Opts(prec=isis.ISIS_F32_REFINE64, inner_cycles=4))
    assert info.status == isis.ISIS_OK and info.res_final <= 1e-10 * info.res_ref
    ref = oracle.solve(p, eta.numpy(), np.full((N,) * 3, g0), tol=1e-12)
    assert ref.status == oracle.OK
    got = phi.cpu().numpy()
    # relative L2 on psi - psi_bg, psi = e^u
    rel = np.linalg.norm(np.exp(got) - np.exp(ref.phi)) / np.linalg.norm(np.exp(ref.phi) - math.exp(g0))
    assert rel <= 1e-9, rel


def test_chameleon_force_matches_oracle(cuda_lib):
    isis = cuda_lib
    N, box, a, n, lam, beta = 32, 64.0, 0.8, 1.0, 2.0, 0.8
    eta, p, par, g0 = _setup(isis, n, lam, N, box, a, beta)
    u = oracle.solve(p, eta.numpy(), np.full((N,) * 3, g0), tol=1e-10).phi
    Phi = oracle.solve(oracle.Problem(oracle.POISSON, N, box, a=a), eta.numpy(), np.zeros((N,) * 3), tol=1e-10).phi
    x, y, z = synth.zeldovich(N, box, seed=5)
    gx, gy, gz = isis.isis_fifth_force(isis.ISIS_CHAMELEON, par, isis.Grid(N, box), a,
                                       torch.from_numpy(Phi).cuda(), torch.from_numpy(u).cuda(), x.cuda(), y.cuda(),
                                       z.cuda())
    ref = oracle.fifth_force(p, Phi, u, x.numpy(), y.numpy(), z.numpy())
    for g, r in zip((gx, gy, gz), ref):
        g = g.cpu().double().numpy()
        assert np.linalg.norm(g - r) <= 2e-6 * np.linalg.norm(r)


def test_chameleon_patch_matches_oracle(cuda_lib):
    isis = cuda_lib
    N, box, a, n, lam = 32, 64.0, 1.0, 1.0, 2.0
    eta, p, par, g0 = _setup(isis, n, lam, N, box, a)
    e = eta.numpy()
    parent = oracle.solve(p, e, np.full((N,) * 3, g0), tol=1e-10).phi
    o, nb = (6, 8, 10), (12, 10, 12)
    box_eta = e[o[0]:o[0] + nb[0], o[1]:o[1] + nb[1], o[2]:o[2] + nb[2]]
    flags = (box_eta >= 1.0).astype(np.uint8)
    flags[0], flags[-1], flags[:, 0], flags[:, -1], flags[:, :, 0], flags[:, :, -1] = 0, 0, 0, 0, 0, 0
    eta_f = np.ascontiguousarray(synth.lognormal_eta(2 * N, box, 1.0, 9).numpy()[:2 * nb[0], :2 * nb[1], :2 * nb[2]])
    ro = oracle.patch_solve(p, oracle.Patch(nb, o, (N, N, N), True, level=1), parent, flags, eta_f, tol=1e-10,
                            max_cycles=60)
    assert ro.status == oracle.OK
    phi = torch.zeros(eta_f.shape, dtype=torch.float64, device="cuda")
    info = isis.isis_patch_scalar_solve(isis.ISIS_CHAMELEON, par, isis.Grid(N, box), a,
                                        isis.Patch(nb, o, (N, N, N), True, level=1), torch.from_numpy(parent).cuda(),
                                        torch.from_numpy(flags).cuda(), torch.from_numpy(eta_f).cuda(), phi,
                                        tol=1e-10, opts=isis.Opts(max_cycles=60, init=isis.ISIS_INIT_PARENT))
    assert info.status == isis.ISIS_OK and info.cycles == ro.cycles
    assert np.abs(phi.cpu().numpy() - ro.phi).max() <= 1e-10
