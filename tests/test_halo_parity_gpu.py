"""GPU-vs-oracle parity on the high-contrast density of the halo workload: a lognormal field with sigma = 1.5
plus 32 seeded NFW haloes (masses 1e13-1e15 Msun/h, c = 5), cell-averaged on 1 Mpc/h cells, so that eta peaks
near 1e3-1e4.  This is the regime the lognormal sigma = 1 cases never reach:
- the symmetron near its symmetry-breaking point (Sect. 4.1): at a = 0.6, a_SSB = 0.5 the background is
  chi_bg = 0.649 and every cell with eta > (a/a_SSB)^3 = 1.73 is screened towards chi = 0;
- the f(R) field where b = e^u varies most (Sect. 3.4, the flux form with face means of e^u): inside a halo u
  falls by up to ~13 below its background.
FP64 path: the oracle's cycles, same inputs, same cycle count, max-abs <= 1e-10 (the domain tests' bar).
Mixed path (FP32 cycles in FP64 defect correction) on the 256^3 grid of a 256 Mpc/h box: relative L2 <= 1e-9
against the oracle converged to 1e-13 (symmetron) or 1e-12 (f(R), its FP64 floor), and max-abs <= 1e-8 on u.
Both sides start from one host-computed guess: the symmetron from the background chi_bg, f(R) from the
cell-wise uniform-density solution u(eta) (a background start overshoots without bound in the haloes)."""
import functools
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1307_6748_gb300 import synth

pytestmark = pytest.mark.gpu

SIGMA, SEED = 1.5, 1
OM, OL = 0.267, 0.733


@functools.lru_cache(maxsize=None)
def _eta(N):
    """The halo density on N^3 cells of 1 Mpc/h (box N Mpc/h)."""
    return synth.nfw_eta(N, float(N), SIGMA, SEED).numpy()


def _guess(model, eta, a, fR0=1e-5, n=1):
    """The initial field both sides start from."""
    if model == oracle.SYMMETRON:
        return np.full(eta.shape, oracle.background_field(oracle.SYMMETRON, a, a_ssb=0.5))
    r = OL / OM
    return np.log(a * a * fR0 * ((1 + 4 * r) / (eta * a ** -3 + 4 * r)) ** (n + 1))


def _gpu(isis, model, eta, phi0, a, N, tol, opts, allow_noconv=False):
    phi = torch.from_numpy(phi0.copy()).cuda()
    m = isis.ISIS_SYMMETRON if model == oracle.SYMMETRON else isis.ISIS_FOFR_HS
    info = isis.isis_scalar_solve(m, isis.Params(a_ssb=0.5), isis.Grid(N, float(N)), a,
                                  torch.from_numpy(eta).cuda(), phi, tol=tol, opts=opts, allow_noconv=allow_noconv)
    return phi.cpu().numpy(), info


CASES_F64 = [(oracle.SYMMETRON, N, a) for N in (64, 128) for a in (0.6, 0.8, 1.0)] + \
            [(oracle.FOFR, N, a) for N in (64, 128) for a in (0.6, 1.0)]


@pytest.mark.parametrize("model,N,a", CASES_F64)
def test_halo_f64_fixed_cycles(cuda_lib, model, N, a):
    isis = cuda_lib
    eta = _eta(N)
    g = _guess(model, eta, a)
    ncyc = 3
    got, info = _gpu(isis, model, eta, g, a, N, 0.0, isis.Opts(max_cycles=ncyc), allow_noconv=True)
    ref = oracle.solve(oracle.Problem(model, N, float(N), a=a), eta, g, tol=0.0, max_cycles=ncyc)
    assert info.status == isis.ISIS_ENOCONV and ref.status == oracle.ENOCONV
    assert info.cycles == ref.cycles == ncyc
    err = np.abs(got - ref.phi).max()
    assert err <= 1e-10, err
    np.testing.assert_allclose(info.hist, ref.hist, rtol=1e-6)
    assert abs(info.res_ref - ref.ref) <= 1e-12 * ref.ref


@pytest.mark.parametrize("model,a", [(oracle.SYMMETRON, 0.6), (oracle.SYMMETRON, 1.0), (oracle.FOFR, 1.0)])
def test_halo_f64_converged(cuda_lib, model, a):
    isis = cuda_lib
    N = 64
    eta = _eta(N)
    g = _guess(model, eta, a)
    got, info = _gpu(isis, model, eta, g, a, N, 1e-10, isis.Opts())
    ref = oracle.solve(oracle.Problem(model, N, float(N), a=a), eta, g, tol=1e-10)
    assert ref.status == oracle.OK and info.status == isis.ISIS_OK
    assert info.cycles == ref.cycles
    assert np.abs(got - ref.phi).max() <= 1e-10
    if model == oracle.SYMMETRON:
        assert got.min() >= -1e-12  # the positive branch


@functools.lru_cache(maxsize=None)
def _oracle_256(model, a):
    N = 256
    eta = _eta(N)
    r = oracle.solve(oracle.Problem(model, N, float(N), a=a), eta, _guess(model, eta, a),
                     tol=1e-12 if model == oracle.FOFR else 1e-13)
    assert r.status == oracle.OK, (r.status, r.res_final / r.ref)
    return r.phi


@pytest.mark.parametrize("model,a", [(oracle.SYMMETRON, 0.6), (oracle.SYMMETRON, 0.8), (oracle.SYMMETRON, 1.0),
                                     (oracle.FOFR, 1.0)])
def test_halo_refine64_256(cuda_lib, model, a):
    """The benchmark's cycle shape (V(2,1), nested-iteration start, coarsest 2^3) on the 256^3 halo density."""
    isis = cuda_lib
    N = 256
    eta = _eta(N)
    opts = isis.Opts(prec=isis.ISIS_F32_REFINE64, inner_cycles=4, fmg=1, nu1=2, nu2=1, n_coarsest=2)
    got, info = _gpu(isis, model, eta, _guess(model, eta, a), a, N, 1e-10, opts)
    assert info.status == isis.ISIS_OK and info.res_final <= 1e-10 * info.res_ref
    ref = _oracle_256(model, a)
    if model == oracle.FOFR:
        fbar = -a ** -2 * math.exp(oracle.background_field(oracle.FOFR, a, fR0_abs=1e-5))
        dfr_ref = -a ** -2 * np.exp(ref) - fbar
        rel = np.linalg.norm(-a ** -2 * np.exp(got) - fbar - dfr_ref) / np.linalg.norm(dfr_ref)
        assert np.abs(got - ref).max() <= 1e-8
    else:
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert got.min() >= -1e-12
    assert rel <= 1e-9, rel


def test_fofr_refine64_256_lognormal(cuda_lib):
    """f(R) on the 256^3 grid of a 256 Mpc/h box with the lognormal sigma = 1 density, |f_R0| = 1e-5, n = 1, in
    the benchmark's cycle shape, against the oracle converged to 1e-12: relative L2 <= 1e-9 on
    delta f_R = f_R - fbar_R and max-abs <= 1e-8 on u."""
    isis = cuda_lib
    N, a = 256, 1.0
    eta = synth.lognormal_eta(N, float(N), 1.0, 1).numpy()
    g = np.full(eta.shape, oracle.background_field(oracle.FOFR, a, fR0_abs=1e-5))
    opts = isis.Opts(prec=isis.ISIS_F32_REFINE64, inner_cycles=4, fmg=1, nu1=2, nu2=1, n_coarsest=2)
    got, info = _gpu(isis, oracle.FOFR, eta, g, a, N, 1e-10, opts)
    assert info.status == isis.ISIS_OK
    ref = oracle.solve(oracle.Problem(oracle.FOFR, N, float(N), a=a), eta, g, tol=1e-12)
    assert ref.status == oracle.OK
    fbar = -math.exp(g.flat[0])
    rel = np.linalg.norm(np.exp(got) - np.exp(ref.phi)) / np.linalg.norm(-np.exp(ref.phi) - fbar)
    assert np.abs(got - ref.phi).max() <= 1e-8
    assert rel <= 1e-9, rel
