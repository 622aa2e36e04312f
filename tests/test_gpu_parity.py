"""GPU-vs-oracle parity of the CUDA path, called through the C ABI.

FP64 path: same inputs, same cycle count, max-abs difference <= 1e-10 on the
scalar field (relative to max|Phi| for the Newtonian potential).  Mixed
precision: relative L2 <= 1e-9 against the oracle's converged solution.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1307_6748_gb300 import synth

pytestmark = pytest.mark.gpu

L32, A1 = 64.0, 1.0


def _prob(model, N, box, a, **kw):
    return oracle.Problem(model, N, box, a=a, **kw)


def _model_setup(isis, model, N, box, a, par):
    """The library's model id and the initial guess both sides start from: the oracle's background field."""
    if model == oracle.SYMMETRON:
        return isis.ISIS_SYMMETRON, oracle.background_field(oracle.SYMMETRON, a, a_ssb=par.a_ssb)
    return isis.ISIS_FOFR_HS, oracle.background_field(oracle.FOFR, a, n=par.n, fR0_abs=par.fR0_abs)


@pytest.mark.parametrize("model", [oracle.SYMMETRON, oracle.FOFR])
@pytest.mark.parametrize("N,box", [(32, 64.0), (64, 128.0)])
def test_scalar_f64_fixed_cycles(cuda_lib, model, N, box):
    isis = cuda_lib
    par = isis.Params()
    eta = synth.lognormal_eta(N, box, 1.0, 1)
    m, g0 = _model_setup(isis, model, N, box, A1, par)
    ncyc = 3
    phi = torch.full((N,) * 3, g0, dtype=torch.float64, device="cuda")
    info = isis.isis_scalar_solve(m, par, isis.Grid(N, box), A1, eta.cuda(), phi, tol=0.0,
                                  opts=isis.Opts(max_cycles=ncyc), allow_noconv=True)
    ref = oracle.solve(_prob(model, N, box, A1), eta.numpy(), np.full((N,) * 3, g0), tol=0.0, max_cycles=ncyc)
    assert info.status == isis.ISIS_ENOCONV and ref.status == oracle.ENOCONV
    assert info.cycles == ref.cycles == ncyc
    err = np.abs(phi.cpu().numpy() - ref.phi).max()
    assert err <= 1e-10, err
    np.testing.assert_allclose(info.hist, ref.hist, rtol=1e-6)
    assert abs(info.res_ref - ref.ref) <= 1e-12 * ref.ref


@pytest.mark.parametrize("model", [oracle.SYMMETRON, oracle.FOFR])
def test_scalar_f64_converged_config1(cuda_lib, model):
    isis = cuda_lib
    N, box = 32, L32
    par = isis.Params()
    eta = synth.lognormal_eta(N, box, 1.0, 1)
    m, g0 = _model_setup(isis, model, N, box, A1, par)
    phi = torch.full((N,) * 3, g0, dtype=torch.float64, device="cuda")
    info = isis.isis_scalar_solve(m, par, isis.Grid(N, box), A1, eta.cuda(), phi, tol=1e-10)
    ref = oracle.solve(_prob(model, N, box, A1), eta.numpy(), np.full((N,) * 3, g0), tol=1e-10)
    assert ref.status == oracle.OK and info.status == isis.ISIS_OK
    assert info.cycles == ref.cycles
    assert np.abs(phi.cpu().numpy() - ref.phi).max() <= 1e-10
    if model == oracle.SYMMETRON:
        assert phi.min().item() >= -1e-12  # positive branch


@pytest.mark.parametrize("N,box", [(32, 64.0), (64, 64.0)])
def test_poisson_f64(cuda_lib, N, box):
    isis = cuda_lib
    eta = synth.lognormal_eta(N, box, 1.0, 1)
    Phi = torch.zeros((N,) * 3, dtype=torch.float64, device="cuda")
    info = isis.isis_poisson_solve(isis.Grid(N, box), A1, eta.cuda(), Phi, tol=1e-10)
    ref = oracle.solve(_prob(oracle.POISSON, N, box, A1), eta.numpy(), np.zeros((N,) * 3), tol=1e-10)
    assert ref.status == 0 and info.cycles == ref.cycles
    scale = np.abs(ref.phi).max()
    assert np.abs(Phi.cpu().numpy() - ref.phi).max() <= 1e-10 * scale
    assert abs(Phi.mean().item()) <= 1e-14 * scale


def test_poisson_sinusoid_exact(cuda_lib):
    """Discrete solution of a sinusoidal source: Phi = -KP delta / ((4/h^2) sin^2(pi m / N))."""
    isis = cuda_lib
    N, box, m = 64, 64.0, 3
    delta = synth.sinusoid(N, m=m, amp=0.5, axis=1)
    eta = 1.0 + delta
    Phi = torch.zeros((N,) * 3, dtype=torch.float64, device="cuda")
    isis.isis_poisson_solve(isis.Grid(N, box), A1, eta.cuda(), Phi, tol=1e-12)
    h = box / N
    KP = 1.5 * 0.267 * isis.H0_MPC ** 2 / A1
    exact = -KP * delta.numpy() / ((4.0 / h ** 2) * np.sin(np.pi * m / N) ** 2)
    assert np.abs(Phi.cpu().numpy() - exact).max() <= 1e-9 * np.abs(exact).max()


@pytest.mark.parametrize("fmg", [0, 1])
@pytest.mark.parametrize("model", [oracle.SYMMETRON, oracle.FOFR, oracle.POISSON])
def test_refine64_matches_oracle(cuda_lib, model, fmg):
    """FP32 correction cycles + FP64 defect correction vs the converged FP64 oracle, with and without the
    nested-iteration start of the FP32 phase."""
    isis = cuda_lib
    N, box = 64, 128.0
    par = isis.Params()
    eta = synth.lognormal_eta(N, box, 1.0, 1)
    opts = isis.Opts(prec=isis.ISIS_F32_REFINE64, fmg=fmg)
    if model == oracle.POISSON:
        phi = torch.zeros((N,) * 3, dtype=torch.float64, device="cuda")
        info = isis.isis_poisson_solve(isis.Grid(N, box), A1, eta.cuda(), phi, tol=1e-10, opts=opts)
        g0 = 0.0
    else:
        m, g0 = _model_setup(isis, model, N, box, A1, par)
        phi = torch.full((N,) * 3, g0, dtype=torch.float64, device="cuda")
        info = isis.isis_scalar_solve(m, par, isis.Grid(N, box), A1, eta.cuda(), phi, tol=1e-10, opts=opts)
    assert info.status == isis.ISIS_OK and info.res_final <= 1e-10 * info.res_ref
    # f(R) reaches its rounding floor near 1e-13 of the reference residual
    ref = oracle.solve(_prob(model, N, box, A1), eta.numpy(), np.full((N,) * 3, g0),
                       tol=1e-12 if model == oracle.FOFR else 1e-13)
    assert ref.status == 0
    got = phi.cpu().numpy()
    if model == oracle.FOFR:
        # relative L2 on delta f_R = f_R - fbar_R, f_R = -a^-2 e^u
        fr_g, fr_o = -np.exp(got), -np.exp(ref.phi)
        fbar = -np.exp(g0)
        rel = np.linalg.norm(fr_g - fr_o) / np.linalg.norm(fr_o - fbar)
        assert np.abs(got - ref.phi).max() <= 1e-8
    else:
        rel = np.linalg.norm(got - ref.phi) / np.linalg.norm(ref.phi)
    assert rel <= 1e-9, rel


@pytest.mark.parametrize("model", [oracle.SYMMETRON, oracle.FOFR])
def test_plain_f32(cuda_lib, model):
    isis = cuda_lib
    N, box = 32, 64.0
    par = isis.Params()
    eta = synth.lognormal_eta(N, box, 1.0, 1)
    m, g0 = _model_setup(isis, model, N, box, A1, par)
    phi = torch.full((N,) * 3, g0, dtype=torch.float32, device="cuda")
    # FP32 u ~ -11.5 carries ~5e-7 absolute rounding: the f(R) residual floors near 1e-4 of the reference
    tol = 1e-5 if model == oracle.SYMMETRON else 1e-3
    info = isis.isis_scalar_solve(m, par, isis.Grid(N, box), A1, eta.float().cuda(), phi, tol=tol,
                                  opts=isis.Opts(prec=isis.ISIS_F32))
    assert info.status == isis.ISIS_OK
    ref = oracle.solve(_prob(model, N, box, A1), eta.numpy(), np.full((N,) * 3, g0), tol=1e-12)
    err = np.abs(phi.double().cpu().numpy() - ref.phi).max()
    assert err <= 1e-4 * max(1.0, np.abs(ref.phi).max()), err


@pytest.mark.parametrize("N", [16, 64])
def test_cic_deposit(cuda_lib, N):
    isis = cuda_lib
    x, y, z = synth.zeldovich(N, float(N), seed=3)
    eta = torch.empty((N,) * 3, dtype=torch.float64, device="cuda")
    isis.isis_cic_deposit(isis.Grid(N, float(N)), x.cuda(), y.cuda(), z.cuda(), eta)
    ref = oracle.cic_deposit(N, x.numpy(), y.numpy(), z.numpy())
    assert np.abs(eta.cpu().numpy() - ref).max() <= 1e-10
    # deterministic: same bits twice
    eta2 = torch.empty_like(eta)
    isis.isis_cic_deposit(isis.Grid(N, float(N)), x.cuda(), y.cuda(), z.cuda(), eta2)
    assert torch.equal(eta, eta2)


def test_cic_lattice_uniform(cuda_lib):
    isis = cuda_lib
    N = 32
    q = (torch.arange(N, dtype=torch.float32) + 0.5)
    X, Y, Z = torch.meshgrid(q, q, q, indexing="ij")
    eta = torch.empty((N,) * 3, dtype=torch.float64, device="cuda")
    isis.isis_cic_deposit(isis.Grid(N, 32.0), X.reshape(-1).cuda(), Y.reshape(-1).cuda(), Z.reshape(-1).cuda(), eta)
    assert torch.all(eta == 1.0)


@pytest.mark.parametrize("model", [oracle.SYMMETRON, oracle.FOFR])
def test_fifth_force(cuda_lib, model):
    isis = cuda_lib
    N, box, a = 32, 64.0, 0.8
    par = isis.Params()
    gen = np.random.Generator(np.random.PCG64(7))
    Phi = gen.standard_normal((N,) * 3) * 1e-6
    if model == oracle.SYMMETRON:
        phi = 0.9 + 0.05 * gen.standard_normal((N,) * 3)
        m = isis.ISIS_SYMMETRON
    else:
        phi = -12.0 + 0.3 * gen.standard_normal((N,) * 3)
        m = isis.ISIS_FOFR_HS
    x, y, z = synth.zeldovich(N, box, seed=5)
    g = isis.isis_fifth_force(m, par, isis.Grid(N, box), a, torch.from_numpy(Phi).cuda(),
                              torch.from_numpy(phi).cuda(), x.cuda(), y.cuda(), z.cuda())
    go = oracle.fifth_force(_prob(model, N, box, a), Phi, phi, x.numpy(), y.numpy(), z.numpy())
    for gd, od in zip(g, go):
        np.testing.assert_allclose(gd.cpu().numpy(), od, rtol=2e-6, atol=2e-6 * np.abs(od).max())


def test_invalid_arguments(cuda_lib):
    isis = cuda_lib
    eta = torch.ones((12,) * 3, dtype=torch.float64, device="cuda")
    phi = torch.ones_like(eta)
    with pytest.raises(isis.IsisError) as e:
        isis.isis_scalar_solve(isis.ISIS_SYMMETRON, isis.Params(), isis.Grid(12, 10.0), 1.0, eta, phi)
    assert e.value.status == isis.ISIS_EINVAL
    eta = torch.ones((16,) * 3, dtype=torch.float64, device="cuda")
    phi = torch.ones_like(eta)
    with pytest.raises(isis.IsisError) as e:
        isis.isis_scalar_solve(isis.ISIS_SYMMETRON, isis.Params(lambda0=-1.0), isis.Grid(16, 10.0), 1.0, eta, phi)
    assert e.value.status == isis.ISIS_EINVAL


def test_nan_density_reports_enan(cuda_lib):
    isis = cuda_lib
    N = 16
    eta = torch.ones((N,) * 3, dtype=torch.float64)
    eta[3, 4, 5] = float("nan")
    phi = torch.full((N,) * 3, 0.9, dtype=torch.float64, device="cuda")
    with pytest.raises(isis.IsisError) as e:
        isis.isis_scalar_solve(isis.ISIS_SYMMETRON, isis.Params(), isis.Grid(N, 32.0), 1.0, eta.cuda(), phi)
    assert e.value.status == isis.ISIS_ENAN


def test_uniform_density_closed_form(cuda_lib):
    """Uniform eta: chi = sqrt(1 - (a_SSB/a)^3 eta); u from the f(R) background formula."""
    isis = cuda_lib
    N, box, a = 16, 32.0, 1.0
    for etav in (0.3, 1.0, 2.5):
        eta = torch.full((N,) * 3, etav, dtype=torch.float64, device="cuda")
        phi = torch.full((N,) * 3, 0.5, dtype=torch.float64, device="cuda")
        isis.isis_scalar_solve(isis.ISIS_SYMMETRON, isis.Params(), isis.Grid(N, box), a, eta, phi, tol=1e-12)
        exact = np.sqrt(max(0.0, 1.0 - 0.125 * etav))
        assert abs(phi.max().item() - exact) <= 1e-12 and abs(phi.min().item() - exact) <= 1e-12


# ---------------------------------------------------------------------------
# Larger grids (N >= 128): the two-cells-per-thread smoother, the tiled prolongation and the fused
# residual + restriction all run with many blocks per level.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("model", [oracle.SYMMETRON, oracle.FOFR, oracle.POISSON])
def test_f32_fixed_cycles_128(cuda_lib, model):
    """Plain FP32 cycles on 128^3 track the FP64 oracle's cycles to FP32 rounding."""
    isis = cuda_lib
    N, box = 128, 128.0
    par = isis.Params()
    eta = synth.lognormal_eta(N, box, 1.0, 1)
    ncyc = 2
    if model == oracle.POISSON:
        phi = torch.zeros((N,) * 3, dtype=torch.float32, device="cuda")
        isis.isis_poisson_solve(isis.Grid(N, box), A1, eta.float().cuda(), phi, tol=0.0,
                                opts=isis.Opts(prec=isis.ISIS_F32, max_cycles=ncyc), allow_noconv=True)
        g0 = 0.0
    else:
        m, g0 = _model_setup(isis, model, N, box, A1, par)
        phi = torch.full((N,) * 3, g0, dtype=torch.float32, device="cuda")
        isis.isis_scalar_solve(m, par, isis.Grid(N, box), A1, eta.float().cuda(), phi, tol=0.0,
                               opts=isis.Opts(prec=isis.ISIS_F32, max_cycles=ncyc), allow_noconv=True)
    ref = oracle.solve(_prob(model, N, box, A1), eta.numpy(), np.full((N,) * 3, g0), tol=0.0, max_cycles=ncyc)
    got = phi.double().cpu().numpy()
    if model == oracle.POISSON:
        err = np.abs(got - ref.phi).max() / np.abs(ref.phi).max()
        assert err <= 1e-5, err
    else:
        err = np.abs(got - ref.phi).max()
        # FP32: ulp(0.9) = 6e-8, ulp(11.5) = 1e-6, amplified by a few cycles
        assert err <= (2e-6 if model == oracle.SYMMETRON else 2e-5), err


@pytest.mark.parametrize("model,N,fmg", [(oracle.SYMMETRON, 128, 0), (oracle.FOFR, 128, 0), (oracle.POISSON, 128, 0),
                                         (oracle.SYMMETRON, 256, 0), (oracle.FOFR, 128, 1), (oracle.POISSON, 128, 1),
                                         (oracle.SYMMETRON, 256, 1)])
def test_refine64_large_matches_oracle(cuda_lib, model, N, fmg):
    isis = cuda_lib
    box = float(N)
    par = isis.Params()
    eta = synth.lognormal_eta(N, box, 1.0, 2)
    opts = isis.Opts(prec=isis.ISIS_F32_REFINE64, inner_cycles=3, fmg=fmg)
    if model == oracle.POISSON:
        phi = torch.zeros((N,) * 3, dtype=torch.float64, device="cuda")
        info = isis.isis_poisson_solve(isis.Grid(N, box), A1, eta.cuda(), phi, tol=1e-10, opts=opts)
        g0 = 0.0
    else:
        m, g0 = _model_setup(isis, model, N, box, A1, par)
        phi = torch.full((N,) * 3, g0, dtype=torch.float64, device="cuda")
        info = isis.isis_scalar_solve(m, par, isis.Grid(N, box), A1, eta.cuda(), phi, tol=1e-10, opts=opts)
    assert info.status == isis.ISIS_OK and info.res_final <= 1e-10 * info.res_ref
    ref = oracle.solve(_prob(model, N, box, A1), eta.numpy(), np.full((N,) * 3, g0),
                       tol=1e-12 if model == oracle.FOFR else 1e-13)
    assert ref.status == 0
    got = phi.cpu().numpy()
    if model == oracle.FOFR:
        fbar = -np.exp(g0)
        rel = np.linalg.norm(np.exp(got) - np.exp(ref.phi)) / np.linalg.norm(-np.exp(ref.phi) - fbar)
        assert np.abs(got - ref.phi).max() <= 1e-8
    else:
        rel = np.linalg.norm(got - ref.phi) / np.linalg.norm(ref.phi)
    assert rel <= 1e-9, rel


def _ff_pairs(n, seed):
    """Normalised float-float pairs (hi, lo) of random doubles over 60 decades, pairs whose exact sum needs more
    than 53 bits (remainders below, at and above half a double ulp, both signs), and pairs with lo = 0."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal(n) * 10.0 ** rng.uniform(-30, 30, n)
    hi = d.astype(np.float32)
    lo = (d - hi.astype(np.float64)).astype(np.float32)
    h2 = (rng.standard_normal(n) * 10.0 ** rng.uniform(-20, 20, n)).astype(np.float32)
    k = rng.integers(-4, 5, n).astype(np.float64)
    # lo = hi 2^-53 (1 + k 2^-20): around half an ulp of hi's FP64 value, k = 0 the exact tie
    l2 = (h2.astype(np.float64) * 2.0 ** -53 * (1.0 + k * 2.0 ** -20)).astype(np.float32)
    sgn = np.where(rng.random(n) < 0.5, -1.0, 1.0).astype(np.float32)
    l2 = l2 * sgn
    h3 = (rng.standard_normal(1000) * 1e3).astype(np.float32)
    hl = np.concatenate([np.stack([hi, lo], 1), np.stack([h2, l2], 1),
                         np.stack([h3, np.zeros_like(h3)], 1)]).astype(np.float32)
    keep = np.abs(hl[:, 1].astype(np.float64)) <= np.spacing(np.abs(hl[:, 0])).astype(np.float64) / 2
    return hl[keep]


def test_ff_to_f64_matches_one_fp64_addition(cuda_lib):
    """The integer FP64 write-back of a float-float value equals one FP64 addition of its two floats, bit for
    bit (round to nearest even, ties included), with subnormal low parts flushed as the library flushes them."""
    import torch
    from paper_1307_6748_gb300 import isis
    hl = _ff_pairs(400_000, 11)
    assert len(hl) > 700_000
    got = isis.selftest_ff_to_f64(torch.from_numpy(hl).cuda()).cpu().numpy()
    lo = hl[:, 1].astype(np.float64)
    lo = np.where(np.abs(lo) < 2.0 ** -126, 0.0, lo)
    want = hl[:, 0].astype(np.float64) + lo
    bad = got.view(np.int64) != want.view(np.int64)
    assert not bad.any(), (int(bad.sum()), hl[bad][:3], got[bad][:3], want[bad][:3])


def test_exp_ff_accuracy(cuda_lib):
    """The float-float exponential of the f(R) residual against CUDA's FP64 exp: relative error within
    the float-float rounding of its argument (about 2^-48 |x|) plus a few float-float ulps."""
    import torch
    from paper_1307_6748_gb300 import isis
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.cat([torch.linspace(-19.9, 19.9, 1_000_001, dtype=torch.float64, device="cuda"),
                   (torch.rand(200_000, generator=g, device="cuda", dtype=torch.float64) - 0.5) * 1e-3,
                   torch.arange(-1400, 1400, dtype=torch.float64, device="cuda") * (math.log(2.0) / 128.0)])
    y = isis.selftest_exp_ff(x)
    rel = ((y - torch.exp(x)) / torch.exp(x)).abs()
    bound = 4e-15 * x.abs() + 1e-14
    assert bool((rel <= bound).all()), float((rel / bound).max())
