"""Pins of the FP64 CPU oracle to facts fixed outside it: the paper's printed
values, closed-form solutions, FFT-exact solutions of the discrete linear
problems, brute force and invariants.  No GPU.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1307_6748_gb300 import synth

H0 = oracle.H0_MPC
OM, OL = 0.267, 0.733
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def lap_eigen(N, h):
    """Eigenvalues of the periodic 7-point Laplacian on the rfft grid: -(4/h^2) sum_d sin^2(pi k_d / N)."""
    k = np.fft.fftfreq(N) * N
    kz = np.fft.rfftfreq(N) * N
    s = lambda q: np.sin(np.pi * q / N) ** 2
    return -(4.0 / h ** 2) * (s(k)[:, None, None] + s(k)[None, :, None] + s(kz)[None, None, :])


def fft_solve(rhs, lam_shift, h):
    """Solve (lap - lam_shift) f = rhs exactly with the discrete eigenvalues (zero mode dropped if singular)."""
    N = rhs.shape[0]
    lam = lap_eigen(N, h) - lam_shift
    R = np.fft.rfftn(rhs)
    F = np.zeros_like(R)
    nz = np.abs(lam) > 0
    F[nz] = R[nz] / lam[nz]
    return np.fft.irfftn(F, s=rhs.shape, axes=(0, 1, 2))


# ---------------------------------------------------------------------------
# Poisson (Sect. 3.1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m,axis", [(1, 0), (3, 2)])
def test_poisson_sinusoid_closed_form(m, axis):
    N, box, a = 32, 64.0, 0.7
    delta = synth.sinusoid(N, m=m, amp=0.3, axis=axis).numpy()
    r = oracle.solve(oracle.Problem(oracle.POISSON, N, box, a=a), 1.0 + delta, np.zeros((N,) * 3), tol=1e-12)
    assert r.status == oracle.OK
    h = box / N
    KP = 1.5 * OM * H0 ** 2 / a
    exact = -KP * delta / ((4.0 / h ** 2) * math.sin(math.pi * m / N) ** 2)
    assert np.abs(r.phi - exact).max() <= 1e-10 * np.abs(exact).max()


def test_poisson_fft_exact():
    N, box, a = 32, 64.0, 1.0
    eta = synth.lognormal_eta(N, box, 1.0, 11).numpy()
    r = oracle.solve(oracle.Problem(oracle.POISSON, N, box, a=a), eta, np.zeros((N,) * 3), tol=1e-12)
    assert r.status == oracle.OK
    KP = 1.5 * OM * H0 ** 2 / a
    exact = fft_solve(KP * (eta - eta.mean()), 0.0, box / N)
    assert np.abs(r.phi - exact).max() <= 1e-9 * np.abs(exact).max()
    assert abs(r.phi.mean()) <= 1e-13 * np.abs(exact).max()


# ---------------------------------------------------------------------------
# Uniform density: closed forms of the field equations
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("a,etav", [(1.0, 0.3), (1.0, 1.0), (0.8, 2.0), (0.6, 1.0), (1.0, 9.0)])
def test_symmetron_uniform_minimum(a, etav):
    """Sect. 4.1: uniform eta -> chi = sqrt(1 - (a_SSB/a)^3 eta) above symmetry breaking, else 0."""
    N, box = 8, 16.0
    r = oracle.solve(oracle.Problem(oracle.SYMMETRON, N, box, a=a, a_ssb=0.5), np.full((N,) * 3, etav),
                     np.full((N,) * 3, 0.7), tol=1e-13)
    v = 1.0 - (0.5 / a) ** 3 * etav
    exact = math.sqrt(v) if v > 0 else 0.0
    assert np.abs(r.phi - exact).max() <= 1e-12


@pytest.mark.parametrize("a,etav,fr0", [(1.0, 1.0, 1e-5), (0.7, 1.0, 1e-6), (1.0, 0.4, 1e-5), (0.8, 5.0, 1e-4)])
def test_fofr_uniform_background(a, etav, fr0):
    """Sect. 4.2: the f_R equation at uniform eta gives
    f_R = -|f_R0| [(1 + 4 OL/Om) / (eta a^-3 + 4 OL/Om)]^(n+1), and u = ln(-a^2 f_R)."""
    N, box = 8, 16.0
    rr = OL / OM
    fR = -fr0 * ((1 + 4 * rr) / (etav * a ** -3 + 4 * rr)) ** 2
    u_exact = math.log(-a * a * fR)
    r = oracle.solve(oracle.Problem(oracle.FOFR, N, box, a=a, fR0_abs=fr0), np.full((N,) * 3, etav),
                     np.full((N,) * 3, u_exact + 0.3), tol=1e-10)
    assert r.status == oracle.OK
    assert np.abs(r.phi - u_exact).max() <= 1e-10


def test_symmetron_zero_is_fixed_point():
    """chi = 0 solves the symmetron equation for any eta: a zero guess never moves."""
    N, box = 16, 32.0
    eta = synth.lognormal_eta(N, box, 1.0, 4).numpy()
    r = oracle.solve(oracle.Problem(oracle.SYMMETRON, N, box), eta, np.zeros((N,) * 3), tol=1e-10)
    assert r.status == oracle.OK and r.cycles == 0 and np.all(r.phi == 0.0)


# ---------------------------------------------------------------------------
# Linearised problems solved exactly by FFT
# ---------------------------------------------------------------------------

def test_symmetron_linearised_fft():
    """eta = 1 + eps nu: the first-order chi - chi_bg solves lap d = A(2 chi_bg^2 d + s chi_bg eps nu)."""
    N, box, a = 32, 32.0, 1.0
    nu = synth.gaussian_field(N, box, 1.0, 21).numpy()
    A, s = a * a / 2.0, (0.5 / a) ** 3
    chib = math.sqrt(1 - s)
    errs = []
    for eps in (1e-4, 1e-3):
        r = oracle.solve(oracle.Problem(oracle.SYMMETRON, N, box, a=a), 1.0 + eps * nu, np.full((N,) * 3, chib),
                         tol=1e-12)
        lin = fft_solve(A * s * chib * eps * nu, 2 * A * chib ** 2, box / N)
        errs.append(np.linalg.norm(r.phi - chib - lin) / np.linalg.norm(lin))
    assert errs[0] <= 5e-4
    assert 5.0 < errs[1] / errs[0] < 20.0  # the difference is second order in eps


def test_fofr_linearised_fft():
    """eta = 1 + eps nu: e^ubar lap d - (K3/(n+1)) d = K1 eps nu (flux form and source linearised)."""
    N, box, a, fr0 = 32, 64.0, 1.0, 1e-5
    nu = synth.gaussian_field(N, box, 1.0, 22).numpy()
    rr = OL / OM
    K1 = OM * a * H0 ** 2
    K3 = OM * a * H0 ** 2 * (1 + 4 * a ** 3 * rr)
    ubar = math.log(a * a * fr0 * ((1 + 4 * rr) / (a ** -3 + 4 * rr)) ** 2)
    errs = []
    for eps in (1e-4, 1e-3):
        r = oracle.solve(oracle.Problem(oracle.FOFR, N, box, a=a, fR0_abs=fr0), 1.0 + eps * nu,
                         np.full((N,) * 3, ubar), tol=1e-12)
        lin = fft_solve(K1 * eps * nu / math.exp(ubar), K3 / 2.0 / math.exp(ubar), box / N)
        errs.append(np.linalg.norm(r.phi - ubar - lin) / np.linalg.norm(lin))
    assert errs[0] <= 5e-4
    assert 5.0 < errs[1] / errs[0] < 20.0


# ---------------------------------------------------------------------------
# Operator structure
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("model", [oracle.POISSON, oracle.SYMMETRON, oracle.FOFR])
def test_diagonal_derivative_matches_finite_difference(model):
    """The Newton denominator dL_c/dphi_c equals a central difference of L_c in phi_c."""
    N, box = 8, 16.0
    gen = np.random.Generator(np.random.PCG64(5))
    eta = np.exp(gen.standard_normal((N,) * 3))
    phi = (0.8 + 0.1 * gen.standard_normal((N,) * 3)) if model != oracle.FOFR else \
        (-11.5 + 0.5 * gen.standard_normal((N,) * 3))
    p = oracle.Problem(model, N, box)
    d = oracle.dL(p, eta, phi)
    for c in [(0, 0, 0), (3, 5, 7), (7, 1, 2), (4, 4, 4)]:
        eps = 1e-5 * max(1.0, abs(phi[c]))
        pp, pm = phi.copy(), phi.copy()
        pp[c] += eps
        pm[c] -= eps
        fd = (oracle.residual(p, eta, pp)[c] - oracle.residual(p, eta, pm)[c]) / (2 * eps)
        assert abs(fd - d[c]) <= 1e-7 * abs(d[c])


def test_fofr_flux_is_conservative_and_second_order():
    """The flux form of Eq. (disc_non_canonical) sums to zero over the periodic box and approaches
    div(e^u grad u) = lap(e^u) at second order in h."""
    a, fr0 = 1.0, 1e-5
    rr = OL / OM
    K1, K2 = OM * a * H0 ** 2, OM * a ** 4 * H0 ** 2 * (1 + 4 * rr) * (fr0 * a * a) ** 0.5
    K3 = OM * a * H0 ** 2 * (1 + 4 * a ** 3 * rr)
    box = 10.0
    errs = []
    for N in (16, 32, 64):
        h = box / N
        x = (np.arange(N) + 0.5) * h
        X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
        kx = 2 * np.pi / box
        u = -11.0 + 0.4 * np.sin(kx * X) * np.cos(kx * Y) + 0.2 * np.sin(kx * Z)
        eta = np.ones((N,) * 3)
        S = K1 * (eta - 1) - K2 * np.exp(-u / 2) + K3
        flux = oracle.residual(oracle.Problem(oracle.FOFR, N, box, a=a, fR0_abs=fr0), eta, u) + S
        assert abs(flux.sum()) <= 1e-9 * np.abs(flux).sum()
        # analytic lap(e^u)
        ux = 0.4 * kx * np.cos(kx * X) * np.cos(kx * Y)
        uy = -0.4 * kx * np.sin(kx * X) * np.sin(kx * Y)
        uz = 0.2 * kx * np.cos(kx * Z)
        lapu = -0.8 * kx * kx * np.sin(kx * X) * np.cos(kx * Y) - 0.2 * kx * kx * np.sin(kx * Z)
        exact = np.exp(u) * (ux ** 2 + uy ** 2 + uz ** 2 + lapu)
        errs.append(np.abs(flux - exact).max())
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_restriction_and_prolongation():
    gen = np.random.Generator(np.random.PCG64(9))
    f = gen.standard_normal((8,) * 3)
    c = oracle.restrict(f)
    assert c.shape == (4,) * 3
    assert abs(c[1, 2, 3] - f[2:4, 4:6, 6:8].mean()) <= 1e-15
    assert abs(c.sum() * 8 - f.sum()) <= 1e-12
    # trilinear, cell centred: a coarse field linear in I gives i/2 - 1/4 at interior fine cells
    NH = 8
    I = np.arange(NH, dtype=float)
    cd = np.broadcast_to(I[:, None, None], (NH,) * 3).copy()
    fine = oracle.prolong_add(cd, np.zeros((2 * NH,) * 3))
    i = np.arange(2, 2 * NH - 2)
    np.testing.assert_allclose(fine[2:-2, 5, 7], i / 2 - 0.25, atol=1e-14)
    assert np.allclose(oracle.prolong_add(np.full((4,) * 3, 2.5), np.zeros((8,) * 3)), 2.5)


# ---------------------------------------------------------------------------
# FAS solution vs an independent dense Newton (brute force on 8^3)
# ---------------------------------------------------------------------------

def numpy_newton(p, eta, phi0, iters=30):
    """Newton on F(phi) = L(phi) with a central finite-difference Jacobian (512 unknowns)."""
    phi = phi0.copy()
    n = phi.size
    for _ in range(iters):
        F = oracle.residual(p, eta, phi).ravel()
        J = np.empty((n, n))
        for q in range(n):
            e = 1e-6 * max(1.0, abs(phi.flat[q]))
            pp = phi.copy()
            pp.flat[q] += e
            pm = phi.copy()
            pm.flat[q] -= e
            J[:, q] = (oracle.residual(p, eta, pp).ravel() - oracle.residual(p, eta, pm).ravel()) / (2 * e)
        dx = np.linalg.solve(J, -F)
        phi = phi + dx.reshape(phi.shape)
        if np.abs(dx).max() <= 1e-14 * max(1.0, np.abs(phi).max()):
            break
    return phi


@pytest.mark.parametrize("model,ncoarse", [(oracle.SYMMETRON, 4), (oracle.SYMMETRON, 2), (oracle.FOFR, 4),
                                           (oracle.CHAMELEON, 4)])
def test_fas_matches_dense_newton_8cubed(model, ncoarse):
    """The FAS fixed point and the oracle's own dense Newton solve (the coarsest-level solver run on the whole
    8^3 grid) both equal a numpy Newton solve with a finite-difference Jacobian.  The dense Newton solve,
    started from the background field, converges quadratically (exact Jacobian): it meets its stop rule
    (max|dx| <= 1e-13 max(1, max|phi|)) within 8 steps, where a Jacobian off by a few per cent converges only
    linearly and needs more."""
    N, box = 8, 16.0 if model in (oracle.SYMMETRON, oracle.CHAMELEON) else 64.0
    eta = synth.lognormal_eta(N, box, 1.0, 13).numpy()
    p = oracle.Problem(model, N, box, a=0.9, lambda0=1.5, cham_n=1.0)
    g0 = math.sqrt(1 - (0.5 / 0.9) ** 3) if model == oracle.SYMMETRON else \
        math.log(0.81 * 1e-5 * ((1 + 4 * OL / OM) / (0.9 ** -3 + 4 * OL / OM)) ** 2) if model == oracle.FOFR else \
        3.0 * math.log(0.9) / 2.0  # chameleon n = 1: u = 3 ln(a) / (1 + n) at eta = 1
    guess = np.full((N,) * 3, g0)
    ref = numpy_newton(p, eta, guess)
    r = oracle.solve(p, eta, guess, tol=1e-12, ncoarse=ncoarse)
    assert r.status == oracle.OK
    assert np.abs(r.phi - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    st, dn, steps = oracle.dense_newton(p, eta, guess)
    assert st == oracle.OK and np.abs(dn - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    assert 2 <= steps <= 8, steps


def test_dense_newton_reports_no_convergence():
    """A Newton solve that does not meet its stop rule within its 50 steps reports ENOCONV, not OK.  On a
    uniform symmetron grid with eta = 0 the equation L(chi) = Sigma reads chi^3 - chi + Sigma/A = 0 in every
    cell, and for Sigma/A = 1/sqrt(2) Newton's method from chi = 0 cycles exactly between 0 and 1/sqrt(2)
    (N(0) = 1/sqrt(2), N(1/sqrt(2)) = 0; the cycle is superattracting, N'(0) = 0), so every step has
    max|dx| = 1/sqrt(2)."""
    N, box = 4, 4.0
    p = oracle.Problem(oracle.SYMMETRON, N, box, a=1.0, a_ssb=0.5, lambda0=1.0)
    A = 0.5  # a^2 / (2 lambda0^2)
    eta = np.zeros((N,) * 3)
    sigma = np.full((N,) * 3, A / math.sqrt(2.0))
    for start in (0.0, 0.3):
        st, phi, steps = oracle.dense_newton(p, eta, np.full((N,) * 3, start), sigma)
        assert st == oracle.ENOCONV and steps == 50, (st, steps)
        # 50 steps (even) end on the cycle's point reached from the start
        assert np.abs(phi - (0.0 if start == 0.0 else 1 / math.sqrt(2.0))).max() < 1e-12


@pytest.mark.parametrize("model", [oracle.POISSON, oracle.SYMMETRON, oracle.FOFR, oracle.CHAMELEON])
def test_jacobian_matches_finite_difference(model):
    """The coarsest solve's dense Jacobian (every entry, all 64 columns of a 4^3 grid) against a central
    difference of the residual L(phi) in each phi_c.  The f(R) and chameleon off-diagonal entries
    (b_f + (b_nb/2)(u_nb - u))/h^2 carry the face average's derivative of Sect. 3.4; Poisson's entries carry the
    shift -(6/h^2)/n that removes the constant null space of the periodic Laplacian."""
    N, box = 4, 8.0
    h = box / N
    gen = np.random.Generator(np.random.PCG64(17))
    eta = np.exp(0.5 * gen.standard_normal((N,) * 3))
    if model == oracle.FOFR:
        phi = -11.5 + 0.6 * gen.standard_normal((N,) * 3)
    elif model == oracle.CHAMELEON:
        phi = 0.4 * gen.standard_normal((N,) * 3)
    elif model == oracle.POISSON:
        phi = 1e-5 * gen.standard_normal((N,) * 3)
    else:
        phi = 0.8 + 0.2 * gen.standard_normal((N,) * 3)
    p = oracle.Problem(model, N, box, a=0.9, lambda0=1.5, cham_n=1.0)
    J = oracle.jacobian(p, eta, phi)
    n = N ** 3
    if model == oracle.POISSON:
        J = J + (6.0 / h ** 2) / n
    Jfd = np.empty((n, n))
    for q in range(n):
        e = 1e-5 * max(1.0, abs(phi.flat[q]))
        pp, pm = phi.copy(), phi.copy()
        pp.flat[q] += e
        pm.flat[q] -= e
        Jfd[:, q] = (oracle.residual(p, eta, pp).ravel() - oracle.residual(p, eta, pm).ravel()) / (2 * e)
    scale = np.abs(Jfd).max()
    assert np.abs(J - Jfd).max() <= 1e-8 * scale, np.abs(J - Jfd).max() / scale
    # the sparsity: the diagonal and the six neighbours of each row (4^3: all distinct)
    assert np.count_nonzero(np.abs(Jfd) > 1e-12 * scale) == 7 * n


@pytest.mark.parametrize("model", [oracle.POISSON, oracle.SYMMETRON, oracle.FOFR])
def test_rms_residual_is_the_root_mean_square(model):
    """The convergence test's norm is sqrt(mean((L(phi) - Sigma)^2)) over the N^3 cells of the grid, here
    computed in numpy from the residual field; the solve reports the same value as its starting residual."""
    N, box = 8, 16.0
    gen = np.random.Generator(np.random.PCG64(23))
    eta = np.exp(gen.standard_normal((N,) * 3))
    phi = (-11.5 + 0.3 * gen.standard_normal((N,) * 3)) if model == oracle.FOFR else \
        (0.8 + 0.1 * gen.standard_normal((N,) * 3))
    p = oracle.Problem(model, N, box)
    sig = 1e-3 * gen.standard_normal((N,) * 3) * np.abs(oracle.residual(p, eta, phi)).max()
    for sigma in (None, sig):
        r = oracle.residual(p, eta, phi, sigma)
        want = math.sqrt(float(np.sum(r * r)) / N ** 3)
        assert oracle.rms_residual(p, eta, phi, sigma) == pytest.approx(want, rel=1e-13)
    res = oracle.solve(p, eta, phi, tol=0.0, max_cycles=0)
    r = oracle.residual(p, eta, phi)
    assert res.res0 == pytest.approx(math.sqrt(float(np.mean(r * r))), rel=1e-13)


# ---------------------------------------------------------------------------
# Paper's static sphere test (Sect. 5.1): far-field and screened plateaus
# ---------------------------------------------------------------------------

def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.mark.parametrize("a", [1.0, 0.5])
def test_static_sphere_symmetron_plateaus(a):
    row = [r for r in _golden_rows("static_sphere.txt") if r[0] == "symmetron"][0]
    delta, R, B = float(row[1]), float(row[2]), float(row[3])
    a_ssb, lam = 0.6, 1.0
    N = 64
    eta = synth.sphere_eta(N, B, R, delta).numpy()
    eta_out = 1.0 / (1.0 + 4 * math.pi / 3 * delta * (R / B) ** 3)
    chi_out = math.sqrt(1 - (a_ssb / a) ** 3 * eta_out)
    p = oracle.Problem(oracle.SYMMETRON, N, B, a=a, a_ssb=a_ssb, lambda0=lam)
    r = oracle.solve(p, eta, np.full((N,) * 3, chi_out), tol=1e-10)
    assert r.status == oracle.OK
    assert abs(r.phi[0, 0, 0] - chi_out) <= 1e-6          # far field (box corner)
    assert abs(r.phi[N // 2, N // 2, N // 2]) <= 1e-2     # screened interior
    assert r.phi.min() >= -1e-12


def test_static_sphere_fofr_far_field():
    row = [r for r in _golden_rows("static_sphere.txt") if r[0] == "fofr"][0]
    delta, R, B = float(row[1]), float(row[2]), float(row[3])
    fr0, a, N = 1e-6, 1.0, 64
    eta = synth.sphere_eta(N, B, R, delta).numpy()
    eta_out = 1.0 / (1.0 + 4 * math.pi / 3 * delta * (R / B) ** 3)
    rr = OL / OM
    fR_out = -fr0 * ((1 + 4 * rr) / (eta_out + 4 * rr)) ** 2
    p = oracle.Problem(oracle.FOFR, N, B, a=a, fR0_abs=fr0)
    # start from the cell-wise uniform-density solution: Newton on e^{-u/2} overshoots
    # without bound when it starts far above the screened value inside the sphere
    guess = np.log(a * a * fr0 * ((1 + 4 * rr) / (eta / a ** 3 + 4 * rr)) ** 2)
    r = oracle.solve(p, eta, guess, tol=1e-9)
    assert r.status == oracle.OK
    assert abs(-np.exp(r.phi[0, 0, 0]) / fR_out - 1) <= 1e-6


def test_table1_fofr_ranges():
    """Table 1's f(R) ranges follow from |f_R0| with the range formula of Sect. 4.2."""
    from paper_1307_6748_gb300 import isis
    for row in _golden_rows("table1_models.txt"):
        if row[0] != "fofr":
            continue
        n, fr0, lam = int(row[2]), float(row[3]), float(row[4])
        assert abs(isis.fofr_range(fr0, n) - lam) <= 0.051 * lam / lam + 0.05 * (lam > 10)
        assert isis.PRESETS[row[1]].fR0_abs == fr0
    for row in _golden_rows("table1_models.txt"):
        if row[0] == "symm":
            p = isis.PRESETS[row[1]]
            assert p.lambda0 == float(row[2]) and abs(p.a_ssb - 1 / (1 + float(row[3]))) < 1e-15
            assert p.beta == float(row[4])


# ---------------------------------------------------------------------------
# CIC (Sect. 5.1) and gradients
# ---------------------------------------------------------------------------

def cic_brute(N, x, y, z):
    """Brute force over every cell: weight = prod_d max(0, 1 - |x_d - c_d|) with periodic distance."""
    eta = np.zeros((N,) * 3)
    c = np.arange(N) + 0.5
    for px, py, pz in zip(x, y, z):
        w = []
        for v in (px, py, pz):
            d = np.abs(((v - c) + N / 2) % N - N / 2)
            w.append(np.maximum(0.0, 1.0 - d))
        eta += w[0][:, None, None] * w[1][None, :, None] * w[2][None, None, :]
    return eta * (N ** 3 / len(x))


@pytest.mark.parametrize("N", [4, 8])
def test_cic_brute_force(N):
    gen = np.random.Generator(np.random.PCG64(N))
    x, y, z = (gen.uniform(0, N, 50).astype(np.float32) for _ in range(3))
    x[0], y[0], z[0] = 0.0, N - 1e-3, 0.5  # edges and an exact centre
    got = oracle.cic_deposit(N, x, y, z)
    ref = cic_brute(N, x.astype(np.float64), y.astype(np.float64), z.astype(np.float64))
    assert np.abs(got - ref).max() <= 1e-12


def test_cic_invariants():
    N = 16
    q = (np.arange(N) + 0.5).astype(np.float32)
    X, Y, Z = np.meshgrid(q, q, q, indexing="ij")
    assert np.all(oracle.cic_deposit(N, X.ravel(), Y.ravel(), Z.ravel()) == 1.0)
    x, y, z = (v.numpy() for v in synth.zeldovich(N, 32.0, seed=3))
    eta = oracle.cic_deposit(N, x, y, z)
    assert abs(eta.sum() - N ** 3) <= 1e-9


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_gradient_of_sinusoid(axis):
    N, box, m = 32, 20.0, 2
    h = box / N
    f = synth.sinusoid(N, m=m, amp=1.0, axis=axis).numpy()
    g = oracle.gradient(f, box)
    k = 2 * math.pi * m / box
    x = (np.arange(N) + 0.5) * h
    shape = [1, 1, 1]
    shape[axis] = N
    exact = (np.cos(k * x) * math.sin(k * h) / h).reshape(shape)
    assert np.abs(g[axis] - exact).max() <= 1e-12
    assert all(np.abs(g[d]).max() == 0 for d in range(3) if d != axis)


def test_force_at_cell_centre():
    """A particle at a cell centre feels the grid force of that cell:
    -[a^2 grad Phi + 6 Om H0^2 (beta lambda0)^2/a_SSB^3 a^2 chi grad chi] (Eq. (symmetron_geodesics_tilde_chi))
    and -[a^2 grad Phi + e^u grad u / 2] for f(R) (Sect. 4.2)."""
    N, box, a = 16, 32.0, 0.8
    h = box / N
    Phi = 1e-6 * synth.sinusoid(N, m=1, axis=0).numpy()
    gPhi = oracle.gradient(Phi, box)
    chi = 0.9 + 0.01 * synth.sinusoid(N, m=2, axis=1).numpy()
    gchi = oracle.gradient(chi, box)
    u = -12.0 + 0.1 * synth.sinusoid(N, m=1, axis=2).numpy()
    gu = oracle.gradient(u, box)
    c = (3, 7, 11)
    x, y, z = (np.array([v + 0.5], dtype=np.float32) for v in c)
    Cs = 6 * OM * H0 ** 2 * (1.0 * 1.0) ** 2 / 0.5 ** 3
    assert abs(Cs - 1.42597e-6) < 1e-10
    g = oracle.fifth_force(oracle.Problem(oracle.SYMMETRON, N, box, a=a), Phi, chi, x, y, z)
    for d in range(3):
        exp_d = -(a * a * gPhi[d][c] + Cs * a * a * chi[c] * gchi[d][c])
        assert abs(g[d][0] - exp_d) <= 1e-12 * (abs(exp_d) + 1e-20)
    g = oracle.fifth_force(oracle.Problem(oracle.FOFR, N, box, a=a), Phi, u, x, y, z)
    for d in range(3):
        exp_d = -(a * a * gPhi[d][c] + 0.5 * math.exp(u[c]) * gu[d][c])
        assert abs(g[d][0] - exp_d) <= 1e-12 * (abs(exp_d) + 1e-20)
    del h


# ---- particle time stepping (Sect. 4.1, Eqs. (leap_frog_1)-(leap_frog_3)) ----

def test_tau_interval_matches_einstein_de_sitter():
    """Omega_m = 1, Omega_L = 0: tau(a0 -> a1) = 2 (a0^-1/2 - a1^-1/2) / H0 in closed form."""
    H0 = oracle.H0_MPC
    for a0, a1 in ((0.1, 0.2), (0.5, 1.0), (0.9, 0.95)):
        got = oracle.tau_interval(a0, a1, 1.0, 0.0, H0)
        assert abs(got / (2.0 * (a0 ** -0.5 - a1 ** -0.5) / H0) - 1.0) < 1e-10


def test_leapfrog_constant_force_is_exact():
    """With a constant acceleration the merged-kick leapfrog lands exactly on x0 + v0 T + g T^2 / 2 at the
    synchronised point (after a final half-kick) for any step sizes."""
    rng = np.random.Generator(np.random.PCG64(3))
    N, h = 1e9, 0.5  # no wrap
    x0 = [rng.uniform(0, 10, 5) for _ in range(3)]
    v0 = [rng.normal(size=5) for _ in range(3)]
    g = [np.full(5, c) for c in (0.3, -0.7, 1.1)]
    pos, vel = [p.copy() for p in x0], [v.copy() for v in v0]
    steps = [0.1, 0.25, 0.05, 0.3]
    prev = 0.0
    for dt in steps:
        oracle.leapfrog_kick_drift(pos, vel, g, 0.5 * (prev + dt), dt, N, h)
        prev = dt
    for d in range(3):
        vel[d] += 0.5 * prev * g[d] / h  # final half-kick
    T = sum(steps)
    for d in range(3):
        np.testing.assert_allclose(pos[d], x0[d] + v0[d] * T + 0.5 * g[d] / h * T * T, rtol=0, atol=1e-12)
        np.testing.assert_allclose(vel[d], v0[d] + g[d] / h * T, rtol=0, atol=1e-12)


def test_leapfrog_time_reversible():
    """A position-dependent force (harmonic): steps forward, velocities reversed, the same steps back
    return every particle to its start (the leapfrog is time-symmetric)."""
    rng = np.random.Generator(np.random.PCG64(4))
    N, h, w2, c = 1e9, 1.0, 0.8, 5.0
    pos = [rng.uniform(0, 10, 7) for _ in range(3)]
    vel = [rng.normal(size=7) for _ in range(3)]
    x0 = [p.copy() for p in pos]
    dt, k = 0.07, 20
    force = lambda: [-w2 * (p - c) for p in pos]
    # forward: half kick, (drift, full kick)^(k-1), drift, half kick
    def run():
        oracle.leapfrog_kick_drift(pos, vel, force(), 0.5 * dt, dt, N, h)
        for _ in range(k - 1):
            oracle.leapfrog_kick_drift(pos, vel, force(), dt, dt, N, h)
        g = force()
        for d in range(3):
            vel[d] += 0.5 * dt * g[d] / h
    run()
    for d in range(3):
        vel[d] *= -1.0
    run()
    for d in range(3):
        np.testing.assert_allclose(pos[d], x0[d], rtol=0, atol=1e-11)


def test_pm_uniform_translation_is_free_streaming():
    """A lattice moving rigidly keeps a uniform CIC density, so every field and force vanishes and the
    positions advance by v * (sum of dtau) exactly (mod N).  (The CIC sees FP32 positions: the velocities
    keep their values to the force of that rounding, 1e-10 here.)"""
    N, box = 8, 16.0
    q = np.arange(N) + 0.5
    X, Y, Z = np.meshgrid(q, q, q, indexing="ij")
    pos = [X.reshape(-1).astype(np.float64), Y.reshape(-1).astype(np.float64), Z.reshape(-1).astype(np.float64)]
    v = (2e-4, -1e-4, 3e-4)
    vel = [np.full(N ** 3, c) for c in v]
    a_steps = [0.8, 0.85, 0.9]
    pos, vel = oracle.pm_run(oracle.SYMMETRON, N, box, pos, vel, a_steps, tol=1e-10)
    T = oracle.tau_interval(0.8, 0.85) + oracle.tau_interval(0.85, 0.9)
    for d, (grid, c) in enumerate(zip((X, Y, Z), v)):
        np.testing.assert_allclose(pos[d], (grid.reshape(-1) + c * T) % N, rtol=0, atol=1e-9)
        np.testing.assert_allclose(vel[d], c, rtol=0, atol=1e-10)


def test_pm_gravity_conserves_momentum():
    """Gravity alone: CIC deposit, the symmetric central difference and CIC interpolation with the same
    kernel exert no net force, so the total momentum stays constant."""
    import torch
    N, box = 16, 32.0
    x, y, z, vx, vy, vz = synth.zeldovich_ic(N, box, 0.8, seed=6)
    pos = [t.double().numpy().copy() for t in (x, y, z)]
    vel = [t.double().numpy().copy() for t in (vx, vy, vz)]
    p0 = [v.sum() for v in vel]
    scale = sum(np.abs(v).sum() for v in vel)
    pos, vel = oracle.pm_run(None, N, box, pos, vel, [0.8, 0.84, 0.88, 0.92], tol=1e-11)
    for d in range(3):
        assert abs(vel[d].sum() - p0[d]) <= 1e-9 * scale
    del torch


# ---- the 1D radial solver of the static sphere test (Sect. 5.1) ----

def _yukawa_sphere(r, R, m, q):
    """Solution of (1/r^2)(r^2 e')' - m^2 e = q [r < R] vanishing at infinity (textbook)."""
    mr, mR = m * r, m * R
    inside = -(q / m ** 2) * (1.0 - (1.0 + mR) * np.exp(-mR) * np.sinh(mr) / mr)
    outside = -(q / m ** 2) * (mR * np.cosh(mR) - np.sinh(mR)) * np.exp(-mr) / mr
    return np.where(r < R, inside, outside)


def test_radial_poisson_matches_uniform_sphere_potential():
    from oracle import sphere1d as S
    R, Rmax, K = 3.0, 20.0, 2.0
    eta_in, eta_out = 50.0, 0.9
    rad = S.Radial(4000, Rmax)
    eta = S.sphere_profile(rad.edges, R, eta_in, eta_out)
    c, D = K * (eta_out - 1.0), K * (eta_in - eta_out)

    def exact(r):
        return c * r * r / 6.0 + D * np.where(r < R, r * r / 6.0 - R * R / 2.0, -R ** 3 / (3.0 * r))
    phi = S.poisson(eta, rad, K, 1.0, float(exact(np.array(Rmax + rad.dr / 2))))
    err = np.abs(phi - exact(rad.r)).max()
    assert err <= 1e-5 * np.abs(exact(rad.r)).max(), err


def test_radial_symmetron_linear_limit_is_yukawa():
    """A weak sphere: chi - chi_out follows the linear (Yukawa) profile with m^2 = 2 A (1 - s eta_out)."""
    from oracle import sphere1d as S
    A, s, R, Rmax = 0.5, 0.4, 2.0, 30.0
    eta_out, d_eta = 1.0, 1e-4
    chi_out = math.sqrt(1.0 - s * eta_out)
    rad = S.Radial(6000, Rmax)
    eta = S.sphere_profile(rad.edges, R, eta_out + d_eta, eta_out)
    chi = S.symmetron(eta, rad, A, s, chi_out)
    m = math.sqrt(2.0 * A * (1.0 - s * eta_out))
    lin = _yukawa_sphere(rad.r, R, m, A * s * d_eta * chi_out)
    assert np.abs((chi - chi_out) - lin).max() <= 2e-3 * np.abs(lin).max()


def test_radial_fofr_linear_limit_is_yukawa():
    """A weak sphere in f(R): u - u_out follows the Yukawa profile with m^2 = K2 e^{-u/(n+1)} / ((n+1) e^u)
    and source K1 d_eta / e^u (the equation linearised about the uniform solution)."""
    from oracle import sphere1d as S
    n, fr0, a, R, Rmax = 1, 1e-5, 1.0, 2.0, 60.0
    K1, K2, K3 = S.fofr_constants(a, OM, OL, S.H0_MPC, n, fr0)
    u_out = (n + 1) * math.log(K2 / K3)  # S(u, eta = 1) = 0
    d_eta = 1e-4
    rad = S.Radial(8000, Rmax)
    eta = S.sphere_profile(rad.edges, R, 1.0 + d_eta, 1.0)
    u = S.fofr(eta, rad, K1, K2, K3, n, u_out)
    b = math.exp(u_out)
    m = math.sqrt(K2 * math.exp(-u_out / (n + 1)) / ((n + 1) * b))
    lin = _yukawa_sphere(rad.r, R, m, K1 * d_eta / b)
    assert np.abs((u - u_out) - lin).max() <= 2e-3 * np.abs(lin).max()


# ---- the chameleon through the free source (Sect. 2) and its mapping to Hu-Sawicki (Sect. 6) ----

@pytest.mark.parametrize("n,a,etav", [(1.0, 1.0, 1.0), (1.0, 0.7, 3.0), (-0.5, 1.0, 0.4), (2.0, 0.5, 10.0)])
def test_chameleon_uniform_minimum(n, a, etav):
    """Uniform eta: the field sits at the minimum of its effective potential, psi^{-(1+n)} = a^-3 eta
    (the chameleon equation of Sect. 6 with a zero Laplacian), u = ln psi."""
    N, box = 8, 16.0
    u_exact = -math.log(etav * a ** -3) / (1.0 + n)
    p = oracle.Problem(oracle.CHAMELEON, N, box, a=a, lambda0=2.0, cham_n=n)
    r = oracle.solve(p, np.full((N,) * 3, etav), np.full((N,) * 3, u_exact + 0.2), tol=1e-10)
    assert r.status == oracle.OK
    assert np.abs(r.phi - u_exact).max() <= 1e-10
    assert abs(oracle.background_field(oracle.CHAMELEON, a, cham_n=n) + math.log(a ** -3) / (1 + n)) < 1e-15


def test_chameleon_range_is_lambda0():
    """eta = 1 + eps nu at a = 1: the first-order field solves lap d - d / lambda0^2 = eps nu / ((1+n) lambda0^2)
    (psi = 1 + d): lambda0 is the range of the field in today's background."""
    N, box, lam, n = 32, 32.0, 2.5, 1.0
    nu = synth.gaussian_field(N, box, 1.0, 23).numpy()
    errs = []
    for eps in (1e-4, 1e-3):
        r = oracle.solve(oracle.Problem(oracle.CHAMELEON, N, box, a=1.0, lambda0=lam, cham_n=n), 1.0 + eps * nu,
                         np.zeros((N,) * 3), tol=1e-12)
        lin = fft_solve(eps * nu / ((1 + n) * lam ** 2), 1.0 / lam ** 2, box / N)
        errs.append(np.linalg.norm(np.expm1(r.phi) - lin) / np.linalg.norm(lin))
    assert errs[0] <= 5e-4
    assert 5.0 < errs[1] / errs[0] < 20.0


def test_chameleon_n_minus_half_is_hu_sawicki_n1():
    """Sect. 6: the Hu-Sawicki model maps to the chameleon with n = -1/2.  Without a cosmological constant
    (OL = 0) the two equations are the same up to u_cham = u_HS + c: with K1 = Om a H0^2 and
    K2 = Om a^4 H0^2 (|f_R0| a^2)^{1/2} of the f(R) source, A_c e^{-c} a^-3 = K1 and A_c e^{-3c/2} = K2 give c and the
    chameleon's A_c = 2 a^2 / lambda0^2 by matching both source terms.  Both start from their backgrounds."""
    N, box, a, fr0 = 16, 64.0, 0.8, 1e-5
    eta = synth.lognormal_eta(N, box, 1.0, 31).numpy()
    K1 = OM * a * H0 ** 2
    K2 = OM * a ** 4 * H0 ** 2 * math.sqrt(fr0 * a * a)
    # A_c e^{-c} a^-3 = K1 and A_c e^{-3c/2} = K2
    c = 2.0 * math.log(K1 * a ** 3 / K2)
    Ac = K1 * a ** 3 * math.exp(c)
    lam = math.sqrt(2.0 * a * a / Ac)
    ph = oracle.Problem(oracle.FOFR, N, box, a=a, Omega_m=OM, Omega_L=0.0, fR0_abs=fr0, n=1)
    pc = oracle.Problem(oracle.CHAMELEON, N, box, a=a, Omega_m=OM, Omega_L=0.0, lambda0=lam, cham_n=-0.5)
    g = np.full((N,) * 3, 2.0 * math.log(K2 / K1))  # the eta = 1 background of the f(R) source
    rh = oracle.solve(ph, eta, g, tol=1e-12)
    rc = oracle.solve(pc, eta, g + c, tol=1e-12)
    assert rh.status == oracle.OK and rc.status == oracle.OK
    assert np.abs((rc.phi - c) - rh.phi).max() <= 1e-9
    assert np.ptp(rh.phi) > 0.5  # a non-trivial field


def test_chameleon_derivative_and_dense_newton():
    N, box = 8, 16.0
    gen = np.random.Generator(np.random.PCG64(6))
    eta = np.exp(gen.standard_normal((N,) * 3))
    p = oracle.Problem(oracle.CHAMELEON, N, box, a=0.9, lambda0=1.5, cham_n=1.0)
    phi = 0.3 * gen.standard_normal((N,) * 3)
    d = oracle.dL(p, eta, phi)
    for c in [(0, 0, 0), (3, 5, 7), (7, 1, 2)]:
        eps = 1e-6
        pp, pm = phi.copy(), phi.copy()
        pp[c] += eps
        pm[c] -= eps
        fd = (oracle.residual(p, eta, pp)[c] - oracle.residual(p, eta, pm)[c]) / (2 * eps)
        assert abs(fd - d[c]) <= 1e-7 * abs(d[c])
    guess = np.zeros((N,) * 3)
    ref = numpy_newton(p, eta, guess)
    r = oracle.solve(p, eta, guess, tol=1e-12)
    assert r.status == oracle.OK
    assert np.abs(r.phi - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())


def test_chameleon_force_at_cell_centre():
    """The chameleon's fifth force is a^2 grad ln A with ln A = beta phi / M_pl = (beta phi_0 / M_pl) e^u and
    beta phi_0 / M_pl = 3 (1+n) beta^2 Om H0^2 lambda0^2 (the background mass today, m0 = 1/lambda0)."""
    N, box, a, lam, beta, n = 16, 32.0, 0.8, 2.0, 0.7, 1.0
    Phi = 1e-6 * synth.sinusoid(N, m=1, axis=0).numpy()
    gPhi = oracle.gradient(Phi, box)
    u = 0.1 * synth.sinusoid(N, m=1, axis=2).numpy()
    gu = oracle.gradient(u, box)
    c = (3, 7, 11)
    x, y, z = (np.array([v + 0.5], dtype=np.float32) for v in c)
    Cc = 3 * (1 + n) * beta ** 2 * OM * H0 ** 2 * lam ** 2
    g = oracle.fifth_force(oracle.Problem(oracle.CHAMELEON, N, box, a=a, lambda0=lam, beta=beta, cham_n=n),
                           Phi, u, x, y, z)
    for d in range(3):
        exp_d = -(a * a * gPhi[d][c] + a * a * Cc * math.exp(u[c]) * gu[d][c])
        assert abs(g[d][0] - exp_d) <= 1e-12 * (abs(exp_d) + 1e-20)


# ---------------------------------------------------------------------------
# The convergence test's reference residual (reading R6)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("model,a", [(oracle.POISSON, 0.7), (oracle.SYMMETRON, 1.0), (oracle.SYMMETRON, 0.8),
                                     (oracle.FOFR, 1.0), (oracle.FOFR, 0.6), (oracle.CHAMELEON, 0.9)])
def test_reference_residual_is_the_background_residual(model, a):
    """R6 defines ref as the RMS of L(phi_bg) for the uniform background field phi_bg; the solver computes it in
    closed form from the density.  The two must agree: L of the uniform background, evaluated by the operator
    itself (pinned above), against the ref the solve reports (no cycles run)."""
    N, box = 8, 16.0
    eta = synth.lognormal_eta(N, box, 0.8, 11).numpy()
    p = oracle.Problem(model, N, box, a=a, a_ssb=0.5, cham_n=1.0)
    bg = oracle.background_field(model, a, a_ssb=0.5, cham_n=1.0)
    phi = np.full((N,) * 3, bg)
    rms = float(np.sqrt(np.mean(oracle.residual(p, eta, phi) ** 2)))
    r = oracle.solve(p, eta, phi, tol=1.0, max_cycles=0)
    assert rms > 0 and r.ref == pytest.approx(rms, rel=1e-12)


# ---- pins found missing by planting mistakes in the Python parts of the oracle ----

def test_radial_flux_form_is_second_order():
    """The 1D finite-volume operator with per-cell b (the f(R) form, face mean of b) approaches
    (1/r^2)(r^2 b u')' at second order in dr, away from r = 0 and the far boundary."""
    from oracle import sphere1d as S
    Rmax = 10.0
    u_f = lambda r: -1.0 + 0.3 * np.sin(0.5 * r) + 0.05 * r
    up = lambda r: 0.15 * np.cos(0.5 * r) + 0.05
    upp = lambda r: -0.075 * np.sin(0.5 * r)

    def exact(r):
        b = np.exp(u_f(r))
        return b * (up(r) ** 2 + upp(r) + 2.0 * up(r) / r)  # (1/r^2)(r^2 e^u u')'
    errs = []
    for M in (200, 400, 800):
        rad = S.Radial(M, Rmax)
        u = u_f(rad.r)
        L, _, _ = rad.div_flux(u, float(u_f(np.array(Rmax + rad.dr / 2))), np.exp(u))
        sel = (rad.r > 2.0) & (rad.r < 8.0)
        errs.append(np.abs(L[sel] - exact(rad.r[sel])).max())
    assert errs[1] / errs[0] < 0.3 and errs[2] / errs[1] < 0.3, errs


def test_radial_sphere_profile_conserves_mass():
    """The cell-averaged sphere profile holds the sphere's mass: sum of eta V over the radial cells equals
    eta_in R^3/3 + eta_out (R_max^3 - R^3)/3 (per unit solid angle) for R between cell edges."""
    from oracle import sphere1d as S
    rad = S.Radial(97, 10.0)
    R, eta_in, eta_out = 3.3, 40.0, 0.7
    eta = S.sphere_profile(rad.edges, R, eta_in, eta_out)
    mass = float(np.sum(eta * rad.vol))
    want = eta_in * R ** 3 / 3.0 + eta_out * (10.0 ** 3 - R ** 3) / 3.0
    assert abs(mass - want) <= 1e-12 * want
    assert eta[0] == eta_in and eta[-1] == eta_out


def test_sphere_densities_contrast_and_mean():
    """Sect. 5.1: the sphere is delta times denser than its surroundings in contrast (eta_in = (1 + delta)
    eta_out) and the box mean is 1."""
    from oracle import sphere1d as S
    for delta, R, B in ((5000.0, 3.0, 40.0), (10.0, 1.0, 8.0)):
        eta_in, eta_out = S.sphere_densities(delta, R, B)
        assert eta_in / eta_out - 1.0 == pytest.approx(delta, rel=1e-14)
        v = 4.0 * math.pi / 3.0 * R ** 3
        assert (eta_in * v + eta_out * (B ** 3 - v)) / B ** 3 == pytest.approx(1.0, rel=1e-13)


@pytest.mark.parametrize("a,n,fr0", [(0.5, 1, 1e-5), (0.8, 2, 1e-6)])
def test_radial_fofr_constants_uniform_solution(a, n, fr0):
    """The 1D solve's K1, K2, K3 give, at eta = 1, the uniform solution u = ln(a^2 |f_R|) with
    |f_R| = |f_R0| [(1 + 4r)/(a^-3 + 4r)]^(n+1) (Sect. 4.2), at a != 1 where every power of a shows."""
    from oracle import sphere1d as S
    K1, K2, K3 = S.fofr_constants(a, OM, OL, S.H0_MPC, n, fr0)
    r = OL / OM
    u = math.log(a * a * fr0 * ((1 + 4 * r) / (a ** -3 + 4 * r)) ** (n + 1))
    assert (n + 1) * math.log(K2 / K3) == pytest.approx(u, abs=1e-12)
    assert K1 == pytest.approx(OM * a * S.H0_MPC ** 2, rel=1e-15)


def test_leapfrog_wraps_into_the_box():
    """Positions are periodic: a particle drifting across x = N re-enters at x - N, one drifting below 0 at
    x + N."""
    N, h = 16, 1.0
    pos = [np.array([15.5, 0.25]), np.array([3.0, 3.0]), np.array([3.0, 3.0])]
    vel = [np.array([1.0, -0.5]), np.zeros(2), np.zeros(2)]
    oracle.leapfrog_kick_drift(pos, vel, [np.zeros(2)] * 3, 0.0, 1.0, N, h)
    np.testing.assert_allclose(pos[0], [0.5, 15.75], rtol=0, atol=1e-15)
