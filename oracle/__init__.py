"""Plain FP64 CPU oracle for the ISIS scalar-field multigrid solve (arXiv:1307.6748).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  The CUDA library never imports it.

The arithmetic lives in ``isis_oracle.c`` (plain C, FP64, one function per
paper passage); this module only compiles it with gcc and marshals numpy
arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import math
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "isis_oracle.c")
_LIB = os.path.join(_HERE, "libisis_oracle.so")

POISSON, SYMMETRON, FOFR, CHAMELEON = 0, 1, 2, 3
OK, EINVAL, ENOCONV, ENAN, ENOMEM = 0, -1, -2, -3, -5

# c = 1 units with lengths in Mpc/h: H0 = 100 h km/s/Mpc / c
H0_MPC = 1.0 / 2997.92458


def build(force: bool = False) -> str:
    """Compile the oracle into ``libisis_oracle.so`` (gcc, OpenMP, no FP contraction).

    With ISIS_ORACLE_SRC set, that C file is compiled next to itself and loaded instead: the mutation tests
    plant one mistake in a copy of the oracle and check that the pins catch it."""
    src, out = _SRC, _LIB
    if os.environ.get("ISIS_ORACLE_SRC"):
        src = os.environ["ISIS_ORACLE_SRC"]
        out = os.path.splitext(src)[0] + ".so"
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", out, src, "-lm"]
        subprocess.run(cmd, check=True)
    return out


class _Problem(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int), ("N", ctypes.c_int), ("box", ctypes.c_double), ("a", ctypes.c_double),
        ("Omega_m", ctypes.c_double), ("Omega_L", ctypes.c_double), ("H0", ctypes.c_double),
        ("lambda0", ctypes.c_double), ("beta", ctypes.c_double), ("a_ssb", ctypes.c_double),
        ("n", ctypes.c_int), ("fR0_abs", ctypes.c_double), ("cham_n", ctypes.c_double),
    ]


class _Info(ctypes.Structure):
    _fields_ = [
        ("cycles", ctypes.c_int), ("coarse_newton_max", ctypes.c_int), ("res0", ctypes.c_double),
        ("ref", ctypes.c_double), ("res_final", ctypes.c_double), ("hist", ctypes.c_double * 256),
    ]


@dataclass
class Problem:
    """Physical set-up of one solve; defaults are the paper's cosmology (Sect. 6.1)."""
    model: int
    N: int
    box: float
    a: float = 1.0
    Omega_m: float = 0.267
    Omega_L: float = 0.733
    H0: float = H0_MPC
    lambda0: float = 1.0
    beta: float = 1.0
    a_ssb: float = 0.5
    n: int = 1
    fR0_abs: float = 1e-5
    cham_n: float = 1.0

    def c(self) -> _Problem:
        return _Problem(self.model, self.N, self.box, self.a, self.Omega_m, self.Omega_L, self.H0,
                        self.lambda0, self.beta, self.a_ssb, self.n, self.fR0_abs, self.cham_n)


class _Patch(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("o", ctypes.c_int * 3), ("pn", ctypes.c_int * 3),
                ("periodic", ctypes.c_int), ("level", ctypes.c_int), ("eta_mean", ctypes.c_double)]


@dataclass
class Patch:
    """A refinement patch (Sects. 3.3.1, 3.4.1): a box of n parent cells at origin o of a parent grid of dims
    pn (periodic: the domain grid), refined by two; level >= 1 sets h = box / (N 2^level)."""
    n: tuple
    o: tuple
    pn: tuple
    periodic: bool
    level: int = 1
    eta_mean: float = 1.0

    def c(self) -> _Patch:
        return _Patch((ctypes.c_int * 3)(*self.n), (ctypes.c_int * 3)(*self.o), (ctypes.c_int * 3)(*self.pn),
                      int(self.periodic), self.level, self.eta_mean)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = P(ctypes.c_double)
        f = P(ctypes.c_float)
        _lib.orc_solve.argtypes = [P(_Problem), d, d, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, P(_Info)]
        _lib.orc_residual.argtypes = [P(_Problem), d, d, d, d]
        _lib.orc_dL.argtypes = [P(_Problem), d, d, d]
        _lib.orc_smooth.argtypes = [P(_Problem), d, d, d]
        _lib.orc_restrict.argtypes = [ctypes.c_int, d, d]
        _lib.orc_restrict.restype = None
        _lib.orc_prolong_add.argtypes = [ctypes.c_int, d, d]
        _lib.orc_prolong_add.restype = None
        _lib.orc_dense_newton.argtypes = [P(_Problem), d, d, d, P(ctypes.c_int)]
        _lib.orc_jacobian.argtypes = [P(_Problem), d, d, d]
        _lib.orc_rms_residual.argtypes = [P(_Problem), d, d, d]
        _lib.orc_rms_residual.restype = ctypes.c_double
        _lib.orc_cic_deposit.argtypes = [ctypes.c_int, ctypes.c_int64, f, f, f, d]
        _lib.orc_gradient.argtypes = [ctypes.c_int, ctypes.c_double, d, d, d, d]
        _lib.orc_fifth_force.argtypes = [P(_Problem), d, d, ctypes.c_int64, f, f, f, d, d, d]
        u8 = P(ctypes.c_uint8)
        _lib.orc_patch_solve.argtypes = [P(_Problem), P(_Patch), d, u8, d, d, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, P(_Info)]
        _lib.orc_patch_eval.argtypes = [P(_Problem), P(ctypes.c_int), ctypes.c_double, d, d, d, d, d,
                                        ctypes.c_double, d, d]
        _lib.orc_patch_prolong_add.argtypes = [P(ctypes.c_int), d, d, d]
    return _lib


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f(a):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


@dataclass
class SolveResult:
    status: int
    phi: np.ndarray
    cycles: int
    res0: float
    ref: float
    res_final: float
    hist: list
    coarse_newton_max: int


def solve(p: Problem, eta: np.ndarray, phi0: np.ndarray, tol: float = 1e-10, nu1: int = 2, nu2: int = 2,
          ncoarse: int = 4, max_cycles: int = 100) -> SolveResult:
    """FAS V(nu1,nu2) solve of L(phi) = 0 from the guess phi0 (Sect. 3.2)."""
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    phi = np.array(phi0, dtype=np.float64, order="C", copy=True)
    assert eta.shape == (p.N,) * 3 and phi.shape == (p.N,) * 3
    info = _Info()
    pc = p.c()
    st = lib().orc_solve(ctypes.byref(pc), _d(eta), _d(phi), tol, nu1, nu2, ncoarse, max_cycles, ctypes.byref(info))
    return SolveResult(st, phi, info.cycles, info.res0, info.ref, info.res_final,
                       [info.hist[i] for i in range(info.cycles)], info.coarse_newton_max)


def residual(p: Problem, eta, phi, sigma=None) -> np.ndarray:
    """L(phi) - Sigma on one grid."""
    out = np.empty((p.N,) * 3)
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    sg = None if sigma is None else np.ascontiguousarray(sigma, dtype=np.float64)
    pc = p.c()
    assert lib().orc_residual(ctypes.byref(pc), _d(eta), _d(phi), _d(sg), _d(out)) == OK
    return out


def dL(p: Problem, eta, phi) -> np.ndarray:
    """Diagonal derivative dL_c/dphi_c on one grid."""
    out = np.empty((p.N,) * 3)
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    pc = p.c()
    assert lib().orc_dL(ctypes.byref(pc), _d(eta), _d(phi), _d(out)) == OK
    return out


def smooth(p: Problem, eta, phi, sigma=None) -> np.ndarray:
    """One red-black Newton-Gauss-Seidel sweep; returns the new field."""
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    out = np.array(phi, dtype=np.float64, order="C", copy=True)
    sg = None if sigma is None else np.ascontiguousarray(sigma, dtype=np.float64)
    pc = p.c()
    assert lib().orc_smooth(ctypes.byref(pc), _d(eta), _d(out), _d(sg)) == OK
    return out


def restrict(fine: np.ndarray) -> np.ndarray:
    fine = np.ascontiguousarray(fine, dtype=np.float64)
    NH = fine.shape[0] // 2
    out = np.empty((NH,) * 3)
    lib().orc_restrict(NH, _d(fine), _d(out))
    return out


def prolong_add(cdelta: np.ndarray, fine: np.ndarray) -> np.ndarray:
    cdelta = np.ascontiguousarray(cdelta, dtype=np.float64)
    out = np.array(fine, dtype=np.float64, order="C", copy=True)
    lib().orc_prolong_add(cdelta.shape[0], _d(cdelta), _d(out))
    return out


def dense_newton(p: Problem, eta, phi0, sigma=None):
    """Dense exact-Jacobian Newton solve of L(phi) = Sigma on one small grid."""
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    phi = np.array(phi0, dtype=np.float64, order="C", copy=True)
    sg = None if sigma is None else np.ascontiguousarray(sigma, dtype=np.float64)
    steps = ctypes.c_int(0)
    pc = p.c()
    st = lib().orc_dense_newton(ctypes.byref(pc), _d(eta), _d(phi), _d(sg), ctypes.byref(steps))
    return st, phi, steps.value


def jacobian(p: Problem, eta, phi) -> np.ndarray:
    """The dense Jacobian dF_r/dphi_c (N^3 x N^3) of the coarsest-level Newton solve at phi.  Poisson's
    carries the shift -(6/h^2)/N^3 in every entry, which removes the periodic Laplacian's null space."""
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    n = p.N ** 3
    out = np.empty((n, n))
    pc = p.c()
    assert lib().orc_jacobian(ctypes.byref(pc), _d(eta), _d(phi), _d(out)) == OK
    return out


def rms_residual(p: Problem, eta, phi, sigma=None) -> float:
    """RMS of L(phi) - Sigma over one grid: the norm of the convergence test."""
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    sg = None if sigma is None else np.ascontiguousarray(sigma, dtype=np.float64)
    pc = p.c()
    return float(lib().orc_rms_residual(ctypes.byref(pc), _d(eta), _d(phi), _d(sg)))


def cic_deposit(N: int, x, y, z) -> np.ndarray:
    """CIC density eta (mean 1) from particle positions in cell units (Sect. 5.1)."""
    x, y, z = (np.ascontiguousarray(v, dtype=np.float32) for v in (x, y, z))
    out = np.empty((N,) * 3)
    assert lib().orc_cic_deposit(N, x.size, _f(x), _f(y), _f(z), _d(out)) == OK
    return out


def gradient(f: np.ndarray, box: float):
    f = np.ascontiguousarray(f, dtype=np.float64)
    N = f.shape[0]
    g = [np.empty_like(f) for _ in range(3)]
    lib().orc_gradient(N, box, _d(f), _d(g[0]), _d(g[1]), _d(g[2]))
    return g


def fifth_force(p: Problem, Phi, phi, x, y, z):
    """Per-particle acceleration -[grad Phi~ + F5] (Sects. 4.1, 4.2); Phi or phi may be None."""
    x, y, z = (np.ascontiguousarray(v, dtype=np.float32) for v in (x, y, z))
    Phi = None if Phi is None else np.ascontiguousarray(Phi, dtype=np.float64)
    phi = None if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
    g = [np.empty(x.size) for _ in range(3)]
    pc = p.c()
    assert lib().orc_fifth_force(ctypes.byref(pc), _d(Phi), _d(phi), x.size, _f(x), _f(y), _f(z),
                                 _d(g[0]), _d(g[1]), _d(g[2])) == OK
    return g


# ---------------------------------------------------------------------------
# Particle time stepping: leapfrog in super-comoving time tau
# (Sect. 4.1, Eqs. (leap_frog_1)-(leap_frog_3); the same scheme for f(R), Sect. 4.2).
# Positions and velocities in cell units, tau in Mpc/h (c = 1):
#   d^2 x / dtau^2 = g = -[grad Phi~ + F5],   dtau = da / (a^3 H0 E(a)).
# ---------------------------------------------------------------------------

def tau_interval(a0: float, a1: float, Omega_m: float = 0.267, Omega_L: float = 0.733, H0: float = H0_MPC,
                 n: int = 256) -> float:
    """Super-comoving time from a0 to a1: the integral of da / (a^3 H0 E(a)), E(a) = sqrt(Om a^-3 + OL),
    by the composite Simpson rule with n (even) intervals."""
    a = np.linspace(a0, a1, n + 1)
    f = 1.0 / (a ** 3 * H0 * np.sqrt(Omega_m / a ** 3 + Omega_L))
    w = np.ones(n + 1)
    w[1:-1:2] = 4.0
    w[2:-1:2] = 2.0
    return float((a1 - a0) / (3.0 * n) * np.dot(w, f))


def leapfrog_kick_drift(pos, vel, g, kick: float, drift: float, N: int, h: float):
    """One merged kick and drift (FP64, in place): v += kick g / h; x += drift v; x wrapped into [0, N).
    kick = (dtau_{n-1} + dtau_n) / 2 joins the second half-kick of the previous step to the first of this one."""
    for d in range(3):
        vel[d] += kick * g[d] / h
        pos[d] += drift * vel[d]
        pos[d] %= N


def background_field(model: int, a: float, Omega_m: float = 0.267, Omega_L: float = 0.733, a_ssb: float = 0.5,
                     n: int = 1, fR0_abs: float = 1e-5, cham_n: float = 1.0, **_) -> float:
    """Uniform-density solution: chi = sqrt(1 - (a_SSB/a)^3) above symmetry breaking, else 0 (Sect. 4.1);
    u = ln(a^2 |f_R|), |f_R| = |f_R0| [(1 + 4 r) / (a^-3 + 4 r)]^(n+1), r = OL/Om (Sect. 4.2);
    chameleon u = ln psi, psi^{-(1+n)} = a^-3: u = 3 ln(a) / (1 + n)."""
    if model == SYMMETRON:
        v = 1.0 - (a_ssb / a) ** 3
        return math.sqrt(v) if v > 0 else 0.0
    if model == FOFR:
        r = Omega_L / Omega_m
        return math.log(a * a * fR0_abs * ((1 + 4 * r) / (a ** -3 + 4 * r)) ** (n + 1))
    if model == CHAMELEON:
        return 3.0 * math.log(a) / (1.0 + cham_n)
    return 0.0


def pm_run(model, N: int, box: float, pos, vel, a_steps, tol: float = 1e-10, ncoarse: int = 4, **params):
    """Leapfrog through a_steps[0] -> ... -> a_steps[-1].  At each a_n: CIC density of the positions, the
    Poisson field, the scalar field (model SYMMETRON or FOFR; None: gravity only), the acceleration of every
    particle, then the merged kick and the drift by dtau_n = tau(a_n -> a_{n+1}).  pos, vel: three FP64 arrays
    each (cell units), updated in place; returns them after the last drift (velocities at the half step)."""
    h = box / N
    Phi = np.zeros((N,) * 3)
    phi = None
    dtau_prev = 0.0
    cos = {k: params[k] for k in ("Omega_m", "Omega_L", "H0") if k in params}
    for a, a_next in zip(a_steps[:-1], a_steps[1:]):
        x, y, z = (np.asarray(p, dtype=np.float32) for p in pos)
        eta = cic_deposit(N, x, y, z)
        pp = Problem(POISSON, N, box, a=a, **params)
        Phi = solve(pp, eta, Phi, tol=tol, ncoarse=ncoarse).phi
        if model is not None:
            ps = Problem(model, N, box, a=a, **params)
            if phi is None:
                bg = background_field(model, a, **{k: params[k] for k in ("Omega_m", "Omega_L", "a_ssb", "n",
                                                                          "fR0_abs", "cham_n") if k in params})
                phi = np.full((N,) * 3, bg)
            phi = solve(ps, eta, phi, tol=tol, ncoarse=ncoarse).phi
            g = fifth_force(ps, Phi, phi, x, y, z)
        else:
            g = fifth_force(pp, Phi, None, x, y, z)
        dtau = tau_interval(a, a_next, **cos)
        leapfrog_kick_drift(pos, vel, g, 0.5 * (dtau_prev + dtau), dtau, N, h)
        dtau_prev = dtau
    return pos, vel


def patch_solve(p: Problem, patch: Patch, parent: np.ndarray, flags: np.ndarray, eta: np.ndarray, u0=None,
                tol: float = 1e-10, nu1: int = 2, nu2: int = 2, max_cycles: int = 100) -> SolveResult:
    """FAS solve on a refinement patch (P1-P7 of isis_oracle.c).  parent: the parent field (patch.pn);
    flags: refined parent cells of the box (patch.n, uint8); eta: finest patch density (2 patch.n);
    u0: guess at the unknowns (None: start from the interpolated parent field)."""
    nf = tuple(2 * v for v in patch.n)
    parent = np.ascontiguousarray(parent, dtype=np.float64)
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    assert parent.shape == tuple(patch.pn) and flags.shape == tuple(patch.n) and eta.shape == nf
    u = np.zeros(nf) if u0 is None else np.array(u0, dtype=np.float64, order="C", copy=True)
    assert u.shape == nf
    info = _Info()
    pc, bc = p.c(), patch.c()
    st = lib().orc_patch_solve(ctypes.byref(pc), ctypes.byref(bc), _d(parent),
                               flags.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _d(eta), _d(u), tol, nu1, nu2,
                               max_cycles, 1 if u0 is None else 0, ctypes.byref(info))
    return SolveResult(st, u, info.cycles, info.res0, info.ref, info.res_final,
                       [info.hist[i] for i in range(info.cycles)], 0)


def patch_eval(p: Problem, h: float, m, eta, u, pre, sig=None, eta_mean: float = 1.0):
    """(L(u) - Sigma, dL/du) at the unknowns (m > 0) of one patch level, ghosts by Eq. (ueq) with u^Pre = pre."""
    m, eta, u, pre = (np.ascontiguousarray(v, dtype=np.float64) for v in (m, eta, u, pre))
    sig = None if sig is None else np.ascontiguousarray(sig, dtype=np.float64)
    F, dF = np.zeros(m.shape), np.zeros(m.shape)
    n = (ctypes.c_int * 3)(*m.shape)
    pc = p.c()
    st = lib().orc_patch_eval(ctypes.byref(pc), n, h, _d(m), _d(eta), _d(u), _d(pre), _d(sig), eta_mean, _d(F),
                              _d(dF))
    assert st == OK, st
    return F, dF


def patch_prolong_add(cdelta, m_fine, fine) -> np.ndarray:
    """fine + P(cdelta) at the fine cells with m > 0 of one patch level (P5); returns the new fine array."""
    cdelta = np.ascontiguousarray(cdelta, dtype=np.float64)
    m_fine = np.ascontiguousarray(m_fine, dtype=np.float64)
    out = np.array(fine, dtype=np.float64, order="C", copy=True)
    assert m_fine.shape == out.shape == tuple(2 * v for v in cdelta.shape)
    nc = (ctypes.c_int * 3)(*cdelta.shape)
    assert lib().orc_patch_prolong_add(nc, _d(cdelta), _d(m_fine), _d(out)) == OK
    return out
