"""Python binding of the C ABI in ``include/isis.h`` (ctypes over libisis_gb300.so).

Argument marshalling only: every step of the solve runs in the CUDA library.
Arrays are torch CUDA tensors (contiguous, on the current device); the stream
is torch's current stream unless one is passed.  The library must have been
built (``paper_1307_6748_gb300.build.build()``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import weakref
from dataclasses import dataclass, field

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libisis_gb300.so")

ISIS_OK, ISIS_EINVAL, ISIS_ENOCONV, ISIS_ENAN, ISIS_ECUDA, ISIS_ENOMEM, ISIS_ETIMEOUT, ISIS_EINTERNAL = (
    0, -1, -2, -3, -4, -5, -6, -7)
ISIS_SYMMETRON, ISIS_FOFR_HS, ISIS_CHAMELEON = 1, 2, 3
ISIS_F64, ISIS_F32, ISIS_F32_REFINE64 = 0, 1, 2

H0_MPC = 1.0 / 2997.92458  # (Mpc/h)^-1 with c = 1

# Every function the header declares (checked by the tests).
EXPORTS = ("isis_cic_deposit", "isis_cic_deposit_noalloc", "isis_poisson_solve", "isis_scalar_solve", "isis_fifth_force",
           "isis_strerror", "isis_release_workspace", "isis_prof_enable", "isis_prof_reset", "isis_prof_read",
           "isis_launch_count", "isis_selftest_exp_ff", "isis_selftest_ff_to_f64", "isis_kick_drift", "isis_patch_poisson_solve",
           "isis_patch_scalar_solve", "isis_background_field", "isis_host_alloc", "isis_host_free")
ISIS_INIT_INPUT, ISIS_INIT_BACKGROUND, ISIS_INIT_LOCAL, ISIS_INIT_PARENT = 0, 1, 2, 3


class isis_grid(ctypes.Structure):
    _fields_ = [("Omega_m", ctypes.c_double), ("Omega_L", ctypes.c_double), ("H0", ctypes.c_double),
                ("box", ctypes.c_double), ("N", ctypes.c_int)]


class isis_params(ctypes.Structure):
    _fields_ = [("lambda0", ctypes.c_double), ("beta", ctypes.c_double), ("a_ssb", ctypes.c_double),
                ("n", ctypes.c_int), ("fR0_abs", ctypes.c_double), ("cham_n", ctypes.c_double)]


class isis_mg_opts(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("n_coarsest", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("prec", ctypes.c_int), ("inner_cycles", ctypes.c_int),
                ("init", ctypes.c_int), ("fmg", ctypes.c_int)]


class isis_patch(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("origin", ctypes.c_int * 3), ("parent_dims", ctypes.c_int * 3),
                ("parent_periodic", ctypes.c_int), ("level", ctypes.c_int), ("eta_mean", ctypes.c_double)]


class isis_prof_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class isis_solve_info(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("outer", ctypes.c_int), ("nhist", ctypes.c_int), ("res0", ctypes.c_double),
                ("res_ref", ctypes.c_double), ("res_final", ctypes.c_double), ("hist", ctypes.c_double * 128)]


class IsisError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1307_6748_gb300.build.build() "
                          "(the solver has no CPU fallback)")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, f_p = ctypes.c_void_p, ctypes.c_void_p
    lib.isis_cic_deposit.argtypes = [P(isis_grid), f_p, f_p, f_p, ctypes.c_int64, vp, ctypes.c_int, vp]
    lib.isis_cic_deposit_noalloc.argtypes = [P(isis_grid), f_p, f_p, f_p, ctypes.c_int64, vp, ctypes.c_int, vp]
    lib.isis_cic_deposit_noalloc.restype = ctypes.c_int
    lib.isis_poisson_solve.argtypes = [P(isis_grid), ctypes.c_double, vp, vp, ctypes.c_double, P(isis_mg_opts),
                                       P(isis_solve_info), vp]
    lib.isis_scalar_solve.argtypes = [ctypes.c_int, P(isis_params), P(isis_grid), ctypes.c_double, vp, vp,
                                      ctypes.c_double, P(isis_mg_opts), P(isis_solve_info), vp]
    lib.isis_fifth_force.argtypes = [ctypes.c_int, P(isis_params), P(isis_grid), ctypes.c_double, vp, vp,
                                     ctypes.c_int, f_p, f_p, f_p, ctypes.c_int64, f_p, f_p, f_p, vp]
    lib.isis_kick_drift.argtypes = [P(isis_grid), f_p, f_p, f_p, f_p, f_p, f_p, f_p, f_p, f_p, ctypes.c_int64,
                                    ctypes.c_double, ctypes.c_double, vp]
    lib.isis_kick_drift.restype = ctypes.c_int
    lib.isis_patch_poisson_solve.argtypes = [P(isis_grid), ctypes.c_double, P(isis_patch), vp, vp, vp, vp,
                                             ctypes.c_double, P(isis_mg_opts), P(isis_solve_info), vp]
    lib.isis_patch_scalar_solve.argtypes = [ctypes.c_int, P(isis_params), P(isis_grid), ctypes.c_double,
                                            P(isis_patch), vp, vp, vp, vp, ctypes.c_double, P(isis_mg_opts),
                                            P(isis_solve_info), vp]
    lib.isis_patch_poisson_solve.restype = ctypes.c_int
    lib.isis_patch_scalar_solve.restype = ctypes.c_int
    lib.isis_background_field.argtypes = [ctypes.c_int, P(isis_params), P(isis_grid), ctypes.c_double,
                                          P(ctypes.c_double)]
    lib.isis_background_field.restype = ctypes.c_int
    lib.isis_strerror.argtypes = [ctypes.c_int]
    lib.isis_strerror.restype = ctypes.c_char_p
    lib.isis_release_workspace.argtypes = []
    lib.isis_release_workspace.restype = None
    lib.isis_prof_enable.argtypes = [ctypes.c_int]
    lib.isis_prof_enable.restype = None
    lib.isis_prof_reset.argtypes = []
    lib.isis_prof_reset.restype = None
    lib.isis_prof_read.argtypes = [P(isis_prof_entry), ctypes.c_int]
    lib.isis_prof_read.restype = ctypes.c_int
    lib.isis_launch_count.argtypes = []
    lib.isis_launch_count.restype = ctypes.c_int64
    lib.isis_host_alloc.argtypes = [ctypes.c_size_t, P(ctypes.c_void_p)]
    lib.isis_host_alloc.restype = ctypes.c_int
    lib.isis_host_free.argtypes = [ctypes.c_void_p]
    lib.isis_host_free.restype = ctypes.c_int
    for name in ("isis_cic_deposit", "isis_poisson_solve", "isis_scalar_solve", "isis_fifth_force"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# Plain-Python mirrors of the structs
# ---------------------------------------------------------------------------

@dataclass
class Grid:
    N: int
    box: float
    Omega_m: float = 0.267
    Omega_L: float = 0.733
    H0: float = H0_MPC

    def c(self):
        return isis_grid(self.Omega_m, self.Omega_L, self.H0, self.box, self.N)


@dataclass
class Params:
    lambda0: float = 1.0
    beta: float = 1.0
    a_ssb: float = 0.5
    n: int = 1
    fR0_abs: float = 1e-5
    cham_n: float = 1.0  # chameleon exponent (ISIS_CHAMELEON uses lambda0, beta and cham_n)

    def c(self):
        return isis_params(self.lambda0, self.beta, self.a_ssb, self.n, self.fR0_abs, self.cham_n)


@dataclass
class Opts:
    nu1: int = 2
    nu2: int = 2
    n_coarsest: int = 4
    max_cycles: int = 100
    prec: int = ISIS_F64
    inner_cycles: int = 2
    init: int = ISIS_INIT_INPUT
    fmg: int = 0  # ISIS_F32_REFINE64: nested-iteration start of the FP32 phase

    def c(self):
        return isis_mg_opts(self.nu1, self.nu2, self.n_coarsest, self.max_cycles, self.prec, self.inner_cycles,
                            self.init, self.fmg)


@dataclass
class Patch:
    """A refinement patch: n parent cells at origin of a parent grid of dims parent_dims (periodic: the domain
    grid, level 1), refined by two; eta_mean is the domain's mean density (Poisson)."""
    n: tuple
    origin: tuple
    parent_dims: tuple
    periodic: bool
    level: int = 1
    eta_mean: float = 1.0

    def c(self):
        return isis_patch((ctypes.c_int * 3)(*self.n), (ctypes.c_int * 3)(*self.origin),
                          (ctypes.c_int * 3)(*self.parent_dims), 1 if self.periodic else 0, self.level,
                          self.eta_mean)

    @property
    def fine_shape(self):
        return tuple(2 * v for v in self.n)


@dataclass
class Info:
    status: int = 0
    cycles: int = 0
    outer: int = 0
    res0: float = 0.0
    res_ref: float = 0.0
    res_final: float = 0.0
    hist: list = field(default_factory=list)


def _ptr(t: torch.Tensor | None, dtype=None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _check(st: int, what: str, allow=(ISIS_OK,)):
    if st not in allow:
        raise IsisError(st, f"{what}: {load().isis_strerror(st).decode()}")
    return st


def _field_dtype(prec: int):
    return torch.float32 if prec == ISIS_F32 else torch.float64


def strerror(status: int) -> str:
    return load().isis_strerror(status).decode()


def release_workspace() -> None:
    load().isis_release_workspace()


def host_empty(n: int, dtype=torch.float32) -> torch.Tensor:
    """A CPU tensor of n elements in page-locked host memory from isis_host_alloc (huge-page backed where the
    kernel grants it), for the arrays copied every step; isis_host_free runs when the last tensor viewing it is
    released.  Zero-filled."""
    lib = load()
    esize = torch.empty((), dtype=dtype).element_size()
    nbytes = int(n) * esize
    ptr = ctypes.c_void_p()
    _check(lib.isis_host_alloc(nbytes, ctypes.byref(ptr)), "isis_host_alloc")
    buf = (ctypes.c_ubyte * nbytes).from_address(ptr.value)
    weakref.finalize(buf, lib.isis_host_free, ptr.value)
    return torch.frombuffer(buf, dtype=dtype, count=int(n))


def prof_enable(on: bool = True) -> None:
    load().isis_prof_enable(1 if on else 0)


def prof_reset() -> None:
    load().isis_prof_reset()


def launch_count() -> int:
    return int(load().isis_launch_count())


def prof_read() -> dict:
    """Per kernel kind, and for the multigrid kernels per model and form ("smooth_fine[fofr/delta]"):
    {name: (launches, ms, algorithmic bytes)} (synchronises the device)."""
    buf = (isis_prof_entry * 256)()
    n = load().isis_prof_read(buf, 256)
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].ms), float(buf[i].bytes)) for i in range(n)}


# ---------------------------------------------------------------------------
# The four calls
# ---------------------------------------------------------------------------

def isis_cic_deposit(grid: Grid, x: torch.Tensor, y: torch.Tensor, z: torch.Tensor, eta: torch.Tensor,
                     stream=None) -> torch.Tensor:
    """CIC density (mean 1) of particles at cell-unit positions x, y, z into eta (float64 or float32)."""
    lib = load()
    f64 = 1 if eta.dtype == torch.float64 else 0
    g = grid.c()
    st = lib.isis_cic_deposit(ctypes.byref(g), _ptr(x, torch.float32), _ptr(y, torch.float32),
                              _ptr(z, torch.float32), x.numel(), _ptr(eta), f64, _stream(stream))
    _check(st, "isis_cic_deposit")
    return eta


def isis_cic_deposit_noalloc(grid: Grid, x: torch.Tensor, y: torch.Tensor, z: torch.Tensor, eta: torch.Tensor,
                             stream=None) -> torch.Tensor:
    """CIC deposit that allocates no device memory (grids up to 64^3; see include/isis.h)."""
    lib = load()
    f64 = 1 if eta.dtype == torch.float64 else 0
    g = grid.c()
    st = lib.isis_cic_deposit_noalloc(ctypes.byref(g), _ptr(x, torch.float32), _ptr(y, torch.float32),
                                      _ptr(z, torch.float32), x.numel(), _ptr(eta), f64, _stream(stream))
    _check(st, "isis_cic_deposit_noalloc")
    return eta


def _info(ci: isis_solve_info, st: int, prec: int) -> Info:
    nh = ci.nhist
    return Info(st, ci.cycles, ci.outer, ci.res0, ci.res_ref, ci.res_final, [ci.hist[i] for i in range(nh)])


def isis_poisson_solve(grid: Grid, a: float, eta: torch.Tensor, Phi: torch.Tensor, tol: float = 1e-10,
                       opts: Opts | None = None, stream=None, allow_noconv: bool = False) -> Info:
    """Solve lap Phi = 1.5 Om H0^2 (eta - <eta>)/a in place on Phi (initial guess in)."""
    lib = load()
    o = opts or Opts()
    dt = _field_dtype(o.prec)
    g, oc, info = grid.c(), o.c(), isis_solve_info()
    st = lib.isis_poisson_solve(ctypes.byref(g), a, _ptr(eta, dt), _ptr(Phi, dt), tol, ctypes.byref(oc),
                                ctypes.byref(info), _stream(stream))
    _check(st, "isis_poisson_solve", (ISIS_OK, ISIS_ENOCONV) if allow_noconv else (ISIS_OK,))
    return _info(info, st, o.prec)


def isis_scalar_solve(model: int, params: Params, grid: Grid, a: float, eta: torch.Tensor, phi: torch.Tensor,
                      tol: float = 1e-10, opts: Opts | None = None, stream=None, allow_noconv: bool = False) -> Info:
    """FAS solve of the symmetron (phi = chi) or f(R) (phi = u) equation in place on phi."""
    lib = load()
    o = opts or Opts()
    dt = _field_dtype(o.prec)
    g, p, oc, info = grid.c(), params.c(), o.c(), isis_solve_info()
    st = lib.isis_scalar_solve(int(model), ctypes.byref(p), ctypes.byref(g), a, _ptr(eta, dt), _ptr(phi, dt),
                               tol, ctypes.byref(oc), ctypes.byref(info), _stream(stream))
    _check(st, "isis_scalar_solve", (ISIS_OK, ISIS_ENOCONV) if allow_noconv else (ISIS_OK,))
    return _info(info, st, o.prec)


def isis_fifth_force(model: int, params: Params, grid: Grid, a: float, Phi: torch.Tensor | None,
                     phi: torch.Tensor | None, x: torch.Tensor, y: torch.Tensor, z: torch.Tensor,
                     out=None, stream=None):
    """Per-particle acceleration -[grad(a^2 Phi) + F5]; returns (gx, gy, gz) float32."""
    lib = load()
    ref = Phi if Phi is not None else phi
    f64 = 1 if (ref is None or ref.dtype == torch.float64) else 0
    n = x.numel()
    if out is None:
        out = tuple(torch.empty(n, device=x.device, dtype=torch.float32) for _ in range(3))
    g, p = grid.c(), params.c()
    st = lib.isis_fifth_force(int(model), ctypes.byref(p), ctypes.byref(g), a, _ptr(Phi), _ptr(phi), f64,
                              _ptr(x, torch.float32), _ptr(y, torch.float32), _ptr(z, torch.float32), n,
                              _ptr(out[0], torch.float32), _ptr(out[1], torch.float32),
                              _ptr(out[2], torch.float32), _stream(stream))
    _check(st, "isis_fifth_force")
    return out


def isis_kick_drift(grid: Grid, x, y, z, vx, vy, vz, g, kick: float, drift: float, stream=None) -> None:
    """Leapfrog kick and drift in place (cell units; g = (gx, gy, gz) per Mpc/h)."""
    lib = load()
    gr = grid.c()
    f = torch.float32
    st = lib.isis_kick_drift(ctypes.byref(gr), _ptr(x, f), _ptr(y, f), _ptr(z, f), _ptr(vx, f), _ptr(vy, f),
                             _ptr(vz, f), _ptr(g[0], f), _ptr(g[1], f), _ptr(g[2], f), x.numel(), float(kick),
                             float(drift), _stream(stream))
    _check(st, "isis_kick_drift")


# ---------------------------------------------------------------------------
# Background fields (initial guesses) and the paper's parameter presets (Table 1, Sect. 6.1)
# ---------------------------------------------------------------------------

def isis_background_field(model: int, params: Params, a: float, grid: Grid | None = None) -> float:
    """The model's uniform background field at expansion factor a (the library's ISIS_INIT_BACKGROUND value)."""
    lib = load()
    g = (grid or Grid(8, 1.0)).c()
    p = params.c()
    out = ctypes.c_double(0.0)
    st = lib.isis_background_field(int(model), ctypes.byref(p), ctypes.byref(g), float(a), ctypes.byref(out))
    _check(st, "isis_background_field")
    return out.value


def fofr_range(fR0_abs: float, n: int = 1, Omega_m: float = 0.267, Omega_L: float = 0.733) -> float:
    """Compton range of the f(R) field today in Mpc/h (Sect. 4.2):
    lambda = 3 sqrt((n+1)/(Om + 4 OL)) sqrt(|f_R0| / 1e-6)."""
    return 3.0 * ((n + 1) / (Omega_m + 4.0 * Omega_L)) ** 0.5 * (fR0_abs / 1e-6) ** 0.5


PRESETS = {
    # symmetron: lambda0 [Mpc/h], a_SSB = 1/(1+z_SSB), beta
    "SymmA": Params(lambda0=1.0, beta=1.0, a_ssb=1.0 / 2.0),
    "SymmB": Params(lambda0=1.0, beta=1.0, a_ssb=1.0 / 3.0),
    "SymmC": Params(lambda0=1.0, beta=2.0, a_ssb=1.0 / 2.0),
    "SymmD": Params(lambda0=1.0, beta=1.0, a_ssb=1.0 / 4.0),
    # Hu-Sawicki f(R): n, |f_R0|
    "fofr4": Params(n=1, fR0_abs=1e-4),
    "fofr5": Params(n=1, fR0_abs=1e-5),
    "fofr6": Params(n=1, fR0_abs=1e-6),
}


def selftest_exp_ff(x: torch.Tensor) -> torch.Tensor:
    """exp of a CUDA FP64 tensor through the library's float-float exponential (self-test)."""
    lib = load()
    fn = lib.isis_selftest_exp_ff
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    x = x.contiguous()
    y = torch.empty_like(x)
    st = fn(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), x.numel(),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise IsisError(st, strerror(st))
    return y


def selftest_ff_to_f64(hl: torch.Tensor) -> torch.Tensor:
    """FP64 values of float-float pairs (a CUDA float32 tensor of shape (n, 2): high, low) through the
    library's integer conversion (self-test)."""
    lib = load()
    fn = lib.isis_selftest_ff_to_f64
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    hl = hl.contiguous()
    out = torch.empty(hl.shape[0], dtype=torch.float64, device=hl.device)
    st = fn(ctypes.c_void_p(hl.data_ptr()), ctypes.c_void_p(out.data_ptr()), hl.shape[0],
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise IsisError(st, strerror(st))
    return out


def isis_patch_poisson_solve(grid: Grid, a: float, patch: Patch, parent: torch.Tensor, flags: torch.Tensor,
                             eta: torch.Tensor, Phi: torch.Tensor, tol: float = 1e-10, opts: Opts | None = None,
                             stream=None, allow_noconv: bool = False) -> Info:
    """Newtonian potential on a refinement patch (float64 tensors; flags uint8 of patch.n)."""
    lib = load()
    o = opts or Opts()
    g, b, oc, info = grid.c(), patch.c(), o.c(), isis_solve_info()
    st = lib.isis_patch_poisson_solve(ctypes.byref(g), a, ctypes.byref(b), _ptr(parent, torch.float64),
                                      _ptr(flags, torch.uint8), _ptr(eta, torch.float64), _ptr(Phi, torch.float64),
                                      tol, ctypes.byref(oc), ctypes.byref(info), _stream(stream))
    _check(st, "isis_patch_poisson_solve", (ISIS_OK, ISIS_ENOCONV) if allow_noconv else (ISIS_OK,))
    return _info(info, st, o.prec)


def isis_patch_scalar_solve(model: int, params: Params, grid: Grid, a: float, patch: Patch, parent: torch.Tensor,
                            flags: torch.Tensor, eta: torch.Tensor, phi: torch.Tensor, tol: float = 1e-10,
                            opts: Opts | None = None, stream=None, allow_noconv: bool = False) -> Info:
    """Symmetron or f(R) field on a refinement patch (float64 tensors; flags uint8 of patch.n)."""
    lib = load()
    o = opts or Opts()
    g, p, b, oc, info = grid.c(), params.c(), patch.c(), o.c(), isis_solve_info()
    st = lib.isis_patch_scalar_solve(int(model), ctypes.byref(p), ctypes.byref(g), a, ctypes.byref(b),
                                     _ptr(parent, torch.float64), _ptr(flags, torch.uint8), _ptr(eta, torch.float64),
                                     _ptr(phi, torch.float64), tol, ctypes.byref(oc), ctypes.byref(info),
                                     _stream(stream))
    _check(st, "isis_patch_scalar_solve", (ISIS_OK, ISIS_ENOCONV) if allow_noconv else (ISIS_OK,))
    return _info(info, st, o.prec)
