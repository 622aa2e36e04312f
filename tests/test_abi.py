"""The CUDA library builds, loads without a GPU and exports every function that
include/isis.h declares; host-side argument checks need no device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(isis_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1307_6748_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 6
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_the_headers(lib):
    from paper_1307_6748_gb300 import isis, unet
    unet._lib()  # binds the learned-guess entry points
    bound = set(isis.EXPORTS) | {n for n in declared() if n.startswith("isis_unet_")}
    assert sorted(bound) == declared()
    for n in declared():
        if n.startswith("isis_unet_"):
            assert getattr(isis.load(), n).argtypes is not None, n


def test_strerror_and_argument_checks_without_gpu(lib):
    from paper_1307_6748_gb300 import isis
    L = isis.load()
    assert isis.strerror(isis.ISIS_ENOCONV) == "no convergence within max_cycles"
    g = isis.isis_grid(0.267, 0.733, isis.H0_MPC, 64.0, 48)  # N not a power of two
    p = isis.isis_params(1.0, 1.0, 0.5, 1, 1e-5)
    st = L.isis_scalar_solve(isis.ISIS_SYMMETRON, ctypes.byref(p), ctypes.byref(g), 1.0, ctypes.c_void_p(16),
                             ctypes.c_void_p(16), 1e-8, None, None, None)
    assert st == isis.ISIS_EINVAL
    g.N = 64
    st = L.isis_scalar_solve(7, ctypes.byref(p), ctypes.byref(g), 1.0, ctypes.c_void_p(16), ctypes.c_void_p(16),
                             1e-8, None, None, None)
    assert st == isis.ISIS_EINVAL
    st = L.isis_cic_deposit(ctypes.byref(g), None, None, None, 10, None, 1, None)
    assert st == isis.ISIS_EINVAL
    # no particles, or more than 2^40, are rejected before any device work
    dev = ctypes.c_void_p(16)
    for npart in (0, -1, (1 << 40) + 1):
        assert L.isis_cic_deposit(ctypes.byref(g), dev, dev, dev, npart, dev, 1, None) == isis.ISIS_EINVAL


def test_patch_argument_checks_without_gpu(lib):
    """The refinement-patch entry points reject bad boxes and options on the host, before any device call."""
    from paper_1307_6748_gb300 import isis
    L = isis.load()
    g = isis.isis_grid(0.267, 0.733, isis.H0_MPC, 64.0, 16)
    p = isis.isis_params(1.0, 1.0, 0.5, 1, 1e-5, 1.0)
    dev = ctypes.c_void_p(16)  # never dereferenced: every case fails its host checks first

    def call(box, opts=None, a=1.0, tol=1e-10):
        o = None if opts is None else ctypes.byref(opts.c())
        return L.isis_patch_scalar_solve(isis.ISIS_SYMMETRON, ctypes.byref(p), ctypes.byref(g), a, ctypes.byref(box),
                                         dev, dev, dev, dev, tol, o, None, None)

    def box(n=(8, 8, 8), o=(0, 0, 0), pn=(16, 16, 16), periodic=1, level=1):
        return isis.Patch(n, o, pn, bool(periodic), level=level).c()

    E = isis.ISIS_EINVAL
    assert call(box(), isis.Opts(prec=isis.ISIS_F32)) == E  # FP32 fields: not offered on patches
    assert call(box(), isis.Opts(prec=isis.ISIS_F32_REFINE64, inner_cycles=0)) == E
    assert call(box(), isis.Opts(prec=isis.ISIS_F32_REFINE64, inner_cycles=17)) == E
    assert call(box(), isis.Opts(nu1=17)) == E
    assert call(box(), isis.Opts(max_cycles=129)) == E
    assert call(box(), isis.Opts(init=isis.ISIS_INIT_BACKGROUND)) == E
    assert call(box(), a=0.0) == E and call(box(), tol=-1.0) == E
    assert call(box(n=(7, 8, 8))) == E and call(box(n=(2, 8, 8))) == E  # odd, too small
    assert call(box(level=0)) == E and call(box(level=2)) == E  # a periodic parent is the domain: level 1
    assert call(box(n=(18, 8, 8))) == E  # wider than the periodic parent
    # a non-periodic parent keeps one cell on each side
    assert call(box(o=(0, 1, 1), pn=(20, 20, 20), periodic=0, level=2)) == E
    assert call(box(o=(12, 1, 1), pn=(20, 20, 20), periodic=0, level=2)) == E
    # the coarsest patch level (one block) holds at most 32768 cells: 2 x 66 -> 66 -> 33 (odd) is 35937
    g.N = 128
    assert call(box(n=(66, 66, 66), pn=(128, 128, 128))) == E


def test_solver_option_and_parameter_checks_without_gpu(lib):
    """The grid, the options and the model parameters of the domain solves are checked on the host."""
    from paper_1307_6748_gb300 import isis
    L = isis.load()
    dev = ctypes.c_void_p(16)  # never dereferenced
    E = isis.ISIS_EINVAL

    def solve(model=isis.ISIS_SYMMETRON, N=16, box=32.0, opts=None, params=None, a=1.0, Om=0.267):
        g = isis.isis_grid(Om, 0.733, isis.H0_MPC, box, N)
        p = (params or isis.Params()).c()
        o = None if opts is None else ctypes.byref(opts.c())
        return L.isis_scalar_solve(model, ctypes.byref(p), ctypes.byref(g), a, dev, dev, 1e-8, o, None, None)

    for N in (4, 12, 2048):
        assert solve(N=N) == E  # a power of two in [8, 1024]
    assert solve(box=0.0) == E and solve(Om=0.0) == E and solve(a=-1.0) == E
    for o in (isis.Opts(n_coarsest=3), isis.Opts(nu1=17), isis.Opts(nu2=-1), isis.Opts(max_cycles=129),
              isis.Opts(prec=5), isis.Opts(inner_cycles=0), isis.Opts(inner_cycles=17), isis.Opts(init=9),
              isis.Opts(fmg=2), isis.Opts(init=isis.ISIS_INIT_PARENT)):
        assert solve(opts=o) == E, o
    assert solve(params=isis.Params(lambda0=0.0)) == E
    assert solve(params=isis.Params(a_ssb=-0.5)) == E
    assert solve(model=isis.ISIS_FOFR_HS, params=isis.Params(fR0_abs=0.0)) == E
    assert solve(model=isis.ISIS_FOFR_HS, params=isis.Params(n=0)) == E
    assert solve(model=isis.ISIS_CHAMELEON, params=isis.Params(cham_n=-1.0)) == E


def test_host_buffer_argument_checks_without_gpu(lib):
    """isis_host_alloc / isis_host_free reject what they must before any driver call."""
    from paper_1307_6748_gb300 import isis
    L = isis.load()
    out = ctypes.c_void_p()
    assert L.isis_host_alloc(0, ctypes.byref(out)) == isis.ISIS_EINVAL
    assert out.value is None
    assert L.isis_host_alloc(64, None) == isis.ISIS_EINVAL
    assert L.isis_host_alloc((1 << 64) - 1, ctypes.byref(out)) == isis.ISIS_EINVAL
    assert L.isis_host_free(None) == isis.ISIS_OK
    # a pointer the allocator did not return
    buf = (ctypes.c_ubyte * 64)()
    assert L.isis_host_free(ctypes.addressof(buf)) == isis.ISIS_EINVAL
