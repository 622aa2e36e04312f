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
