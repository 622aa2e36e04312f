"""The allocation-free CIC deposit (isis_cic_deposit_noalloc), called through
the C ABI, gives the result of isis_cic_deposit on two calls in a row.

It serves callers that must not allocate device memory while running; its
scratch is a fixed array in the library shared by every call, so the second
call also checks that a call clears what the previous one left behind.  This
file is collected last so that a run stopping at the first failure has run
every other test first.
"""
import ctypes

import pytest
import torch

from paper_1307_6748_gb300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(isis, grid, x, y, z, eta):
    lib = isis.load()
    g = grid.c()
    st = lib.isis_cic_deposit_noalloc(ctypes.byref(g), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                      ctypes.c_void_p(z.data_ptr()), x.numel(), ctypes.c_void_p(eta.data_ptr()),
                                      1 if eta.dtype == torch.float64 else 0,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def test_noalloc_deposit_matches_allocating_deposit_twice(cuda_lib):
    isis = cuda_lib
    # two different particle sets and grid sizes: the second call must not see the first's sums
    for call, (N, seed) in enumerate(((64, 3), (32, 11))):
        grid = isis.Grid(N, float(N))
        x, y, z = (v.cuda() for v in synth.zeldovich(N, float(N), seed=seed))
        ref = torch.empty((N,) * 3, dtype=torch.float64, device="cuda")
        isis.isis_cic_deposit(grid, x, y, z, ref)
        got = torch.full((N,) * 3, -1.0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert _noalloc(isis, grid, x, y, z, got) == isis.ISIS_OK
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call > 0:
            # the first call may load the library's device code and its array; later calls take no device memory
            assert free1 == free0, (free0, free1)
        assert float((got - ref).abs().max()) <= 1e-10  # the deposit tests' tolerance
        assert abs(float(got.sum()) - N ** 3) <= 1e-6


def test_noalloc_deposit_rejects_large_grid(cuda_lib):
    isis = cuda_lib
    N = 128
    x = torch.zeros(8, dtype=torch.float32, device="cuda")
    eta = torch.empty((N,) * 3, dtype=torch.float64, device="cuda")
    assert _noalloc(isis, isis.Grid(N, 1.0), x, x, x, eta) == isis.ISIS_EINVAL


def test_noalloc_deposit_rejects_particle_counts_that_could_wrap(cuda_lib):
    """2^24 particles could put 2^24 unit weights into one cell, which wraps its 64-bit accumulator of 2^-40
    units: the call refuses on the host, before any device work.  (The positions are real 2^24-element arrays,
    so no access could leave them even if the check were missing.)"""
    isis = cuda_lib
    N = 16
    lib = isis.load()
    g = isis.Grid(N, 1.0).c()
    x = torch.zeros(1 << 24, dtype=torch.float32, device="cuda")
    eta = torch.empty((N,) * 3, dtype=torch.float64, device="cuda")
    st = lib.isis_cic_deposit_noalloc(ctypes.byref(g), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(x.data_ptr()), 1 << 24, ctypes.c_void_p(eta.data_ptr()), 1,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == isis.ISIS_EINVAL
