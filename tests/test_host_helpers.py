"""Host-side helpers of the package (no GPU): the background fields the solves start from, against the
oracle's uniform-density solutions; the sphere workload's densities and radial profile; the density
recipes' normalisation."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import sphere1d
from paper_1307_6748_gb300 import isis, sphere, synth


@pytest.mark.gpu
@pytest.mark.parametrize("a", [0.3, 0.5, 0.8, 1.0])
def test_background_fields_match_the_oracle(cuda_lib, a):
    """The library's background fields (isis_background_field, the ISIS_INIT_BACKGROUND values) against the
    oracle's uniform-density solutions."""
    bgf = isis.isis_background_field
    assert bgf(isis.ISIS_SYMMETRON, isis.Params(a_ssb=0.5), a) == pytest.approx(
        oracle.background_field(oracle.SYMMETRON, a, a_ssb=0.5), abs=1e-15)
    for n, f in ((1, 1e-5), (2, 1e-6)):
        assert bgf(isis.ISIS_FOFR_HS, isis.Params(n=n, fR0_abs=f), a) == pytest.approx(
            oracle.background_field(oracle.FOFR, a, n=n, fR0_abs=f), rel=1e-14)
    for cn in (-0.5, 1.0, 2.0):
        assert bgf(isis.ISIS_CHAMELEON, isis.Params(cham_n=cn, lambda0=2.0), a) == pytest.approx(
            oracle.background_field(oracle.CHAMELEON, a, cham_n=cn), abs=1e-15)


def test_sphere_exterior_density_keeps_the_mean():
    for delta, R, B in ((5000.0, 3.0, 40.0), (5000.0, 5.0, 100.0), (10.0, 1.0, 8.0)):
        eta_in, eta_out = sphere1d.sphere_densities(delta, R, B)
        assert sphere.exterior_density(delta, R, B) == pytest.approx(eta_out, rel=1e-15)
        v = 4.0 * math.pi / 3.0 * R ** 3
        assert (eta_in * v + eta_out * (B ** 3 - v)) / B ** 3 == pytest.approx(1.0, rel=1e-13)


@pytest.mark.parametrize("name", ["symmetron_z0", "fofr_z0"])
def test_radial_profile_of_a_constant_field(name):
    case = sphere.CASES[name]
    N, nbins, c = 16, 8, -0.75
    rows = sphere.radial_profile(case, torch.full((N,) * 3, c, dtype=torch.float64), nbins)
    want = c if case["model"] == "symmetron" else -math.exp(c) * (1.0 + case["z"]) ** 2
    assert np.allclose(rows[:, 1:], want, rtol=1e-14, atol=0.0)
    w = case["B"] / (2 * nbins)
    assert np.allclose(np.diff(rows[:, 0]) % w, 0.0, atol=1e-12) and rows[0, 0] >= 0.5 * w


def test_density_recipes_have_mean_one():
    e = synth.lognormal_eta(16, 32.0, 1.0, 5)
    assert float(e.mean()) == pytest.approx(1.0, rel=1e-12) and float(e.min()) > 0.0
    h1 = synth.nfw_eta(16, 32.0, 0.5, 5, nhalo=4)
    h2 = synth.nfw_eta(16, 32.0, 0.5, 5, nhalo=4)
    assert torch.equal(h1, h2)
    assert float(h1.mean()) == pytest.approx(1.0, rel=1e-12) and float(h1.min()) > 0.0
    # the haloes add mass concentrations beyond the lognormal field's
    assert float(h1.max()) > float(synth.lognormal_eta(16, 32.0, 0.5, 5).max())


def test_halo_density_recipe_is_high_contrast():
    """The halo workload's density (lognormal sigma = 1.5 plus 32 NFW haloes, 1 Mpc/h cells) has mean 1 and
    peaks above 1e3 in the haloes, with voids below 0.05."""
    eta = synth.nfw_eta(64, 64.0, 1.5, 1).numpy()
    assert abs(eta.mean() - 1.0) <= 1e-12
    assert eta.max() >= 1e3 and eta.min() < 0.05
    assert (eta > 0).all()


class _Ev:
    """A stand-in for a CUDA event: elapsed_time is the difference of two stamps."""

    def __init__(self, t):
        self.t = t

    def elapsed_time(self, other):
        return other.t - self.t


def test_copy_times_groups_copies_per_step():
    """bench.copy_times: the mean copy time per step and the slowest step, per loop and direction; the
    pipelined loop reads back each model's forces as its own group (two D2H groups per step)."""
    import bench
    ev = {"serial": [("h2d", _Ev(0), _Ev(7)), ("d2h", _Ev(0), _Ev(16)), ("h2d", _Ev(0), _Ev(9)),
                     ("d2h", _Ev(0), _Ev(100))],
          "pipelined": [("h2d", _Ev(0), _Ev(7)), ("h2d", _Ev(0), _Ev(8)), ("d2h", _Ev(0), _Ev(8)),
                        ("d2h", _Ev(0), _Ev(9)), ("d2h", _Ev(0), _Ev(50)), ("d2h", _Ev(0), _Ev(8))]}
    out = bench.copy_times(ev, 2)
    assert out["serial_h2d"] == {"mean": 8.0, "max_step": 9}
    assert out["serial_d2h"] == {"mean": 58.0, "max_step": 100}
    assert out["pipelined_h2d"] == {"mean": 7.5, "max_step": 8}
    assert out["pipelined_d2h"] == {"mean": 37.5, "max_step": 58}


def test_host_buffer_of_no_bytes_is_rejected():
    """isis.host_empty(0): isis_host_alloc refuses zero bytes before any driver call."""
    from paper_1307_6748_gb300 import build
    build.build()
    with pytest.raises(isis.IsisError):
        isis.host_empty(0)
