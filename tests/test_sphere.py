"""The static sphere test of Sect. 5.1 on the FP64 oracle: the 3D solution on the paper's 128^3 domain grid
against the 1D spherically symmetric profile, band by band, and its error falling when h halves (64^3 ->
128^3).  The GPU versions are in test_sphere_gpu.py."""
import math

import pytest

import oracle
import sphere_cases as SC


@pytest.mark.parametrize("name", sorted(SC.TOL_128))
def test_oracle_sphere_profile_converges(name):
    errs = {}
    for N in (64, 128):
        eta = SC.eta_3d(name, N)
        r = oracle.solve(SC.problem(name, N), eta, SC.guess_3d(name, eta), tol=1e-10)
        assert r.status == oracle.OK
        errs[N] = SC.band_errors(name, r.phi, N)
    SC.check_tol(name, errs[128])
    SC.check_ratio(name, errs[64], errs[128])


def test_sphere_cases_match_the_golden_table():
    c = SC.cases()
    assert sorted(c) == ["fofr_z0", "symmetron_z0", "symmetron_z1"]
    assert c["symmetron_z1"]["a"] == 0.5 and c["symmetron_z0"]["params"] == dict(lambda0=1.0, a_ssb=0.6)
    assert c["fofr_z0"]["params"] == dict(n=1, fR0_abs=1e-6) and c["fofr_z0"]["B"] == 100.0
    # the far-field plateaus quoted for this set-up (uniform solution at the exterior density)
    assert abs(SC.far_value(c["symmetron_z0"]) - 0.988959) < 1e-6
    assert abs(SC.far_value(c["symmetron_z1"]) - 0.907917) < 1e-6
    assert abs(math.exp(SC.far_value(c["fofr_z0"])) / 1.13268e-6 - 1.0) < 1e-5  # |f_R| far, a = 1


@pytest.mark.parametrize("name", sorted(SC.TOL_128))
def test_oracle_sphere_refinement_levels(name):
    """Two refinement levels over the 128^3 domain (the paper's set-up of Sect. 5.1): closer to the 1D profile."""
    levels = SC.oracle_levels(name)
    assert len(levels) == 3
    SC.check_levels(name, [SC.level_errors(name, *lv) for lv in levels])
