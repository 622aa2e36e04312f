"""Host logic of the refinement levels (no GPU): the refine flags and patch boxes of synth.py, and the
patch-box argument rules of the C ABI as the oracle applies them."""
import numpy as np
import pytest

import oracle
from paper_1307_6748_gb300 import synth


def test_refine_flags_threshold_and_dilation():
    eta = np.ones((16, 16, 16))
    eta[8, 8, 8] = 9.0  # one cell above 8 mean-density domain cells
    f0 = synth.refine_flags(eta, 1, expand=0)
    assert f0.sum() == 1 and f0[8, 8, 8]
    f1 = synth.refine_flags(eta, 1, expand=1)  # the six face neighbours
    assert f1.sum() == 7 and f1[7, 8, 8] and f1[8, 9, 8] and f1[8, 8, 7] and not f1[7, 7, 8]
    assert synth.refine_flags(eta, 1, expand=2).sum() == 25
    # level 2 counts a level-1 cell as 1/8 of a domain cell: 9 is below 8 * 8
    assert synth.refine_flags(eta, 2, expand=0).sum() == 0
    eta[8, 8, 8] = 65.0
    assert synth.refine_flags(eta, 2, expand=0).sum() == 1
    # kept inside the parent's refined cells
    within = np.zeros_like(f1)
    within[8, 8, 8] = True
    assert synth.refine_flags(eta, 1, expand=1, within=within).sum() == 1


def test_refine_flags_periodic_dilation_wraps():
    eta = np.ones((8, 8, 8))
    eta[0, 0, 0] = 20.0
    f = synth.refine_flags(eta, 1, expand=1, periodic=True)
    assert f.sum() == 7 and f[7, 0, 0] and f[0, 0, 7] and f[1, 0, 0]
    g = synth.refine_flags(eta, 1, expand=1, periodic=False)
    assert g.sum() == 4 and not g[7, 0, 0]


@pytest.mark.parametrize("periodic", [True, False])
def test_patch_box_covers_flags_with_margin(periodic):
    rng = np.random.default_rng(4)
    pn = (40, 36, 44)
    f = np.zeros(pn, bool)
    f[12:19, 9:14, 20:31] = rng.random((7, 5, 11)) < 0.5
    f[12, 9, 20] = f[18, 13, 30] = True
    o, n = synth.patch_box(f, periodic=periodic)
    assert all(v % 8 == 0 for v in n)
    flags = synth.box_flags(f, o, n, periodic)
    assert flags.sum() == f.sum()  # every flag inside the box
    # the outer layer of the box is never flagged (the C ABI rejects that)
    assert not flags[0].any() and not flags[-1].any() and not flags[:, 0].any() and not flags[:, -1].any()
    assert not flags[:, :, 0].any() and not flags[:, :, -1].any()
    if not periodic:
        assert all(o[a] >= 1 and o[a] + n[a] + 1 <= pn[a] for a in range(3))


def test_patch_box_wraps_round_a_periodic_parent():
    f = np.zeros((32, 32, 32), bool)
    f[30:32, 5:8, 5:8] = True
    f[0:2, 5:8, 5:8] = True
    o, n = synth.patch_box(f, periodic=True)
    # the flags span x = 30..33 across the periodic edge: a box of 8 cells wrapping round it
    assert n[0] == 8 and (o[0] + n[0]) % 32 < o[0]
    flags = synth.box_flags(f, o, n, True)
    assert flags.sum() == f.sum()
    assert synth.patch_box(np.zeros((8, 8, 8), bool)) is None


def test_sphere_eta_box_matches_the_domain_recipe():
    N, B, R, delta = 32, 40.0, 3.0, 5000.0
    full = synth.sphere_eta(N, B, R, delta).numpy()
    h = B / N
    sub = synth.sphere_eta_box((8, 6, 10), (12 * h, 13 * h, 11 * h), h, B, R, delta)
    np.testing.assert_array_equal(sub, full[12:20, 13:19, 11:21])


def test_oracle_rejects_bad_patches():
    p = oracle.Problem(oracle.SYMMETRON, 16, 32.0)
    eta = np.ones((16, 16, 16))
    parent = np.zeros((16, 16, 16))
    good = np.zeros((8, 8, 8), np.uint8)
    good[3, 3, 3] = 1
    r = oracle.patch_solve(p, oracle.Patch((8, 8, 8), (2, 2, 2), (16, 16, 16), True), parent, good, eta, tol=1e-8)
    assert r.status == oracle.OK
    edge = good.copy()
    edge[0, 4, 4] = 1
    r = oracle.patch_solve(p, oracle.Patch((8, 8, 8), (2, 2, 2), (16, 16, 16), True), parent, edge, eta, tol=1e-8)
    assert r.status == oracle.EINVAL
    # a non-periodic parent needs one parent cell beyond the box on every side
    r = oracle.patch_solve(p, oracle.Patch((8, 8, 8), (0, 2, 2), (16, 16, 16), False, level=2), parent, good, eta,
                           tol=1e-8)
    assert r.status == oracle.EINVAL


def test_refine_builds_nested_levels_and_passes_the_precision(monkeypatch):
    """amr.refine's host flow with the library's patch solve replaced by a recorder: level 2 lies inside level 1,
    its parent is level 1's field, and the options carry the precision, inner cycles and parent start."""
    import torch

    from paper_1307_6748_gb300 import amr, isis
    calls = []

    def fake_solve(model, params, grid, a, patch, parent, flags, eta, phi, tol, opts, stream=None):
        calls.append(dict(patch=patch, parent=parent, flags=flags.clone(), opts=opts, model=model, tol=tol))
        phi.fill_(float(len(calls)))  # level l's field is l everywhere
        return isis.Info(isis.ISIS_OK, 1, 1, 0.0, 1.0, 0.0, [])

    monkeypatch.setattr(isis, "isis_patch_scalar_solve", fake_solve)
    N, B = 32, 64.0
    eta = np.ones((N, N, N))
    eta[14:18, 14:18, 14:18] = 600.0  # above 8 domain-cell masses at level 1 and 64 at level 2
    phi0 = torch.zeros((N, N, N), dtype=torch.float64)
    dens = lambda dims, corner, h: np.full(dims, 600.0)
    levels = amr.refine(isis.ISIS_SYMMETRON, isis.Params(), isis.Grid(N, B), 1.0, eta, phi0, dens, levels=2,
                        expand=1, tol=1e-9, prec=isis.ISIS_F32_REFINE64, inner_cycles=3)
    assert [lv.level for lv in levels] == [1, 2] and len(calls) == 2
    for c in calls:
        assert c["opts"].prec == isis.ISIS_F32_REFINE64 and c["opts"].inner_cycles == 3
        assert c["opts"].init == isis.ISIS_INIT_PARENT and c["tol"] == 1e-9
    p1, p2 = calls[0]["patch"], calls[1]["patch"]
    assert p1.periodic and p1.level == 1 and tuple(p1.parent_dims) == (N, N, N)
    assert not p2.periodic and p2.level == 2 and tuple(p2.parent_dims) == tuple(2 * v for v in p1.n)
    assert calls[1]["parent"] is levels[0].phi and calls[0]["parent"] is phi0
    # level 2's cells lie inside level 1's unknowns, and its fine cells are half the size
    assert levels[1].h == levels[0].h / 2
    o2 = np.array(p2.origin)
    inner = levels[0].unknowns[o2[0]:o2[0] + p2.n[0], o2[1]:o2[1] + p2.n[1], o2[2]:o2[2] + p2.n[2]]
    assert not (calls[1]["flags"].numpy().astype(bool) & ~inner).any()


def test_patch_box_without_room_for_the_rounding():
    """A non-periodic parent of 16 cells with flags at 2..13: the multiple of 8 (16) leaves no cell on each
    side, so the box takes the next even size (14) at origin 1; flags that reach the parent's edge raise."""
    f = np.zeros((16, 16, 16), bool)
    f[2:14, 2:14, 2:14] = True
    o, n = synth.patch_box(f, periodic=False)
    assert o == (1, 1, 1) and n == (14, 14, 14)
    assert synth.box_flags(f, o, n, False).sum() == f.sum()
    g = np.zeros((16, 16, 16), bool)
    g[0:5, 4:6, 4:6] = True
    with pytest.raises(ValueError):
        synth.patch_box(g, periodic=False)
