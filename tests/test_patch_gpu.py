"""Refinement patches on the GPU (Sects. 3.3.1, 3.4.1) against the oracle's patch solve, through the C ABI.

Same parent, flags and density on both sides: a level-1 patch over the periodic domain grid (its box
wrapping round the domain along one axis) and a level-2 patch over the level-1 patch.  FP64: max-abs
1e-10 after a fixed number of cycles and after convergence (same cycle count).  FP32 correction cycles in
FP64 defect correction (ISIS_F32_REFINE64): relative L2 over the unknowns within 1e-9 of the oracle's
solution, both converged (the library to 1e-11, the oracle to 5e-12: its FP64 floor on the f(R) level-2
patch is 2.9e-12 of ref)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1307_6748_gb300 import synth

pytestmark = pytest.mark.gpu

N, BOX, A1 = 32, 64.0, 1.0
MODELS = [oracle.POISSON, oracle.SYMMETRON, oracle.FOFR]


def _flags(eta_box, thr):
    f = (eta_box >= thr).astype(np.uint8)
    f[0, :, :] = f[-1, :, :] = 0
    f[:, 0, :] = f[:, -1, :] = 0
    f[:, :, 0] = f[:, :, -1] = 0
    return f


def _prob(model):
    return oracle.Problem(model, N, BOX, a=A1)


def _domain(model):
    eta = synth.lognormal_eta(N, BOX, 1.0, 4).numpy()
    if model == oracle.POISSON:
        g0 = np.zeros((N,) * 3)
    elif model == oracle.SYMMETRON:
        g0 = np.full((N,) * 3, np.sqrt(1 - 0.5 ** 3))
    else:
        r = 0.733 / 0.267
        g0 = np.log(1e-5 * ((1 + 4 * r) / (eta + 4 * r)) ** 2)
    sol = oracle.solve(_prob(model), eta, g0, tol=1e-10)
    assert sol.status == oracle.OK
    return eta, sol.phi


def _fine_eta(shape, seed):
    # a density field at the patch resolution (a lognormal realisation cut to the box)
    e = synth.lognormal_eta(2 * N, BOX, 1.0, seed).numpy()
    return np.ascontiguousarray(e[:shape[0], :shape[1], :shape[2]])


def _run_both(isis, model, patch_o, parent, flags, eta_f, tol, max_cycles, init_parent=True, prec=None,
              tol_oracle=None):
    # oracle
    ro = oracle.patch_solve(_prob(model), patch_o, parent, flags, eta_f, tol=tol if tol_oracle is None else tol_oracle,
                            max_cycles=max_cycles)
    # GPU
    patch = isis.Patch(patch_o.n, patch_o.o, patch_o.pn, patch_o.periodic, level=patch_o.level,
                       eta_mean=patch_o.eta_mean)
    phi = torch.zeros(patch.fine_shape, dtype=torch.float64, device="cuda")
    opts = isis.Opts(max_cycles=max_cycles, init=isis.ISIS_INIT_PARENT if init_parent else isis.ISIS_INIT_INPUT,
                     prec=isis.ISIS_F64 if prec is None else prec, inner_cycles=4)
    args = (isis.Grid(N, BOX), A1, patch, torch.from_numpy(parent).cuda(), torch.from_numpy(flags).cuda(),
            torch.from_numpy(eta_f).cuda(), phi)
    if model == oracle.POISSON:
        info = isis.isis_patch_poisson_solve(*args, tol=tol, opts=opts, allow_noconv=True)
    else:
        m = isis.ISIS_SYMMETRON if model == oracle.SYMMETRON else isis.ISIS_FOFR_HS
        info = isis.isis_patch_scalar_solve(m, isis.Params(), *args, tol=tol, opts=opts, allow_noconv=True)
    torch.cuda.synchronize()
    return ro, info, phi.cpu().numpy()


def _level1(model):
    eta, parent = _domain(model)
    o, n = (26, 6, 10), (12, 10, 14)  # wraps round the domain along x
    box_eta = np.take(eta, [(o[0] + i) % N for i in range(n[0])], axis=0)[:, o[1]:o[1] + n[1], o[2]:o[2] + n[2]]
    flags = _flags(box_eta, 1.0)
    assert 10 < flags.sum() < flags.size // 2
    patch = oracle.Patch(n, o, (N, N, N), True, level=1, eta_mean=float(eta.mean()))
    return patch, parent, flags, _fine_eta(tuple(2 * v for v in n), 9)


@pytest.mark.parametrize("model", MODELS)
def test_patch_level1_fixed_cycles(cuda_lib, model):
    isis = cuda_lib
    patch, parent, flags, eta_f = _level1(model)
    ro, info, got = _run_both(isis, model, patch, parent, flags, eta_f, tol=0.0, max_cycles=3)
    assert ro.status == oracle.ENOCONV and info.status == isis.ISIS_ENOCONV and info.cycles == ro.cycles == 3
    assert np.abs(got - ro.phi).max() <= 1e-10 * max(1.0, np.abs(ro.phi).max())
    np.testing.assert_allclose(info.hist, ro.hist, rtol=1e-6)
    assert abs(info.res_ref - ro.ref) <= 1e-12 * ro.ref


@pytest.mark.parametrize("model", MODELS)
def test_patch_levels_1_and_2_converged(cuda_lib, model):
    isis = cuda_lib
    patch, parent, flags, eta_f = _level1(model)
    ro, info, got = _run_both(isis, model, patch, parent, flags, eta_f, tol=1e-10, max_cycles=60)
    assert ro.status == oracle.OK and info.status == isis.ISIS_OK and info.cycles == ro.cycles
    assert np.abs(got - ro.phi).max() <= 1e-10 * max(1.0, np.abs(ro.phi).max())
    # level 2 inside level 1, with the oracle's level-1 field as parent
    nf = tuple(2 * v for v in patch.n)
    o2, n2 = (4, 3, 6), (14, 12, 14)
    e1 = eta_f[o2[0]:o2[0] + n2[0], o2[1]:o2[1] + n2[1], o2[2]:o2[2] + n2[2]]
    flags2 = _flags(e1, 1.2)
    assert flags2.sum() > 10
    p2 = oracle.Patch(n2, o2, nf, False, level=2, eta_mean=patch.eta_mean)
    ro2, info2, got2 = _run_both(isis, model, p2, ro.phi, flags2, _fine_eta(tuple(2 * v for v in n2), 12),
                                 tol=1e-10, max_cycles=60)
    assert ro2.status == oracle.OK and info2.status == isis.ISIS_OK and info2.cycles == ro2.cycles
    assert np.abs(got2 - ro2.phi).max() <= 1e-10 * max(1.0, np.abs(ro2.phi).max())


def _rel_l2(got, ref, unk):
    return float(np.linalg.norm(got[unk] - ref[unk]) / np.linalg.norm(ref[unk]))


def _unknowns(flags):
    return np.repeat(np.repeat(np.repeat(flags, 2, 0), 2, 1), 2, 2) > 0


@pytest.mark.parametrize("model", MODELS)
def test_patch_refine64_levels_1_and_2(cuda_lib, model):
    isis = cuda_lib
    patch, parent, flags, eta_f = _level1(model)
    ro, info, got = _run_both(isis, model, patch, parent, flags, eta_f, tol=1e-11, max_cycles=60,
                              prec=isis.ISIS_F32_REFINE64, tol_oracle=5e-12)
    assert ro.status == oracle.OK and info.status == isis.ISIS_OK and info.outer >= 1
    assert info.res_final <= 1e-11 * info.res_ref and info.cycles <= 4 * info.outer
    assert _rel_l2(got, ro.phi, _unknowns(flags)) <= 1e-9
    # the cells that are not unknowns hold the interpolated parent on both sides
    assert np.abs(got[~_unknowns(flags)] - ro.phi[~_unknowns(flags)]).max() <= 1e-12 * max(1.0, np.abs(ro.phi).max())
    # level 2 inside level 1, with the oracle's level-1 field as parent
    nf = tuple(2 * v for v in patch.n)
    o2, n2 = (4, 3, 6), (14, 12, 14)
    e1 = eta_f[o2[0]:o2[0] + n2[0], o2[1]:o2[1] + n2[1], o2[2]:o2[2] + n2[2]]
    flags2 = _flags(e1, 1.2)
    p2 = oracle.Patch(n2, o2, nf, False, level=2, eta_mean=patch.eta_mean)
    ro2, info2, got2 = _run_both(isis, model, p2, ro.phi, flags2, _fine_eta(tuple(2 * v for v in n2), 12),
                                 tol=1e-11, max_cycles=60, prec=isis.ISIS_F32_REFINE64, tol_oracle=5e-12)
    assert ro2.status == oracle.OK and info2.status == isis.ISIS_OK and info2.outer >= 1
    assert _rel_l2(got2, ro2.phi, _unknowns(flags2)) <= 1e-9


def test_patch_input_guess_and_argument_checks(cuda_lib):
    isis = cuda_lib
    patch, parent, flags, eta_f = _level1(oracle.SYMMETRON)
    ro = oracle.patch_solve(_prob(oracle.SYMMETRON), patch, parent, flags, eta_f, tol=1e-10, max_cycles=60)
    P = isis.Patch(patch.n, patch.o, patch.pn, True, level=1)
    args = [isis.Grid(N, BOX), A1, P, torch.from_numpy(parent).cuda(), torch.from_numpy(flags).cuda(),
            torch.from_numpy(eta_f).cuda()]
    # ISIS_INIT_INPUT from the converged answer: already converged, zero cycles, masked cells re-interpolated
    phi = torch.from_numpy(ro.phi.copy()).cuda()
    info = isis.isis_patch_scalar_solve(isis.ISIS_SYMMETRON, isis.Params(), *args, phi, tol=1e-10)
    assert info.cycles == 0 and np.abs(phi.cpu().numpy() - ro.phi).max() <= 1e-12
    # flags on the outer layer of the box, odd sizes, a periodic parent above level 1, F32
    bad = flags.copy()
    bad[0, 3, 3] = 1
    a2 = list(args)
    a2[4] = torch.from_numpy(bad).cuda()
    with pytest.raises(isis.IsisError):
        isis.isis_patch_scalar_solve(isis.ISIS_SYMMETRON, isis.Params(), *a2, phi)
    for Pbad in (isis.Patch((11, 10, 14), patch.o, patch.pn, True, level=1),
                 isis.Patch(patch.n, patch.o, patch.pn, True, level=2)):
        a3 = list(args)
        a3[2] = Pbad
        with pytest.raises(isis.IsisError):
            isis.isis_patch_scalar_solve(isis.ISIS_SYMMETRON, isis.Params(), *a3, phi)
    with pytest.raises(isis.IsisError):
        isis.isis_patch_scalar_solve(isis.ISIS_SYMMETRON, isis.Params(), *args, phi,
                                     opts=isis.Opts(prec=isis.ISIS_F32))
    with pytest.raises(isis.IsisError):
        isis.isis_patch_scalar_solve(isis.ISIS_SYMMETRON, isis.Params(), *args, phi,
                                     opts=isis.Opts(prec=isis.ISIS_F32_REFINE64, inner_cycles=0))
