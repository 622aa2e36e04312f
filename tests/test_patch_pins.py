"""Pins of the oracle's refinement-patch solve (Sects. 3.3.1, 3.4.1; readings P1-P7 of isis_oracle.c).

- A linear field is an exact discrete solution when the density makes the source vanish (symmetron,
  Poisson) or equal the flux form's closed value on a linear u (f(R)); the trilinear interpolation of a
  linear parent is exact, so the patch solve must return the linear field at every unknown, for irregular
  masks, a periodic (domain) parent and a non-periodic (patch) parent.
- dL/du at an unknown, including the terms through the ghost values of masked neighbours (Eq. (ueq)),
  equals a central difference of L, for fractional masks.
- On a tiny patch the FAS fixed point equals a dense Newton solve (finite-difference Jacobian) of the
  unknowns with every other cell at its own trilinear interpolation of the parent.
"""
import math

import numpy as np
import pytest

import oracle

OM, OL = 0.267, 0.733
MODELS = [oracle.POISSON, oracle.SYMMETRON, oracle.FOFR]


def _fofr_consts(p):
    a, H02, r = p.a, p.H0 ** 2, OL / OM
    np1 = p.n + 1.0
    K1 = OM * a * H02
    K2 = OM * a ** 4 * H02 * (1 + 4 * r) * (p.fR0_abs * a * a) ** (1 / np1)
    K3 = OM * a * H02 * (1 + 4 * a ** 3 * r)
    return K1, K2, K3, np1


def _centres(n, o, h):
    """Cell-centre coordinates of a box of n cells starting at cell o of a grid of spacing h."""
    return [(o[a] + np.arange(n[a]) + 0.5) * h for a in range(3)]


def _linear(xs, c0, g):
    return c0 + g[0] * xs[0][:, None, None] + g[1] * xs[1][None, :, None] + g[2] * xs[2][None, None, :]


def _flags(n, seed, frac=0.6):
    rng = np.random.default_rng(seed)
    f = (rng.random(n) < frac).astype(np.uint8)
    f[0, :, :] = f[-1, :, :] = 0
    f[:, 0, :] = f[:, -1, :] = 0
    f[:, :, 0] = f[:, :, -1] = 0
    return f


def _linear_case(model, periodic):
    N, box = 16, 32.0
    p = oracle.Problem(model, N, box, a=1.0, a_ssb=0.5, lambda0=1.0, n=1, fR0_abs=1e-5)
    if periodic:
        level, pn, o, n = 1, (N, N, N), (3, 4, 2), (8, 6, 10)
    else:
        level, pn, o, n = 2, (20, 18, 22), (3, 2, 5), (12, 10, 12)
    hp = box / (N * 2 ** (level - 1))
    h = hp / 2
    if model == oracle.POISSON:
        c0, g = 0.3, (0.02, -0.01, 0.015)
    elif model == oracle.SYMMETRON:
        c0, g = 0.5, (0.004, -0.003, 0.005)
    else:
        K1, K2, K3, np1 = _fofr_consts(p)
        c0, g = np1 * math.log(K2 / K3) - 0.01, (0.0006, -0.0004, 0.0005)
    xs_p = _centres(pn, (0, 0, 0), hp)
    parent = _linear(xs_p, c0, g)
    nf = tuple(2 * v for v in n)
    xs_f = [(o[a] * hp + (np.arange(nf[a]) + 0.5) * h) for a in range(3)]
    uf = _linear(xs_f, c0, g)
    if model == oracle.POISSON:
        eta = np.full(nf, 1.3)
    elif model == oracle.SYMMETRON:
        s = (p.a_ssb / p.a) ** 3
        eta = (1.0 - uf ** 2) / s
    else:
        # the flux form on a linear u: sum over axes of g e^u sinh(g h) / h
        D = np.exp(uf) * sum(ga * math.sinh(ga * h) / h for ga in g)
        eta = 1.0 + (D + K2 * np.exp(-uf / np1) - K3) / K1
    assert eta.min() > 0
    patch = oracle.Patch(n, o, pn, periodic, level=level, eta_mean=1.3)
    return p, patch, parent, eta, uf


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("model", MODELS)
def test_patch_linear_field_is_exact(model, periodic):
    p, patch, parent, eta, uf = _linear_case(model, periodic)
    flags = _flags(patch.n, seed=5 + model)
    # start off the answer (the interpolated parent already is the linear field)
    u0 = uf + np.random.default_rng(1).normal(0.0, 0.01, uf.shape)
    # a fixed 40 cycles (tol 0): the residual reaches its rounding floor after about 20
    r = oracle.patch_solve(p, patch, parent, flags, eta, u0=u0, tol=0.0, max_cycles=40)
    assert r.status == oracle.ENOCONV and r.cycles == 40
    # every cell: the unknowns solved, the rest interpolated from the parent
    scale = np.abs(uf).max()
    assert np.abs(r.phi - uf).max() <= 1e-11 * max(scale, 1.0)
    assert r.cycles >= 1 and r.res0 > r.res_final  # the start was not already the answer


@pytest.mark.parametrize("model", MODELS)
def test_patch_derivative_includes_ghost_terms(model):
    rng = np.random.default_rng(11 + model)
    n = (8, 7, 9)
    m = rng.uniform(-1.0, 1.0, n)
    m[np.abs(m) < 0.05] = 0.3
    for ax in range(3):
        sl = [slice(None)] * 3
        for e in (0, -1):
            sl[ax] = e
            m[tuple(sl)] = -rng.uniform(0.0, 1.0, m[tuple(sl)].shape)
    p = oracle.Problem(model, 16, 16.0, a=1.0, a_ssb=0.5, lambda0=1.0, n=1, fR0_abs=1e-5)
    if model == oracle.FOFR:
        base = math.log(1e-5) + rng.normal(0, 0.3, n)
    else:
        base = 0.6 + rng.normal(0, 0.2, n)
    eta = rng.uniform(0.2, 3.0, n)
    u = base.copy()
    pre = base + rng.normal(0, 0.05, n)
    h = 0.7
    F, dF = oracle.patch_eval(p, h, m, eta, u, pre)
    unknowns = np.argwhere(m > 0)
    assert len(unknowns) > 50
    eps = 1e-6
    nghost = 0
    for (i, j, k) in unknowns:
        up, um = u.copy(), u.copy()
        up[i, j, k] += eps
        um[i, j, k] -= eps
        Fp, _ = oracle.patch_eval(p, h, m, eta, up, pre)
        Fm, _ = oracle.patch_eval(p, h, m, eta, um, pre)
        fd = (Fp[i, j, k] - Fm[i, j, k]) / (2 * eps)
        assert abs(fd - dF[i, j, k]) <= 1e-6 * abs(dF[i, j, k]), (i, j, k, fd, dF[i, j, k])
        nb = [m[i + 1, j, k], m[i - 1, j, k], m[i, j + 1, k], m[i, j - 1, k], m[i, j, k + 1], m[i, j, k - 1]]
        nghost += any(v <= 0 for v in nb)
    assert nghost > 20  # many cells next to masked cells


def _interp_numpy(parent, o, nf, periodic):
    """Cell-centred trilinear interpolation of the parent at the fine cells of a box (brute force)."""
    pn = parent.shape
    out = np.zeros(nf)
    for i in range(nf[0]):
        for j in range(nf[1]):
            for k in range(nf[2]):
                # fine cell centre in parent-cell coordinates (parent centres at integers + 1/2)
                x = [o[0] + (i + 0.5) / 2, o[1] + (j + 0.5) / 2, o[2] + (k + 0.5) / 2]
                lo = [int(math.floor(v - 0.5)) for v in x]
                t = [v - 0.5 - l for v, l in zip(x, lo)]
                v = 0.0
                for a in (0, 1):
                    for b in (0, 1):
                        for c in (0, 1):
                            idx = [lo[0] + a, lo[1] + b, lo[2] + c]
                            if periodic:
                                idx = [q % s for q, s in zip(idx, pn)]
                            w = (t[0] if a else 1 - t[0]) * (t[1] if b else 1 - t[1]) * (t[2] if c else 1 - t[2])
                            v += w * parent[tuple(idx)]
                out[i, j, k] = v
    return out


def _op_numpy(model, p, h, eta, u):
    """L(u) at every interior cell of a box, 7-point stencil (Sect. 3.1 / Eq. (disc_non_canonical))."""
    K1, K2, K3, np1 = _fofr_consts(p)
    A, s = p.a ** 2 / (2 * p.lambda0 ** 2), (p.a_ssb / p.a) ** 3
    KP = 1.5 * OM * p.H0 ** 2 / p.a
    c = u[1:-1, 1:-1, 1:-1]
    nbs = [u[2:, 1:-1, 1:-1], u[:-2, 1:-1, 1:-1], u[1:-1, 2:, 1:-1], u[1:-1, :-2, 1:-1], u[1:-1, 1:-1, 2:],
           u[1:-1, 1:-1, :-2]]
    e = eta[1:-1, 1:-1, 1:-1]
    if model == oracle.FOFR:
        flux = sum(0.5 * (np.exp(c) + np.exp(v)) * (v - c) for v in nbs) / h ** 2
        return flux - (K1 * (e - 1) - K2 * np.exp(-c / np1) + K3)
    lap = (sum(nbs) - 6 * c) / h ** 2
    if model == oracle.SYMMETRON:
        return lap - A * ((s * e - 1) * c + c ** 3)
    return lap - KP * (e - 1.1)


@pytest.mark.parametrize("model", MODELS)
def test_patch_fixed_point_matches_dense_newton(model):
    rng = np.random.default_rng(3 + model)
    N, box = 8, 16.0
    p = oracle.Problem(model, N, box, a=1.0, a_ssb=0.5, lambda0=1.0, n=1, fR0_abs=1e-5)
    pn, o, n = (N, N, N), (6, 1, 3), (4, 4, 4)  # wraps round the periodic parent along x
    flags = np.zeros(n, np.uint8)
    flags[1, 1, 1] = flags[2, 1, 1] = flags[1, 2, 1] = flags[2, 2, 2] = flags[1, 2, 2] = 1
    if model == oracle.FOFR:
        K1, K2, K3, np1 = _fofr_consts(p)
        parent = np1 * math.log(K2 / K3) + rng.normal(0, 0.2, pn)
    else:
        parent = 0.7 + rng.normal(0, 0.1, pn)
    nf = tuple(2 * v for v in n)
    eta = rng.uniform(0.3, 2.5, nf)
    patch = oracle.Patch(n, o, pn, True, level=1, eta_mean=1.1)
    r = oracle.patch_solve(p, patch, parent, flags, eta, tol=0.0, max_cycles=40)
    assert r.status == oracle.ENOCONV and r.hist[-1] <= 1e-12 * r.res0
    uint = _interp_numpy(parent, o, nf, True)
    m = np.repeat(np.repeat(np.repeat(flags, 2, 0), 2, 1), 2, 2) > 0
    idx = np.argwhere(m)
    h = box / (N * 2)

    def F(v):
        u = uint.copy()
        u[m] = v
        Lv = np.zeros(nf)
        Lv[1:-1, 1:-1, 1:-1] = _op_numpy(model, p, h, eta, u)
        return Lv[m]

    v = uint[m].copy()
    for _ in range(30):
        f0 = F(v)
        J = np.zeros((len(v), len(v)))
        for q in range(len(v)):
            d = 1e-6 * max(1.0, abs(v[q]))
            vp, vm = v.copy(), v.copy()
            vp[q] += d
            vm[q] -= d
            J[:, q] = (F(vp) - F(vm)) / (2 * d)
        dv = np.linalg.solve(J, -f0)
        v += dv
        if np.abs(dv).max() <= 1e-14 * max(1.0, np.abs(v).max()):
            break
    assert len(idx) == 40
    assert np.abs(r.phi[m] - v).max() <= 1e-10 * max(1.0, np.abs(v).max())
    assert np.abs(r.phi[~m] - uint[~m]).max() <= 1e-13 * max(1.0, np.abs(uint).max())


@pytest.mark.parametrize("model,a", [(oracle.POISSON, 0.7), (oracle.SYMMETRON, 0.9), (oracle.FOFR, 0.8),
                                     (oracle.CHAMELEON, 1.0)])
def test_patch_reference_residual_is_the_background_residual(model, a):
    """P7: the patch's ref is R6's closed form over its unknowns.  It must equal the RMS over the unknowns of L
    at the uniform background field, evaluated by the patch operator, with the domain mean for Poisson."""
    rng = np.random.default_rng(21 + model)
    n = (8, 6, 10)
    flags = (rng.uniform(size=n) < 0.5).astype(np.uint8)
    flags[0, :, :] = flags[-1, :, :] = 0
    flags[:, 0, :] = flags[:, -1, :] = 0
    flags[:, :, 0] = flags[:, :, -1] = 0
    nf = tuple(2 * v for v in n)
    eta = rng.uniform(0.2, 4.0, nf)
    p = oracle.Problem(model, 16, 16.0, a=a, a_ssb=0.5, cham_n=1.0)
    bg = oracle.background_field(model, a, a_ssb=0.5, cham_n=1.0)
    patch = oracle.Patch(n, (3, 4, 2), (16, 16, 16), True, level=1, eta_mean=1.3)
    r = oracle.patch_solve(p, patch, np.full((16, 16, 16), bg), flags, eta, tol=1.0, max_cycles=0)
    m = np.where(np.repeat(np.repeat(np.repeat(flags, 2, 0), 2, 1), 2, 2) > 0, 1.0, -1.0)
    u = np.full(nf, bg)
    F, _ = oracle.patch_eval(p, 16.0 / 32, m, eta, u, u, eta_mean=patch.eta_mean)
    rms = float(np.sqrt(np.mean(F[m > 0] ** 2)))
    assert rms > 0 and r.ref == pytest.approx(rms, rel=1e-12)


def test_patch_prolongation_reproduces_a_linear_correction():
    """P5: the cell-centred trilinear prolongation of a linear coarse correction is the same linear function at
    every fine unknown whose coarse stencil lies in the box; cells that are not unknowns are left alone, and at
    the box's edge the missing coarse cells contribute nothing (their weights are not redistributed)."""
    rng = np.random.default_rng(5)
    nc = (5, 4, 6)
    H = 1.0  # coarse cell size; fine h = 1/2
    g = rng.normal(size=3)
    ctr = [(np.arange(n) + 0.5) * H for n in nc]
    cdelta = 0.3 + g[0] * ctr[0][:, None, None] + g[1] * ctr[1][None, :, None] + g[2] * ctr[2][None, None, :]
    nf = tuple(2 * n for n in nc)
    m = np.where(rng.uniform(size=nf) < 0.7, 1.0, -0.5)
    out = oracle.patch_prolong_add(cdelta, m, np.zeros(nf))
    f = [(np.arange(n) + 0.5) * (H / 2) for n in nf]
    lin = 0.3 + g[0] * f[0][:, None, None] + g[1] * f[1][None, :, None] + g[2] * f[2][None, None, :]
    inside = np.ones(nf, bool)
    for ax, n in enumerate(nf):
        edge = np.zeros(n, bool)
        edge[0] = edge[-1] = True  # the first and last fine cells reach a coarse cell outside the box
        shape = [1, 1, 1]
        shape[ax] = n
        inside &= ~edge.reshape(shape)
    sel = inside & (m > 0)
    assert sel.sum() > 100
    assert np.abs(out[sel] - lin[sel]).max() <= 1e-13
    assert np.all(out[m <= 0] == 0.0)
    # at a corner unknown only the in-box coarse cell of each axis contributes: weight (3/4)^3
    c = (0, 0, 0)
    m2 = np.full(nf, -1.0)
    m2[c] = 1.0
    one = np.zeros(nc)
    one[0, 0, 0] = 1.0
    assert oracle.patch_prolong_add(one, m2, np.zeros(nf))[c] == 0.75 ** 3
