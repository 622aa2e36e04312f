"""Mutation tests of the oracle's pins: each case plants one plausible mistake in a copy of the oracle (a
dropped or wrong factor, a flipped sign, a wrong neighbour or offset, a wrong constant), in its C part or its
Python part, and runs the pin tests against that copy, which must fail.  The oracle stays pinned to facts
outside itself only if every such mistake is caught.  CPU only; the copies live in a temporary directory."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")

PINS = "tests/test_oracle_pins.py"
PATCH_PINS = "tests/test_patch_pins.py"
NET_PINS = "tests/test_unet_ref.py"

C, PY, SPH, NET = "isis_oracle.c", "__init__.py", "sphere1d.py", "unet_ref.py"

# (name, oracle file, exact text in it, its planted replacement, the pin file that must catch it)
MUTATIONS = [
    ("symmetron cubic term sign", C,
     "c->A * ((c->s * eta - 1.0) * phi + phi * phi * phi)",
     "c->A * ((c->s * eta - 1.0) * phi - phi * phi * phi)", PINS),
    ("symmetron derivative factor", C,
     "c->A * (c->s * eta - 1.0 + 3.0 * phi * phi)",
     "c->A * (c->s * eta - 1.0 + 2.0 * phi * phi)", PINS),
    ("Poisson source sign", C, "return c->KP * (eta - c->eta_mean);", "return -c->KP * (eta - c->eta_mean);", PINS),
    ("f(R) K3 power of a", C, "(1.0 + 4.0 * a * a * a * r)", "(1.0 + 4.0 * a * a * r)", PINS),
    ("f(R) face value: the cell's b instead of the face mean", C,
     "div += bf * (un - u);",
     "div += bu * (un - u);", PINS),
    ("f(R) derivative factor 1/2", C,
     "acc += -bf + 0.5 * bu * (un - u);\n    }\n    return acc / h2",
     "acc += -bf + bu * (un - u);\n    }\n    return acc / h2", PINS),
    ("f(R) source exponent", C, "c->K2 * exp(-phi / c->np1) + c->K3", "c->K2 * exp(-phi * c->np1) + c->K3", PINS),
    ("chameleon exponent", C, "c->np1 = 1.0 / (1.0 + p->cham_n);", "c->np1 = 1.0 + p->cham_n;", PINS),
    ("restriction weight", C, "coarse[IDX(NH, I, J, K)] = s / 8.0;", "coarse[IDX(NH, I, J, K)] = s / 4.0;", PINS),
    ("prolongation neighbour", C,
     "ci[1] = WRAP(i / 2 + ((i & 1) ? 1 : -1), NH);",
     "ci[1] = WRAP(i / 2 + ((i & 1) ? -1 : 1), NH);", PINS),
    ("CIC cell-centre offset", C, "double xs = x - 0.5;", "double xs = x;", PINS),
    ("gradient spacing", C,
     "gx[q] = (f[IDX(N, WRAP(i + 1, N), j, k)] - f[IDX(N, WRAP(i - 1, N), j, k)]) / (2.0 * h);",
     "gx[q] = (f[IDX(N, WRAP(i + 1, N), j, k)] - f[IDX(N, WRAP(i - 1, N), j, k)]) / h;", PINS),
    ("symmetron force constant power of a_SSB", C, "/ pow(p->a_ssb, 3.0);", "/ pow(p->a_ssb, 2.0);", PINS),
    ("FAS coarse source without L_H(R phi)", C,
     "C->sigma[IDX(C->N, i, j, k)] += op_L(&H->coef, C, C->phi, i, j, k);",
     "C->sigma[IDX(C->N, i, j, k)] += 0.0;", PINS),
    ("coarse correction without R phi", C, "C->phi0[q] = C->phi[q] - C->phi0[q];", "C->phi0[q] = C->phi[q];", PINS),
    ("Newton step sign", C, "L->phi[q] = L->phi[q] - F / dF;", "L->phi[q] = L->phi[q] + F / dF;", PINS),
    ("Poisson mean kept", C,
     "if (p->model == ORC_POISSON) remove_mean(p->N, phi);",
     "if (0) remove_mean(p->N, phi);", PINS),
    ("symmetron reference residual without s", C,
     "scale = H.coef.A * H.coef.s * background(p, &H.coef);\n"
     "    else if (H.coef.model == ORC_FOFR) scale = H.coef.K1;\n    else scale = H.coef.KP;\n"
     "    info->ref = scale * sqrt(sum2 / (double)n3);",
     "scale = H.coef.A * background(p, &H.coef);\n    else if (H.coef.model == ORC_FOFR) scale = H.coef.K1;\n"
     "    else scale = H.coef.KP;\n    info->ref = scale * sqrt(sum2 / (double)n3);", PINS),
    ("f(R) reference residual constant", C,
     "scale = H.coef.K1;\n    else scale = H.coef.KP;\n    info->ref = scale * sqrt(sum2 / (double)n3);",
     "scale = H.coef.K3;\n    else scale = H.coef.KP;\n    info->ref = scale * sqrt(sum2 / (double)n3);", PINS),
    ("CIC normalisation", C,
     "for (size_t q = 0; q < n3; ++q) eta[q] /= nbar;",
     "for (size_t q = 0; q < n3; ++q) eta[q] *= nbar;", PINS),
    ("f(R) K2 exponent", C, "pow(p->fR0_abs * a * a, 1.0 / c->np1)", "pow(p->fR0_abs * a * a, c->np1)", PINS),
    ("symmetron A", C,
     "c->A = a * a / (2.0 * p->lambda0 * p->lambda0);",
     "c->A = a * a / (p->lambda0 * p->lambda0);", PINS),
    ("chameleon force constant", C, "double Cc = 3.0 * (1.0 + p->cham_n)", "double Cc = 3.0 * (2.0 + p->cham_n)", PINS),
    ("f(R) force factor", C, "else pref = 0.5 * exp(phi[q]);", "else pref = exp(phi[q]);", PINS),
    ("force sign", C, "gx[q] = -acc[0];", "gx[q] = acc[0];", PINS),
    ("patch ghost: mask ratio sign", C, "*mu = mn / L->m[q];", "*mu = -mn / L->m[q];", PATCH_PINS),
    ("patch interpolation neighbour", C,
     "pc[a][1] = pc[a][0] + ((f[a] & 1) ? 1 : -1);",
     "pc[a][1] = pc[a][0] + ((f[a] & 1) ? -1 : 1);", PATCH_PINS),
    ("patch restriction weight", C,
     "coarse[PIDX(nc, I, J, K)] = s / 8.0;",
     "coarse[PIDX(nc, I, J, K)] = s / 4.0;", PATCH_PINS),
    ("patch prolongation neighbour", C,
     "int ci[2] = {i / 2, i / 2 + ((i & 1) ? 1 : -1)};",
     "int ci[2] = {i / 2, i / 2 + ((i & 1) ? -1 : 1)};", PATCH_PINS),
    ("patch prolongation weights", C,
     "double w[2] = {0.75, 0.25}, v = 0.0;\n        for (int a = 0; a < 2; ++a)\n"
     "          for (int b = 0; b < 2; ++b)\n            for (int d = 0; d < 2; ++d) {",
     "double w[2] = {0.5, 0.5}, v = 0.0;\n        for (int a = 0; a < 2; ++a)\n"
     "          for (int b = 0; b < 2; ++b)\n            for (int d = 0; d < 2; ++d) {", PATCH_PINS),
    ("patch reference residual without s", C,
     "scale = H.coef.A * H.coef.s * background(p, &H.coef);\n"
     "    else if (H.coef.model == ORC_FOFR) scale = H.coef.K1;\n    else scale = H.coef.KP;\n    info->ref = cnt",
     "scale = H.coef.A * background(p, &H.coef);\n    else if (H.coef.model == ORC_FOFR) scale = H.coef.K1;\n"
     "    else scale = H.coef.KP;\n    info->ref = cnt", PATCH_PINS),
    ("patch Poisson reference density", C,
     "double eref = (p->model == ORC_POISSON) ? P->eta_mean : 1.0, s2 = 0.0;",
     "double eref = 1.0, s2 = 0.0;", PATCH_PINS),
    ("patch ghost: the neighbour's u^Pre", C,
     "(*mu) * (L->u[q] - L->pre[q]);",
     "(*mu) * (L->u[qn] - L->pre[qn]);", PATCH_PINS),
    ("patch f(R) ghost derivative factor", C,
     "dacc += mu * (0.5 * bn * (un - u) + bf);",
     "dacc += mu * (bn * (un - u) + bf);", PATCH_PINS),
    ("patch f(R) derivative factor 1/2", C,
     "dacc += -bf + 0.5 * bu * (un - u);",
     "dacc += -bf + bu * (un - u);", PATCH_PINS),
    ("coarsest Jacobian: f(R) off-diagonal derivative factor", C,
     "J[row * n + col] += (bf + 0.5 * bn * (un - u)) / h2;",
     "J[row * n + col] += (bf + bn * (un - u)) / h2;", PINS),
    ("coarsest Jacobian: f(R) off-diagonal without the face mean", C,
     "J[row * n + col] += (bf + 0.5 * bn * (un - u)) / h2;",
     "J[row * n + col] += (0.5 * bn + 0.5 * bn * (un - u)) / h2;", PINS),
    ("coarsest Jacobian: Poisson null-space shift", C,
     "double shift = 6.0 / h2 / (double)n;",
     "double shift = 12.0 / h2 / (double)n;", PINS),
    ("coarsest Newton: OK without meeting the stop rule", C,
     "int st = ORC_ENOCONV, it;", "int st = ORC_OK, it;", PINS),
    ("RMS residual normalisation", C,
     "return sqrt(tot / ((double)N * N * N));", "return sqrt(tot / ((double)N * N));", PINS),
    ("CIC weights swapped", C, "*w0 = 1.0 - t;\n  *w1 = t;", "*w0 = t;\n  *w1 = 1.0 - t;", PINS),
    ("symmetron force without a^2", C, "pref = Cs * (a * phi[q]) * a;", "pref = Cs * phi[q];", PINS),
    ("force gather weight", C, "double w = wx[aa] * wy[b] * wz[d];", "double w = wx[aa] * wy[b] * wz[1 - d];", PINS),
    ("1D face area", SPH,
     "area = self.edges[1:] ** 2  # outer face of cell i",
     "area = self.edges[1:] ** 1  # outer face of cell i", PINS),
    ("1D symmetron cubic term", SPH,
     "F = L - A * ((s * eta - 1.0) * u + u ** 3)",
     "F = L - A * ((s * eta - 1.0) * u + u ** 2)", PINS),
    ("1D f(R) face: the inner cell's b", SPH, "bf = 0.5 * (be[:-1] + be[1:])", "bf = be[:-1]", PINS),
    ("1D f(R) K3 power of a", SPH,
     "K3 = Omega_m * a * H0 * H0 * (1 + 4 * a ** 3 * r)",
     "K3 = Omega_m * a * H0 * H0 * (1 + 4 * a ** 2 * r)", PINS),
    ("1D Poisson source sign", SPH, "F = L - K * (eta - eta_mean)", "F = L + K * (eta - eta_mean)", PINS),
    ("1D sphere profile by length", SPH,
     "inside = np.clip(np.minimum(hi, R) ** 3 - lo ** 3, 0.0, None) / (hi ** 3 - lo ** 3)",
     "inside = np.clip(np.minimum(hi, R) - lo, 0.0, None) / (hi - lo)", PINS),
    ("sphere contrast", SPH, "return (1.0 + delta) * eta_out, eta_out", "return delta * eta_out, eta_out", PINS),
    ("tau Simpson weight", PY, "w[1:-1:2] = 4.0", "w[1:-1:2] = 2.0", PINS),
    ("tau power of a", PY,
     "f = 1.0 / (a ** 3 * H0 * np.sqrt(Omega_m / a ** 3 + Omega_L))",
     "f = 1.0 / (a ** 2 * H0 * np.sqrt(Omega_m / a ** 3 + Omega_L))", PINS),
    ("leapfrog kick units", PY, "vel[d] += kick * g[d] / h", "vel[d] += kick * g[d]", PINS),
    ("leapfrog wrap", PY, "pos[d] %= N", "pos[d] %= N + 1", PINS),
    ("background f(R) exponent", PY,
     "((1 + 4 * r) / (a ** -3 + 4 * r)) ** (n + 1))",
     "((1 + 4 * r) / (a ** -3 + 4 * r)) ** n)", PINS),
    ("background chameleon", PY,
     "return 3.0 * math.log(a) / (1.0 + cham_n)",
     "return 3.0 * math.log(a) / (2.0 + cham_n)", PINS),
    ("net: ReLU derivative", NET, "dZ = dY * (Y > 0)", "dZ = dY", NET_PINS),
    ("net: pooling adjoint weight", NET, "return np.repeat(np.repeat(np.repeat(dY, 2, 0), 2, 1), 2, 2) / 8.0",
     "return np.repeat(np.repeat(np.repeat(dY, 2, 0), 2, 1), 2, 2) / 4.0", NET_PINS),
    ("net: upsampling adjoint as a mean", NET, "return dY.reshape(n, 2, n, 2, n, 2, -1).sum(axis=(1, 3, 5))",
     "return dY.reshape(n, 2, n, 2, n, 2, -1).mean(axis=(1, 3, 5))", NET_PINS),
    ("net: data gradient shift", NET, "dX += shift(dZ, (-d[0], -d[1], -d[2])) @ W[t]", "dX += shift(dZ, d) @ W[t]",
     NET_PINS),
    ("net: weight gradient shift", NET, "return np.stack([Z.T @ shift(X, d).reshape(n3, -1) for d in TAPS])",
     "return np.stack([Z.T @ shift(X, (-d[0], -d[1], -d[2])).reshape(n3, -1) for d in TAPS])", NET_PINS),
    ("net: head bias gradient", NET, "[dpred.sum()]", "[0.0]", NET_PINS),
    ("net: loss gradient factor", NET, "dpred = 2.0 * r / V", "dpred = r / V", NET_PINS),
    ("net: tap order", NET,
     "TAPS = [(di, dj, dk) for di in (-1, 0, 1) for dj in (-1, 0, 1) for dk in (-1, 0, 1)]",
     "TAPS = [(di, dj, dk) for dk in (-1, 0, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)]", NET_PINS),
    ("net: skip split in the backward pass", NET, "dd1, de0 = up_bwd(dx[..., :32]), dx[..., 32:]",
     "dd1, de0 = up_bwd(dx[..., 16:]), dx[..., :16]", NET_PINS),
]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Every mutant's pin run, one per core at a time.
    name -> (occurrences of the mutated text, pytest exit or None if the copy does not build, output).
    A C mistake goes into a copy of isis_oracle.c (ISIS_ORACLE_SRC); a Python one into a copy of the whole
    oracle package, put first on the path (ISIS_ORACLE_PKG_DIR, read by conftest.py)."""
    d = tmp_path_factory.mktemp("mutants")
    import oracle
    oracle.build()  # the Python copies take the built library along (copied with its time stamp: no rebuild)

    def run(i, m):
        name, fname, old, new, pins = m
        with open(os.path.join(ORACLE_DIR, fname)) as f:
            src = f.read()
        if src.count(old) != 1:
            return src.count(old), None, ""
        env = dict(os.environ, OMP_NUM_THREADS="1")
        if fname == C:
            mutant = d / f"isis_oracle_mutant{i}.c"
            mutant.write_text(src.replace(old, new))
            # the copy must compile: a build error would fail the pins for the wrong reason
            cc = subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                                 str(mutant.with_suffix(".so")), str(mutant), "-lm"], capture_output=True, text=True)
            if cc.returncode != 0:
                return 1, None, cc.stderr[-3000:]
            env["ISIS_ORACLE_SRC"] = str(mutant)
        else:
            pkg = d / f"pkg{i}"
            shutil.copytree(ORACLE_DIR, pkg / "oracle", ignore=shutil.ignore_patterns("__pycache__"))
            (pkg / "oracle" / fname).write_text(src.replace(old, new))
            env["ISIS_ORACLE_PKG_DIR"] = str(pkg)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider",
                            pins], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
        return 1, r.returncode, r.stdout[-3000:]

    runs = MUTATIONS + CONTROLS
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        res = list(ex.map(lambda im: run(*im), enumerate(runs)))
    return {m[0]: r for m, r in zip(runs, res)}


# the copies without a planted mistake, through the same routes: the pins must pass
CONTROLS = [("control C " + pins, C, "int orc_solve(", "int orc_solve(", pins) for pins in (PINS, PATCH_PINS)] + \
           [("control Python " + PINS, PY, "def tau_interval(", "def tau_interval(", PINS)]


@pytest.mark.parametrize("name", [c[0] for c in CONTROLS])
def test_unmutated_copy_passes(outcomes, name):
    count, code, out = outcomes[name]
    assert count == 1 and code == 0, out


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(outcomes, name):
    count, code, out = outcomes[name]
    assert count == 1, f"{name}: the text to mutate must occur exactly once (found {count})"
    assert code is not None, f"{name}: the copy does not compile\n{out}"
    assert code == 1, f"{name}: no pin failed (pytest exit {code})\n{out}"
