"""Mutation tests of the oracle's pins: each case plants one plausible mistake in a copy of the oracle (a
dropped or wrong factor, a flipped sign, a wrong neighbour or offset, a wrong constant) and runs the pin
tests against that copy, which must fail.  The oracle stays pinned to facts outside itself only if every
such mistake is caught.  CPU only; the copy is compiled in a temporary directory."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "isis_oracle.c")

PINS = "tests/test_oracle_pins.py"
PATCH_PINS = "tests/test_patch_pins.py"

# (name, exact text in the oracle, its planted replacement, the pin file that must catch it)
MUTATIONS = [
    ("symmetron cubic term sign",
     "c->A * ((c->s * eta - 1.0) * phi + phi * phi * phi)", "c->A * ((c->s * eta - 1.0) * phi - phi * phi * phi)",
     PINS),
    ("symmetron derivative factor",
     "c->A * (c->s * eta - 1.0 + 3.0 * phi * phi)", "c->A * (c->s * eta - 1.0 + 2.0 * phi * phi)", PINS),
    ("Poisson source sign", "return c->KP * (eta - c->eta_mean);", "return -c->KP * (eta - c->eta_mean);", PINS),
    ("f(R) K3 power of a", "(1.0 + 4.0 * a * a * a * r)", "(1.0 + 4.0 * a * a * r)", PINS),
    ("f(R) face value: the cell's b instead of the face mean", "div += bf * (un - u);", "div += bu * (un - u);",
     PINS),
    ("f(R) derivative factor 1/2", "acc += -bf + 0.5 * bu * (un - u);\n    }\n    return acc / h2",
     "acc += -bf + bu * (un - u);\n    }\n    return acc / h2", PINS),
    ("f(R) source exponent", "c->K2 * exp(-phi / c->np1) + c->K3", "c->K2 * exp(-phi * c->np1) + c->K3", PINS),
    ("chameleon exponent", "c->np1 = 1.0 / (1.0 + p->cham_n);", "c->np1 = 1.0 + p->cham_n;", PINS),
    ("restriction weight", "coarse[IDX(NH, I, J, K)] = s / 8.0;", "coarse[IDX(NH, I, J, K)] = s / 4.0;", PINS),
    ("prolongation neighbour", "ci[1] = WRAP(i / 2 + ((i & 1) ? 1 : -1), NH);",
     "ci[1] = WRAP(i / 2 + ((i & 1) ? -1 : 1), NH);", PINS),
    ("CIC cell-centre offset", "double xs = x - 0.5;", "double xs = x;", PINS),
    ("gradient spacing",
     "gx[q] = (f[IDX(N, WRAP(i + 1, N), j, k)] - f[IDX(N, WRAP(i - 1, N), j, k)]) / (2.0 * h);",
     "gx[q] = (f[IDX(N, WRAP(i + 1, N), j, k)] - f[IDX(N, WRAP(i - 1, N), j, k)]) / h;", PINS),
    ("symmetron force constant power of a_SSB", "/ pow(p->a_ssb, 3.0);", "/ pow(p->a_ssb, 2.0);", PINS),
    ("FAS coarse source without L_H(R phi)",
     "C->sigma[IDX(C->N, i, j, k)] += op_L(&H->coef, C, C->phi, i, j, k);", "C->sigma[IDX(C->N, i, j, k)] += 0.0;",
     PINS),
    ("coarse correction without R phi", "C->phi0[q] = C->phi[q] - C->phi0[q];", "C->phi0[q] = C->phi[q];", PINS),
    ("Newton step sign", "L->phi[q] = L->phi[q] - F / dF;", "L->phi[q] = L->phi[q] + F / dF;", PINS),
    ("Poisson mean kept", "if (p->model == ORC_POISSON) remove_mean(p->N, phi);", "if (0) remove_mean(p->N, phi);",
     PINS),
    ("symmetron reference residual without s",
     "scale = H.coef.A * H.coef.s * background(p, &H.coef);\n    else if (H.coef.model == ORC_FOFR) scale = H.coef.K1;"
     "\n    else scale = H.coef.KP;\n    info->ref = scale * sqrt(sum2 / (double)n3);",
     "scale = H.coef.A * background(p, &H.coef);\n    else if (H.coef.model == ORC_FOFR) scale = H.coef.K1;"
     "\n    else scale = H.coef.KP;\n    info->ref = scale * sqrt(sum2 / (double)n3);", PINS),
    ("f(R) reference residual constant",
     "scale = H.coef.K1;\n    else scale = H.coef.KP;\n    info->ref = scale * sqrt(sum2 / (double)n3);",
     "scale = H.coef.K3;\n    else scale = H.coef.KP;\n    info->ref = scale * sqrt(sum2 / (double)n3);", PINS),
    ("CIC normalisation", "for (size_t q = 0; q < n3; ++q) eta[q] /= nbar;",
     "for (size_t q = 0; q < n3; ++q) eta[q] *= nbar;", PINS),
    ("f(R) K2 exponent", "pow(p->fR0_abs * a * a, 1.0 / c->np1)", "pow(p->fR0_abs * a * a, c->np1)", PINS),
    ("symmetron A", "c->A = a * a / (2.0 * p->lambda0 * p->lambda0);", "c->A = a * a / (p->lambda0 * p->lambda0);",
     PINS),
    ("chameleon force constant", "double Cc = 3.0 * (1.0 + p->cham_n)", "double Cc = 3.0 * (2.0 + p->cham_n)", PINS),
    ("f(R) force factor", "else pref = 0.5 * exp(phi[q]);", "else pref = exp(phi[q]);", PINS),
    ("force sign", "gx[q] = -acc[0];", "gx[q] = acc[0];", PINS),
    ("patch ghost: mask ratio sign", "*mu = mn / L->m[q];", "*mu = -mn / L->m[q];", PATCH_PINS),
    ("patch interpolation neighbour", "pc[a][1] = pc[a][0] + ((f[a] & 1) ? 1 : -1);",
     "pc[a][1] = pc[a][0] + ((f[a] & 1) ? -1 : 1);", PATCH_PINS),
    ("patch restriction weight", "coarse[PIDX(nc, I, J, K)] = s / 8.0;", "coarse[PIDX(nc, I, J, K)] = s / 4.0;",
     PATCH_PINS),
    ("patch prolongation neighbour", "int ci[2] = {i / 2, i / 2 + ((i & 1) ? 1 : -1)};",
     "int ci[2] = {i / 2, i / 2 + ((i & 1) ? -1 : 1)};", PATCH_PINS),
    ("patch prolongation weights",
     "double w[2] = {0.75, 0.25}, v = 0.0;\n        for (int a = 0; a < 2; ++a)\n          for (int b = 0; b < 2; ++b)"
     "\n            for (int d = 0; d < 2; ++d) {",
     "double w[2] = {0.5, 0.5}, v = 0.0;\n        for (int a = 0; a < 2; ++a)\n          for (int b = 0; b < 2; ++b)"
     "\n            for (int d = 0; d < 2; ++d) {", PATCH_PINS),
    ("patch reference residual without s",
     "scale = H.coef.A * H.coef.s * background(p, &H.coef);\n    else if (H.coef.model == ORC_FOFR) scale = H.coef.K1;"
     "\n    else scale = H.coef.KP;\n    info->ref = cnt",
     "scale = H.coef.A * background(p, &H.coef);\n    else if (H.coef.model == ORC_FOFR) scale = H.coef.K1;"
     "\n    else scale = H.coef.KP;\n    info->ref = cnt", PATCH_PINS),
    ("patch Poisson reference density", "double eref = (p->model == ORC_POISSON) ? P->eta_mean : 1.0, s2 = 0.0;",
     "double eref = 1.0, s2 = 0.0;", PATCH_PINS),
    ("patch ghost: the neighbour's u^Pre", "(*mu) * (L->u[q] - L->pre[q]);", "(*mu) * (L->u[qn] - L->pre[qn]);",
     PATCH_PINS),
    ("patch f(R) ghost derivative factor", "dacc += mu * (0.5 * bn * (un - u) + bf);",
     "dacc += mu * (bn * (un - u) + bf);", PATCH_PINS),
    ("patch f(R) derivative factor 1/2", "dacc += -bf + 0.5 * bu * (un - u);", "dacc += -bf + bu * (un - u);",
     PATCH_PINS),
]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Every mutant's pin run, one per core at a time.
    name -> (occurrences of the mutated text, pytest exit, output)."""
    with open(SRC) as f:
        src = f.read()
    d = tmp_path_factory.mktemp("mutants")

    def run(i, m):
        name, old, new, pins = m
        if src.count(old) != 1:
            return src.count(old), None, ""
        mutant = d / f"isis_oracle_mutant{i}.c"
        mutant.write_text(src.replace(old, new))
        # the copy must compile: a build error would fail the pins for the wrong reason
        cc = subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                             str(mutant.with_suffix(".so")), str(mutant), "-lm"], capture_output=True, text=True)
        if cc.returncode != 0:
            return 1, None, cc.stderr[-3000:]
        env = dict(os.environ, ISIS_ORACLE_SRC=str(mutant), OMP_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider",
                            pins], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
        return 1, r.returncode, r.stdout[-3000:]

    runs = MUTATIONS + [CONTROL(PINS), CONTROL(PATCH_PINS)]
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        res = list(ex.map(lambda im: run(*im), enumerate(runs)))
    return {m[0]: r for m, r in zip(runs, res)}


def CONTROL(pins):
    """The copy without a planted mistake, through the same mechanism: the pins must pass."""
    return (f"control {pins}", "int orc_solve(", "int orc_solve(", pins)


@pytest.mark.parametrize("pins", [PINS, PATCH_PINS])
def test_unmutated_copy_passes(outcomes, pins):
    count, code, out = outcomes[f"control {pins}"]
    assert count == 1 and code == 0, out


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(outcomes, name):
    count, code, out = outcomes[name]
    assert count == 1, f"{name}: the text to mutate must occur exactly once (found {count})"
    assert code is not None, f"{name}: the copy does not compile\n{out}"
    assert code == 1, f"{name}: no pin failed (pytest exit {code})\n{out}"
