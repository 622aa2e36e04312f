"""Particle-mesh time stepping with the scalar field: the leapfrog in super-comoving time of
Sect. 4.1 (Eqs. (leap_frog_1)-(leap_frog_3)), the same for f(R) (Sect. 4.2).

Each step at expansion factor a_n runs the library's force step -- CIC density of the particles,
Poisson solve, scalar-field solve, per-particle acceleration g = -[grad Phi~ + F5] -- and its fused
kick-drift kernel with kick = (dtau_{n-1} + dtau_n)/2 (the second half-kick of the previous step
joined to the first of this one, as the paper reuses the second velocity evaluation) and drift
dtau_n.  The fields of the previous step are the initial guesses of the next solves.

Units: positions and velocities in cell units; tau in Mpc/h (c = 1), dtau = da / (a^3 H0 E(a)),
E(a) = sqrt(Omega_m a^-3 + Omega_L).  The tau integral is host arithmetic (Gauss-Legendre); all
per-particle and per-cell work runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import isis

_GL_X, _GL_W = np.polynomial.legendre.leggauss(16)


def dtau(a0: float, a1: float, Omega_m: float = 0.267, Omega_L: float = 0.733, H0: float = isis.H0_MPC) -> float:
    """Super-comoving time from a0 to a1 (16-point Gauss-Legendre on [a0, a1])."""
    a = 0.5 * (a1 - a0) * _GL_X + 0.5 * (a1 + a0)
    f = 1.0 / (a ** 3 * H0 * np.sqrt(Omega_m / a ** 3 + Omega_L))
    return float(0.5 * (a1 - a0) * np.dot(_GL_W, f))


class PM:
    """Particles (float32 device arrays, cell units) evolved with the force step of one model
    (isis.ISIS_SYMMETRON, isis.ISIS_FOFR_HS, or None for gravity alone)."""

    def __init__(self, grid: isis.Grid, model, params: isis.Params, x, y, z, vx, vy, vz,
                 prec: int = isis.ISIS_F32_REFINE64, tol: float = 1e-8, inner: int = 4, ncoarse: int = 2):
        self.grid, self.model, self.params = grid, model, params
        self.x, self.y, self.z, self.vx, self.vy, self.vz = x, y, z, vx, vy, vz
        self.prec, self.tol, self.inner, self.ncoarse = prec, tol, inner, ncoarse
        dev = x.device
        dt = torch.float64 if prec != isis.ISIS_F32 else torch.float32
        N = grid.N
        self.eta = torch.empty((N,) * 3, dtype=dt, device=dev)
        self.Phi = torch.zeros((N,) * 3, dtype=dt, device=dev)
        self.phi = torch.empty((N,) * 3, dtype=dt, device=dev) if model is not None else None
        self.g = tuple(torch.empty(x.numel(), dtype=torch.float32, device=dev) for _ in range(3))
        self.dtau_prev = 0.0
        self.nsteps = 0
        self.infos = []

    def _opts(self, init):
        return isis.Opts(prec=self.prec, inner_cycles=self.inner, n_coarsest=self.ncoarse, init=init)

    def step(self, a: float, a_next: float):
        """Forces at a (current positions), then kick and drift to a_next; returns the solve infos."""
        g, first = self.grid, self.nsteps == 0
        isis.isis_cic_deposit(g, self.x, self.y, self.z, self.eta)
        init = isis.ISIS_INIT_BACKGROUND if first else isis.ISIS_INIT_INPUT
        info = {"poisson": isis.isis_poisson_solve(g, a, self.eta, self.Phi, tol=self.tol, opts=self._opts(init))}
        if self.model is not None:
            info["scalar"] = isis.isis_scalar_solve(self.model, self.params, g, a, self.eta, self.phi, tol=self.tol,
                                                    opts=self._opts(init))
        isis.isis_fifth_force(self.model if self.model is not None else isis.ISIS_SYMMETRON, self.params, g, a,
                              self.Phi, self.phi, self.x, self.y, self.z, out=self.g)
        dt = dtau(a, a_next, g.Omega_m, g.Omega_L, g.H0)
        isis.isis_kick_drift(g, self.x, self.y, self.z, self.vx, self.vy, self.vz, self.g,
                             0.5 * (self.dtau_prev + dt), dt)
        self.dtau_prev = dt
        self.nsteps += 1
        self.infos.append(info)
        return info

    def run(self, a_steps):
        """Steps a_steps[0] -> ... -> a_steps[-1]; velocities end at the last half step."""
        for a, a_next in zip(a_steps[:-1], a_steps[1:]):
            self.step(a, a_next)
        return self


def main():
    """python -m paper_1307_6748_gb300.pm [--N 512] [--box 256] [--model symmetron|fofr|chameleon|none]
    [--steps 10] [--cham-n -0.5 --lambda0 7.5 --beta 0.408]
    Zel'dovich particles at a0, steps of da; prints one JSON line per step (ms, cycles of each solve).
    The chameleon defaults are the Hu-Sawicki-equivalent exponent and coupling of Sect. 6 (n = -1/2,
    beta = 1/sqrt(6)) with the 7.5 Mpc/h range of |f_R0| = 1e-5 (Table 1)."""
    import argparse
    import json

    from . import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=512)
    ap.add_argument("--box", type=float, default=256.0)
    ap.add_argument("--model", default="symmetron", choices=["symmetron", "fofr", "chameleon", "none"])
    ap.add_argument("--cham-n", type=float, default=-0.5)
    ap.add_argument("--lambda0", type=float, default=7.5)
    ap.add_argument("--beta", type=float, default=6 ** -0.5)
    ap.add_argument("--a0", type=float, default=0.9)
    ap.add_argument("--da", type=float, default=0.01)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--inner", type=int, default=4)
    args = ap.parse_args()
    isis.load()
    model = {"symmetron": isis.ISIS_SYMMETRON, "fofr": isis.ISIS_FOFR_HS, "chameleon": isis.ISIS_CHAMELEON,
             "none": None}[args.model]
    ic = synth.zeldovich_ic(args.N, args.box, args.a0, seed=3, device="cuda")
    par = isis.Params(lambda0=args.lambda0, beta=args.beta, cham_n=args.cham_n) if args.model == "chameleon" \
        else isis.Params()
    run = PM(isis.Grid(args.N, args.box), model, par, *ic, tol=args.tol, inner=args.inner)
    for k in range(args.steps):
        a = args.a0 + k * args.da
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        info = run.step(a, a + args.da)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"step": k, "a": a, "ms": e0.elapsed_time(e1),
                          "cycles": {name: v.cycles for name, v in info.items()},
                          "outer": {name: v.outer for name, v in info.items()}}), flush=True)


if __name__ == "__main__":
    main()
