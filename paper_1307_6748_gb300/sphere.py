"""The static sphere workload of Sect. 5.1 ("Potential solver") on the GPU.

A sphere of radius R and density contrast delta at the centre of a periodic box of side B (mean density
1), as a cell-averaged density on a uniform grid; the scalar field is solved with the library's FAS
solver and its radial profile binned, the data of the paper's Fig. of the static tests.  Cases as in
Sect. 5.1: delta = 5000; symmetron R = 3, B = 40 Mpc/h, lambda0 = 1 Mpc/h, a_SSB = 0.6 at z = 0 and 1;
f(R) R = 5, B = 100 Mpc/h, n = 1, |f_R0| = 1e-6 at z = 0.

python -m paper_1307_6748_gb300.sphere [--N 128] [--prec f64|refine] [--levels 0] [--expand 4]
                                       [--profile-dir DIR]
prints one JSON line per case (solve time from CUDA events after one untimed solve, cycles, residuals);
--levels L adds L refinement levels (amr.refine, in --prec as the domain) on the domain solution and times each;
with --profile-dir, writes r, mean, min, max of the field (chi, or f_R = -e^u / a^2) per radial bin.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import amr, isis, synth

CASES = {
    "symmetron_z0": dict(model="symmetron", z=0.0, delta=5000.0, R=3.0, B=40.0, params=dict(lambda0=1.0, a_ssb=0.6)),
    "symmetron_z1": dict(model="symmetron", z=1.0, delta=5000.0, R=3.0, B=40.0, params=dict(lambda0=1.0, a_ssb=0.6)),
    "fofr_z0": dict(model="fofr", z=0.0, delta=5000.0, R=5.0, B=100.0, params=dict(n=1, fR0_abs=1e-6)),
}


def exterior_density(delta: float, R: float, B: float) -> float:
    """Density outside the sphere for a box mean of 1 (the rho(r) of Sect. 5.1)."""
    return 1.0 / (1.0 + 4.0 * math.pi / 3.0 * delta * (R / B) ** 3)


def initial_field(case: dict, N: int, device="cuda") -> tuple[torch.Tensor, int]:
    """(phi, init mode): the symmetron starts from the exterior minimum sqrt(1 - (a_SSB/a)^3 eta_out)
    everywhere (at z = 1 the eta = 1 background is the unbroken chi = 0, a fixed point of the iteration);
    f(R) from the library's cell-wise uniform-density solution."""
    a = 1.0 / (1.0 + case["z"])
    phi = torch.empty((N,) * 3, dtype=torch.float64, device=device)
    if case["model"] == "symmetron":
        eta_out = exterior_density(case["delta"], case["R"], case["B"])
        phi.fill_(math.sqrt(max(0.0, 1.0 - (case["params"]["a_ssb"] / a) ** 3 * eta_out)))
        return phi, isis.ISIS_INIT_INPUT
    return phi, isis.ISIS_INIT_LOCAL


def solve(case: dict, N: int, prec: int, tol: float, eta: torch.Tensor | None = None):
    """One solve of a case on an N^3 grid; returns (phi, info, eta)."""
    a = 1.0 / (1.0 + case["z"])
    if eta is None:
        eta = synth.sphere_eta(N, case["B"], case["R"], case["delta"]).cuda()
    phi, init = initial_field(case, N)
    model = isis.ISIS_SYMMETRON if case["model"] == "symmetron" else isis.ISIS_FOFR_HS
    info = isis.isis_scalar_solve(model, isis.Params(**case["params"]), isis.Grid(N, case["B"]), a, eta, phi,
                                  tol=tol, opts=isis.Opts(prec=prec, init=init, inner_cycles=4))
    return phi, info, eta


def radial_profile(case: dict, phi: torch.Tensor, nbins: int) -> np.ndarray:
    """Rows (r, mean, min, max) of the field per radial bin of width B / (2 nbins) about the centre."""
    N, B = phi.shape[0], case["B"]
    h = B / N
    x = (torch.arange(N, device=phi.device, dtype=torch.float64) + 0.5) * h - B / 2
    r = torch.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2).reshape(-1)
    f = phi.reshape(-1)
    if case["model"] == "fofr":
        a = 1.0 / (1.0 + case["z"])
        f = -torch.exp(f) / (a * a)
    w = B / (2 * nbins)
    k = (r / w).long()
    keep = k < nbins
    k, f = k[keep], f[keep]
    cnt = torch.zeros(nbins, dtype=torch.float64, device=phi.device).index_add_(0, k, torch.ones_like(f))
    s = torch.zeros(nbins, dtype=torch.float64, device=phi.device).index_add_(0, k, f)
    lo = torch.full((nbins,), math.inf, dtype=torch.float64, device=phi.device).scatter_reduce(0, k, f, "amin")
    hi = torch.full((nbins,), -math.inf, dtype=torch.float64, device=phi.device).scatter_reduce(0, k, f, "amax")
    rc = (torch.arange(nbins, dtype=torch.float64) + 0.5) * w
    rows = torch.stack([rc, (s / cnt.clamp(min=1)).cpu(), lo.cpu(), hi.cpu()], 1).numpy()
    return rows[cnt.cpu().numpy() > 0]


def main():
    import argparse
    import json
    import os

    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--prec", default="refine", choices=["f64", "refine"])
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--cases", default=",".join(CASES))
    ap.add_argument("--levels", type=int, default=0)
    ap.add_argument("--expand", type=int, default=4)
    ap.add_argument("--prof", action="store_true", help="per-kernel-kind event times of the level solves")
    ap.add_argument("--profile-dir", default=None)
    args = ap.parse_args()
    isis.load()
    prec = isis.ISIS_F64 if args.prec == "f64" else isis.ISIS_F32_REFINE64
    for name in args.cases.split(","):
        case = CASES[name]
        phi, info, eta = solve(case, args.N, prec, args.tol)  # untimed: allocations, caches
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        phi, info, _ = solve(case, args.N, prec, args.tol, eta)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"case": name, "N": args.N, "prec": args.prec, "ms": round(e0.elapsed_time(e1), 3),
                          "cycles": info.cycles, "outer": info.outer, "res_final_over_ref":
                          info.res_final / info.res_ref}), flush=True)
        if args.levels > 0:
            a = 1.0 / (1.0 + case["z"])
            model = isis.ISIS_SYMMETRON if case["model"] == "symmetron" else isis.ISIS_FOFR_HS

            def dens(dims, corner, h, case=case):
                return synth.sphere_eta_box(dims, corner, h, case["B"], case["R"], case["delta"])

            run = lambda: amr.refine(model, isis.Params(**case["params"]), isis.Grid(args.N, case["B"]), a,
                                     eta.cpu().numpy(), phi, dens, levels=args.levels, expand=args.expand,
                                     tol=args.tol, prec=prec)
            run()  # untimed: the flags, boxes and patch densities on the host, then the solves
            # time each level's solve alone, on its own inputs
            levels = run()
            for lv in levels:
                phi_l = torch.empty_like(lv.phi)
                opts = isis.Opts(max_cycles=100, init=isis.ISIS_INIT_PARENT, prec=prec, inner_cycles=4)
                parent = phi if lv.level == 1 else levels[lv.level - 2].phi
                torch.cuda.synchronize()
                if args.prof:
                    isis.prof_reset()
                    isis.prof_enable(True)
                e0.record()
                info = isis.isis_patch_scalar_solve(model, isis.Params(**case["params"]),
                                                    isis.Grid(args.N, case["B"]), a, lv.patch, parent, lv.flags,
                                                    lv.eta, phi_l, tol=args.tol, opts=opts)
                e1.record()
                torch.cuda.synchronize()
                print(json.dumps({"case": name, "level": lv.level, "prec": args.prec, "box": list(lv.patch.n),
                                  "fine_cells": int(lv.phi.numel()), "unknowns": int(lv.unknowns.sum()),
                                  "ms": round(e0.elapsed_time(e1), 3), "cycles": info.cycles, "outer": info.outer,
                                  "res_final_over_ref": info.res_final / info.res_ref}), flush=True)
                if args.prof:
                    isis.prof_enable(False)
                    kinds = {k: [v[0], round(v[1], 3)] for k, v in isis.prof_read().items()}
                    print(json.dumps({"case": name, "level": lv.level, "kinds": kinds}), flush=True)
        if args.profile_dir:
            os.makedirs(args.profile_dir, exist_ok=True)
            rows = radial_profile(case, phi, args.N)
            np.savetxt(os.path.join(args.profile_dir, f"sphere_{name}_{args.N}.txt"), rows,
                       header="r[Mpc/h] mean min max (" + ("chi" if case["model"] == "symmetron" else "f_R") + ")")


if __name__ == "__main__":
    main()
