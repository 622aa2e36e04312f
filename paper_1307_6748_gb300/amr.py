"""Refinement levels over the domain grid: the level-by-level solve of Sects. 3.3.1 and 3.4.1.

Each level refines, by two, the cells of its parent level whose mass reaches m_ref mean-density domain cells
(the quasi-Lagrangian rule with one particle per domain cell), dilated by `expand` cells and kept inside the
parent's refined cells; one dense box (a patch) holds them.  The parent's converged field gives the values of
the patch cells that do not exist, and the patch is solved by the library's patch solver
(isis_patch_poisson_solve / isis_patch_scalar_solve) before the next level is built on it, as the paper
solves each refined level after its parent.

Host logic only: the flags and boxes come from the input recipes of synth.py, the densities of the patch cells
from a caller's function, and every step of every solve runs in the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import isis, synth


@dataclass
class Level:
    level: int
    patch: isis.Patch
    corner: tuple       # lower corner of the patch's first fine cell, Mpc/h
    h: float            # fine cell size
    flags: torch.Tensor  # uint8, patch.n, device
    eta: torch.Tensor    # float64, fine dims, device
    phi: torch.Tensor    # float64, fine dims, device: the solution
    info: isis.Info
    unknowns: np.ndarray  # bool, fine dims (host): the children of flagged cells


def refine(model, params: isis.Params | None, grid: isis.Grid, a: float, eta_domain: np.ndarray,
           phi_domain: torch.Tensor, eta_box, levels: int = 2, m_ref: float = 8.0, expand: int = 1,
           tol: float = 1e-10, max_cycles: int = 100, nu1: int = 2, nu2: int = 2, prec: int = isis.ISIS_F64,
           inner_cycles: int = 4, stream=None) -> list[Level]:
    """Solve up to `levels` refinement levels on top of a converged domain field.

    model: isis.ISIS_SYMMETRON, isis.ISIS_FOFR_HS, or None for the Newtonian potential.
    eta_domain: host array (N^3) of the domain density; phi_domain: the domain field on the device (float64).
    eta_box(dims, corner, h) -> host array: the density of a box of cells of size h whose first cell's lower
    corner is `corner`.  prec: isis.ISIS_F64, or isis.ISIS_F32_REFINE64 (FP32 correction cycles, inner_cycles
    per FP64 outer iteration).  Stops early when a level has nothing to refine."""
    N, B = grid.N, grid.box
    out: list[Level] = []
    parent, peta, pdims = phi_domain, np.asarray(eta_domain), (N, N, N)
    corner, within = (0.0, 0.0, 0.0), None
    eta_mean = float(np.mean(eta_domain))
    for lev in range(1, levels + 1):
        periodic = lev == 1
        f = synth.refine_flags(peta, lev, m_ref=m_ref, expand=expand, periodic=periodic, within=within)
        ob = synth.patch_box(f, periodic=periodic)
        if ob is None:
            break
        o, n = ob
        hp = B / (N * 2 ** (lev - 1))
        h = hp / 2
        flags = synth.box_flags(f, o, n, periodic)
        nf = tuple(2 * v for v in n)
        fc = tuple(corner[ax] + o[ax] * hp for ax in range(3))
        eta_f = np.ascontiguousarray(eta_box(nf, fc, h), dtype=np.float64)
        patch = isis.Patch(tuple(n), tuple(o), pdims, periodic, level=lev, eta_mean=eta_mean)
        dev = phi_domain.device
        tf = torch.from_numpy(flags).to(dev)
        te = torch.from_numpy(eta_f).to(dev)
        phi = torch.empty(nf, dtype=torch.float64, device=dev)
        opts = isis.Opts(nu1=nu1, nu2=nu2, max_cycles=max_cycles, init=isis.ISIS_INIT_PARENT, prec=prec,
                         inner_cycles=inner_cycles)
        if model is None:
            info = isis.isis_patch_poisson_solve(grid, a, patch, parent, tf, te, phi, tol=tol, opts=opts,
                                                 stream=stream)
        else:
            info = isis.isis_patch_scalar_solve(model, params, grid, a, patch, parent, tf, te, phi, tol=tol,
                                                opts=opts, stream=stream)
        unk = np.repeat(np.repeat(np.repeat(flags, 2, 0), 2, 1), 2, 2) > 0
        out.append(Level(lev, patch, fc, h, tf, te, phi, info, unk))
        parent, peta, pdims, corner, within = phi, eta_f, nf, fc, unk
    return out
