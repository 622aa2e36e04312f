"""A domain-decomposed FAS V-cycle on the host (test infrastructure): the layout a multi-GPU solve would take,
run as CPU ranks over torch.distributed (gloo), to show that partitioning the grid does not change the
solution (the serial-vs-parallel agreement of Sect. 5.1, whose static sphere test gives the same results on one
and on eight processes).

Partition.  Rank r of P owns the planes i in [r n, (r+1) n), n = N/P, of every level that keeps at least two
planes per rank and has N >= gather_n; each slab carries one ghost plane on either side in i.  Before each
colour pass of the red-black Newton-Gauss-Seidel smoother (Sect. 3.2), before a residual and before a
prolongation, each rank sends its first own plane to the rank below and its last to the rank above (periodic
ring) and receives its ghosts: one plane exchanged per colour pass.  Restriction (the mean of 8 children)
needs no exchange: a coarse plane's children are two own planes.  The residual norm of the convergence test is
a sum over ranks (all_reduce), and so is the Poisson mean.  The coarser levels are gathered (all_gather) and
every rank runs the same serial V-cycle on them, down to the coarsest dense Newton solve (the oracle's own),
then keeps its slab of the result.

Arithmetic.  FP64 numpy, the oracle's algorithm in its order (R1-R7 of the readings: V(nu1, nu2), red first,
R = mean of 8 children, P = cell-centred trilinear, Sigma_H = L_H(R phi) + R(Sigma - L(phi)), the Poisson mean
removed after every cycle), for the symmetron (Sect. 4.1) and Poisson (Sect. 3.1).  With P = 1 the same code is
the serial solve; it matches oracle.solve at a fixed cycle count to rounding."""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch
import torch.distributed as dist

import oracle

POISSON, SYMMETRON = oracle.POISSON, oracle.SYMMETRON


@dataclass
class Coef:
    model: int
    A: float = 0.0      # symmetron: a^2 / (2 lambda0^2)
    s: float = 0.0      # (a_SSB / a)^3
    KP: float = 0.0     # Poisson: 1.5 Om H0^2 / a
    eta_mean: float = 1.0


def coef_of(p: oracle.Problem, eta_mean: float) -> Coef:
    if p.model == SYMMETRON:
        return Coef(SYMMETRON, A=p.a * p.a / (2.0 * p.lambda0 ** 2), s=(p.a_ssb / p.a) ** 3)
    return Coef(POISSON, KP=1.5 * p.Omega_m * p.H0 ** 2 / p.a, eta_mean=eta_mean)


class Comm:
    """Ghost exchange and sums over the ranks (world size 1: the periodic wrap of one slab)."""

    def __init__(self):
        self.rank = dist.get_rank() if dist.is_initialized() else 0
        self.size = dist.get_world_size() if dist.is_initialized() else 1

    def ghosts(self, x: np.ndarray) -> None:
        """x[0] <- the last own plane of the rank below, x[-1] <- the first own plane of the rank above."""
        if self.size == 1:
            x[0] = x[-2]
            x[-1] = x[1]
            return
        below, above = (self.rank - 1) % self.size, (self.rank + 1) % self.size
        first, last = torch.from_numpy(x[1].copy()), torch.from_numpy(x[-2].copy())
        g0, g1 = torch.empty_like(first), torch.empty_like(first)
        reqs = [dist.isend(first, below, tag=1), dist.isend(last, above, tag=2),
                dist.irecv(g0, below, tag=2), dist.irecv(g1, above, tag=1)]
        for r in reqs:
            r.wait()
        x[0] = g0.numpy()
        x[-1] = g1.numpy()

    def sum(self, v: float) -> float:
        if self.size == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64)
        dist.all_reduce(t)
        return float(t.item())

    def gather(self, slab: np.ndarray) -> np.ndarray:
        """The whole grid from every rank's own planes (stacked along i)."""
        if self.size == 1:
            return slab.copy()
        t = torch.from_numpy(np.ascontiguousarray(slab))
        parts = [torch.empty_like(t) for _ in range(self.size)]
        dist.all_gather(parts, t)
        return np.concatenate([p.numpy() for p in parts], axis=0)


class Level:
    """One level's slab: own planes [i0, i0 + n) of an N^3 grid, x with one ghost plane on either side."""

    def __init__(self, N: int, h: float, i0: int, n: int):
        self.N, self.h, self.i0, self.n = N, h, i0, n
        self.x = np.zeros((n + 2, N, N))
        self.x0 = np.zeros((n, N, N))
        self.eta = np.zeros((n, N, N))
        self.sig = np.zeros((n, N, N))

    def colour_mask(self, color: int) -> np.ndarray:
        i = np.arange(self.i0, self.i0 + self.n)[:, None, None]
        j = np.arange(self.N)[None, :, None]
        k = np.arange(self.N)[None, None, :]
        return ((i + j + k) & 1) == color


def op_L(c: Coef, L: Level, x: np.ndarray) -> np.ndarray:
    """L(x) at the own cells, the neighbours summed in the oracle's order (i+1, i-1, j+1, j-1, k+1, k-1);
    x has its ghost planes filled."""
    u = x[1:-1]
    s = x[2:] + x[:-2]
    s = s + np.roll(u, -1, axis=1)
    s = s + np.roll(u, 1, axis=1)
    s = s + np.roll(u, -1, axis=2)
    s = s + np.roll(u, 1, axis=2)
    lap = (s - 6.0 * u) / (L.h * L.h)
    if c.model == SYMMETRON:
        return lap - c.A * ((c.s * L.eta - 1.0) * u + u * u * u)
    return lap - c.KP * (L.eta - c.eta_mean)


def op_dL(c: Coef, L: Level, x: np.ndarray) -> np.ndarray:
    u = x[1:-1]
    d = -6.0 / (L.h * L.h)
    if c.model == SYMMETRON:
        return d - c.A * (c.s * L.eta - 1.0 + 3.0 * u * u)
    return np.full(u.shape, d)


def smooth(c: Coef, L: Level, comm: Comm) -> None:
    """One red-black Newton-Gauss-Seidel sweep (red = (i+j+k) even first), a ghost exchange before each colour."""
    for color in (0, 1):
        comm.ghosts(L.x)
        F = op_L(c, L, L.x) - L.sig
        dF = op_dL(c, L, L.x)
        m = L.colour_mask(color)
        own = L.x[1:-1]
        own[m] = own[m] - F[m] / dF[m]


def restrict(f: np.ndarray) -> np.ndarray:
    """Mean of the 8 children of each coarse cell (own planes only)."""
    return 0.125 * (f[0::2, 0::2, 0::2] + f[0::2, 0::2, 1::2] + f[0::2, 1::2, 0::2] + f[0::2, 1::2, 1::2] +
                    f[1::2, 0::2, 0::2] + f[1::2, 0::2, 1::2] + f[1::2, 1::2, 0::2] + f[1::2, 1::2, 1::2])


def prolong_add(C: Level, fine: Level, comm: Comm) -> None:
    """fine += P(x_H - x0_H): cell-centred trilinear, weights 3/4 (own coarse cell) and 1/4 (the neighbour on
    the child's side), the coarse correction's ghost planes exchanged first."""
    d = np.zeros_like(C.x)
    d[1:-1] = C.x[1:-1] - C.x0
    comm.ghosts(d)
    n, N = fine.n, fine.N
    out = np.zeros((n, N, N))
    for ai, wa in ((0, 0.75), (1, 0.25)):
        # child plane i (own, local) of coarse plane i//2 (local + 1 in d); its second coarse plane is on its side
        ii = np.arange(n)
        ci = ii // 2 + 1 + (0 if ai == 0 else np.where(ii % 2 == 1, 1, -1))
        for bj, wb in ((0, 0.75), (1, 0.25)):
            jj = np.arange(N)
            cj = (jj // 2 + (0 if bj == 0 else np.where(jj % 2 == 1, 1, -1))) % C.N
            for ck_, wc in ((0, 0.75), (1, 0.25)):
                kk = np.arange(N)
                ck = (kk // 2 + (0 if ck_ == 0 else np.where(kk % 2 == 1, 1, -1))) % C.N
                out += wa * wb * wc * d[ci[:, None, None], cj[None, :, None], ck[None, None, :]]
    fine.x[1:-1] += out


class SlabFAS:
    """FAS V(nu1, nu2) cycles on the partitioned hierarchy, down to a coarsest grid of ncoarse^3; levels with
    N < gather_n, or fewer than two planes per rank, are gathered and solved by every rank alike."""

    def __init__(self, p: oracle.Problem, eta_full: np.ndarray, phi_full: np.ndarray, comm: Comm, nu1=2, nu2=2,
                 ncoarse=4, gather_n=16):
        self.p, self.comm, self.nu1, self.nu2, self.ncoarse = p, comm, nu1, nu2, ncoarse
        self.c = coef_of(p, float(eta_full.mean()))
        P, r = comm.size, comm.rank
        self.levels, self.dist = [], []  # per level: Level, and whether it is partitioned
        N, eta = p.N, eta_full
        etas = [eta_full]
        while N > ncoarse:
            N //= 2
            eta = oracle.restrict(eta)
            etas.append(eta)
        N = p.N
        for l, e in enumerate(etas):
            part = N >= gather_n and N // P >= 2 and all(self.dist) if l > 0 else True
            n = N // P if part else N
            i0 = r * n if part else 0
            L = Level(N, p.box / N, i0, n)
            L.eta = e[i0:i0 + n].copy()
            self.levels.append(L)
            self.dist.append(part)
            N //= 2
        L0 = self.levels[0]
        L0.x[1:-1] = phi_full[L0.i0:L0.i0 + L0.n]

    def serial_comm(self) -> Comm:
        c = Comm.__new__(Comm)
        c.rank, c.size = 0, 1
        return c

    def vcycle(self, l: int) -> None:
        L = self.levels[l]
        comm = self.comm if self.dist[l] else self.serial_comm()
        if l == len(self.levels) - 1:
            # the oracle's dense Newton solve on the coarsest grid (every rank alike)
            pc = oracle.Problem(self.p.model, L.N, self.p.box, a=self.p.a, lambda0=self.p.lambda0,
                                a_ssb=self.p.a_ssb, Omega_m=self.p.Omega_m, H0=self.p.H0)
            st, phi, _ = oracle.dense_newton(pc, L.eta, L.x[1:-1].copy(), L.sig)
            assert st == oracle.OK, st
            L.x[1:-1] = phi
            return
        for _ in range(self.nu1):
            smooth(self.c, L, comm)
        comm.ghosts(L.x)
        r = L.sig - op_L(self.c, L, L.x)
        C = self.levels[l + 1]
        xr, rr = restrict(L.x[1:-1]), restrict(r)
        if self.dist[l] and not self.dist[l + 1]:
            xr, rr = comm.gather(xr), comm.gather(rr)  # the coarser levels on every rank
        C.x[1:-1] = xr
        C.x0 = xr.copy()
        ccomm = self.comm if self.dist[l + 1] else self.serial_comm()
        ccomm.ghosts(C.x)
        C.sig = op_L(self.c, C, C.x) + rr
        self.vcycle(l + 1)
        if self.dist[l] and not self.dist[l + 1]:
            # back to this rank's slab of the coarse level (with its ghosts from the whole grid)
            nc = L.n // 2
            i0c = L.i0 // 2
            full = C.x[1:-1]
            full0 = C.x0
            Cs = Level(C.N, C.h, i0c, nc)
            Cs.x[1:-1] = full[i0c:i0c + nc]
            Cs.x0 = full0[i0c:i0c + nc]
            prolong_add(Cs, L, comm)
        else:
            prolong_add(C, L, ccomm if self.dist[l + 1] else self.serial_comm())
        for _ in range(self.nu2):
            smooth(self.c, L, comm)

    def rms(self) -> float:
        L = self.levels[0]
        self.comm.ghosts(L.x)
        F = op_L(self.c, L, L.x)
        return math.sqrt(self.comm.sum(float(np.sum(F * F))) / L.N ** 3)

    def cycle(self) -> float:
        self.vcycle(0)
        L = self.levels[0]
        if self.p.model == POISSON:
            mean = self.comm.sum(float(np.sum(L.x[1:-1]))) / L.N ** 3
            L.x[1:-1] -= mean
        return self.rms()

    def field(self) -> np.ndarray:
        L = self.levels[0]
        return self.comm.gather(L.x[1:-1])
