"""Seeded synthetic inputs: density fields and particle sets.

These stand in for the paper's cosmological initial conditions (generated
with Cosmics) and its particle snapshots, which are not available.  This
module holds none of the solver's arithmetic; the oracle tests and the CUDA
path both take their inputs from here.

Recipes
  gaussian_field   Gaussian random field with P(k) ~ k^-2: white noise filtered
                   by |k|^-1 in Fourier space, modes with k = 0 or |k| > k_Nyq
                   = pi N / L removed, rescaled to sample mean 0 and std sigma.
  lognormal_eta    eta = exp(g - sigma^2/2), divided by its sample mean.
  nfw_eta          lognormal eta plus seeded NFW haloes (log-uniform masses,
                   uniform centres, concentration c), cell-averaged with 4^3
                   sub-samples per cell, renormalised to mean 1.
  zeldovich        one particle per cell on the lattice q = i + 1/2 (cell units)
                   displaced by Psi, Psi_hat = i k delta_hat / k^2, scaled to a
                   per-component rms displacement (default 0.5 cell).
  sphere_eta       the paper's static test density (Sect. 5.1): a uniform sphere
                   of radius R and contrast delta in a box B, cell-averaged.
  sphere_eta_box   the same density on a box of cells of any size h (a patch).
  refine_flags     the cells of a level to refine: mass per cell at least m_ref
                   mean-density domain cells (RAMSES's quasi-Lagrangian rule with
                   one particle per domain cell), dilated by `expand` cells.
  patch_box        the box of parent cells of a patch: the flags' bounding box
                   widened by a margin and rounded to a multiple of 8 cells (so
                   the patch's multigrid halves it at least four times).
"""
from __future__ import annotations

import math

import numpy as np
import torch

RHO_CRIT = 2.775e11  # h^2 Msun / Mpc^3


def _kgrid(N: int, L: float, device):
    k1 = torch.fft.fftfreq(N, d=L / N, device=device, dtype=torch.float64) * (2 * math.pi)
    kz = torch.fft.rfftfreq(N, d=L / N, device=device, dtype=torch.float64) * (2 * math.pi)
    return k1.view(N, 1, 1), k1.view(1, N, 1), kz.view(1, 1, -1)


def _white(N: int, seed: int) -> torch.Tensor:
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return torch.randn((N, N, N), generator=g, dtype=torch.float64)


def gaussian_field(N: int, L: float, sigma: float, seed: int, device="cpu") -> torch.Tensor:
    """Seeded Gaussian field, P(k) ~ k^-2 cut at the grid Nyquist, mean 0, std sigma (float64)."""
    w = _white(N, seed).to(device)
    W = torch.fft.rfftn(w)
    kx, ky, kz = _kgrid(N, L, device)
    k = torch.sqrt(kx * kx + ky * ky + kz * kz)
    knyq = math.pi * N / L
    filt = torch.where((k > 0) & (k <= knyq), 1.0 / torch.clamp(k, min=1e-300), torch.zeros_like(k))
    g = torch.fft.irfftn(W * filt, s=(N, N, N))
    g = g - g.mean()
    return g * (sigma / g.std())


def lognormal_eta(N: int, L: float, sigma: float, seed: int, device="cpu") -> torch.Tensor:
    g = gaussian_field(N, L, sigma, seed, device)
    eta = torch.exp(g - 0.5 * sigma * sigma)
    return eta / eta.mean()


def nfw_eta(N: int, L: float, sigma: float, seed: int, nhalo: int = 32, halo_seed: int = 2,
            mmin: float = 1e13, mmax: float = 1e15, conc: float = 5.0, Omega_m: float = 0.267,
            device="cpu") -> torch.Tensor:
    """Lognormal field plus NFW haloes, mean 1 (masses in Msun/h, lengths in Mpc/h)."""
    eta = lognormal_eta(N, L, sigma, seed, device="cpu").numpy()
    h = L / N
    rho_m = Omega_m * RHO_CRIT
    mass = eta * rho_m * h ** 3
    rng = np.random.Generator(np.random.PCG64(halo_seed))
    logm = rng.uniform(math.log(mmin), math.log(mmax), size=nhalo)
    centres = rng.uniform(0.0, L, size=(nhalo, 3))
    sub = (np.arange(4) + 0.5) / 4.0
    for lm, c in zip(logm, centres):
        M = math.exp(lm)
        r200 = (3.0 * M / (4.0 * math.pi * 200.0 * RHO_CRIT)) ** (1.0 / 3.0)
        rs = r200 / conc
        reach = int(math.ceil(r200 / h)) + 1
        ci = np.floor(c / h).astype(int)
        offs = np.arange(-reach, reach + 1)
        cells = []
        vals = []
        for di in offs:
            for dj in offs:
                for dk in offs:
                    cell = ci + np.array([di, dj, dk])
                    base = cell * h
                    px = (base[0] + sub * h)[:, None, None]
                    py = (base[1] + sub * h)[None, :, None]
                    pz = (base[2] + sub * h)[None, None, :]
                    r = np.sqrt((px - c[0]) ** 2 + (py - c[1]) ** 2 + (pz - c[2]) ** 2)
                    x = np.maximum(r / rs, 1e-3)
                    rho = np.where(r < r200, 1.0 / (x * (1.0 + x) ** 2), 0.0)
                    cells.append(tuple(np.mod(cell, N)))
                    vals.append(rho.mean())
        vals = np.asarray(vals)
        if vals.sum() <= 0:
            continue
        vals *= M / vals.sum()
        for cell, v in zip(cells, vals):
            mass[cell] += v
    eta = mass / mass.mean()
    return torch.from_numpy(np.ascontiguousarray(eta)).to(device)


def zeldovich(N: int, L: float, seed: int = 3, disp_rms: float = 0.5, device="cpu"):
    """N^3 particles: lattice plus Zel'dovich displacement; float32 positions in cell units [0, N)."""
    delta = gaussian_field(N, L, 1.0, seed, device)
    D = torch.fft.rfftn(delta)
    kx, ky, kz = _kgrid(N, L, device)
    k2 = kx * kx + ky * ky + kz * kz
    inv = torch.where(k2 > 0, 1.0 / torch.clamp(k2, min=1e-300), torch.zeros_like(k2))
    out = []
    q = (torch.arange(N, device=device, dtype=torch.float64) + 0.5)
    grids = torch.meshgrid(q, q, q, indexing="ij")
    for kk, qq in zip((kx, ky, kz), grids):
        psi = torch.fft.irfftn(1j * kk * D * inv, s=(N, N, N))
        out.append(psi)
    rms = torch.sqrt(sum((p * p).mean() for p in out) / 3.0)
    pos = []
    for p, qq in zip(out, grids):
        x = torch.remainder(qq + p * (disp_rms / rms), float(N))
        pos.append(x.to(torch.float32).reshape(-1).contiguous())
    return pos


def zeldovich_ic(N: int, L: float, a: float, seed: int = 3, disp_rms: float = 0.5, Omega_m: float = 0.267,
                 Omega_L: float = 0.733, H0: float = 1.0 / 2997.92458, device="cpu"):
    """Particles and velocities of the growing mode at expansion factor a (cell units).

    Positions as zeldovich(); velocities v = dx/dtau = a^2 H0 E(a) Psi in cells per unit of
    super-comoving time (growth D proportional to a), with E(a) = sqrt(Om a^-3 + OL) and Psi
    the displacement of each particle from its lattice site.
    Returns (x, y, z, vx, vy, vz), float32 in [0, N) and cells per unit tau."""
    x, y, z = zeldovich(N, L, seed, disp_rms, device)
    q = (torch.arange(N, device=device, dtype=torch.float64) + 0.5)
    grids = [g.reshape(-1) for g in torch.meshgrid(q, q, q, indexing="ij")]
    fac = a * a * H0 * math.sqrt(Omega_m / a ** 3 + Omega_L)
    vel = []
    for p, qq in zip((x, y, z), grids):
        psi = torch.remainder(p.double() - qq + N / 2, float(N)) - N / 2  # displacement, periodic
        vel.append((fac * psi).to(torch.float32).contiguous())
    return (x, y, z, *vel)


def sphere_eta(N: int, B: float, R: float, delta: float, sub: int = 4) -> torch.Tensor:
    """Cell-averaged uniform sphere of radius R and contrast delta at the box centre (Sect. 5.1)."""
    h = B / N
    s = (np.arange(sub) + 0.5) / sub
    x = (np.arange(N)[:, None] + s[None, :]).reshape(-1) * h - B / 2
    inside = np.zeros((N, N, N))
    r2x = (x ** 2).reshape(N, sub)
    for a in range(sub):
        for b in range(sub):
            for c in range(sub):
                rr = r2x[:, a][:, None, None] + r2x[:, b][None, :, None] + r2x[:, c][None, None, :]
                inside += (rr < R * R)
    frac = inside / sub ** 3
    rho_out = 1.0 / (1.0 + 4.0 * math.pi / 3.0 * delta * (R / B) ** 3)
    eta = rho_out * (1.0 + delta * frac)
    return torch.from_numpy(eta)


def sphere_eta_box(dims, corner, h: float, B: float, R: float, delta: float, sub: int = 4) -> np.ndarray:
    """Cell average of the Sect. 5.1 sphere (centre B/2 on each axis) on a box of dims cells of size h whose
    first cell's lower corner sits at `corner` (Mpc/h, per axis)."""
    s = (np.arange(sub) + 0.5) / sub
    ax = [((np.arange(dims[a])[:, None] + s[None, :]) * h + corner[a] - B / 2) ** 2 for a in range(3)]
    inside = np.zeros(tuple(dims))
    for a in range(sub):
        for b in range(sub):
            for c in range(sub):
                rr = ax[0][:, a][:, None, None] + ax[1][:, b][None, :, None] + ax[2][:, c][None, None, :]
                inside += (rr < R * R)
    rho_out = 1.0 / (1.0 + 4.0 * math.pi / 3.0 * delta * (R / B) ** 3)
    return rho_out * (1.0 + delta * inside / sub ** 3)


def refine_flags(eta: np.ndarray, level: int, m_ref: float = 8.0, expand: int = 1, periodic: bool = False,
                 within: np.ndarray | None = None) -> np.ndarray:
    """Bool flags of the cells of refinement level `level` - 1 (cell volume 8^-(level-1) of a domain cell) that
    level `level` refines: eta 8^-(level-1) >= m_ref, dilated `expand` times by the six face neighbours, and
    kept inside `within` (the parent level's refined cells) when given."""
    f = eta * 8.0 ** (-(level - 1)) >= m_ref
    for _ in range(expand):
        g = f.copy()
        for ax in range(3):
            for sh in (-1, 1):
                if periodic:
                    g |= np.roll(f, sh, axis=ax)
                else:
                    r = np.zeros_like(f)
                    src = [slice(None)] * 3
                    dst = [slice(None)] * 3
                    src[ax] = slice(0, -1) if sh == 1 else slice(1, None)
                    dst[ax] = slice(1, None) if sh == 1 else slice(0, -1)
                    r[tuple(dst)] = f[tuple(src)]
                    g |= r
        f = g
    if within is not None:
        f &= within
    return f


def patch_box(flags: np.ndarray, margin: int = 1, multiple: int = 8, periodic: bool = False):
    """(origin, n) of the box of parent cells holding every flag with `margin` unflagged cells round it, n
    rounded up to a multiple of `multiple` (to the next even size where a non-periodic parent has no room for
    that); None without flags.  A non-periodic parent keeps one more cell outside the box on each side (the
    interpolation's stencil); a periodic box may wrap."""
    idx = np.argwhere(flags)
    if len(idx) == 0:
        return None
    pn = flags.shape
    origin, n = [], []
    for a in range(3):
        lo, hi = int(idx[:, a].min()) - margin, int(idx[:, a].max()) + margin + 1
        if periodic:
            # the flagged coordinates may wrap round the domain: start after the largest circular gap
            occ = np.unique(idx[:, a])
            gaps = np.diff(np.concatenate([occ, occ[:1] + pn[a]]))
            g = int(np.argmax(gaps))
            start = int(occ[(g + 1) % len(occ)])
            span = int(occ[g]) - start
            span = span + pn[a] if span < 0 else span
            lo, hi = start - margin, start + span + margin + 1
        need = hi - lo
        size = -(-need // multiple) * multiple
        if not periodic and size > pn[a] - 2:
            size = need + (need & 1)
        lo0, hi0 = lo, hi
        lo -= (size - need) // 2
        if not periodic:
            lo = max(1, min(lo, pn[a] - 1 - size))
            if lo > lo0 or lo + size < hi0 or lo + size + 1 > pn[a]:
                raise ValueError("the flagged region does not fit inside its parent")
        elif size > pn[a]:
            raise ValueError("the flagged region is wider than the domain")
        origin.append(lo % pn[a] if periodic else lo)
        n.append(size)
    return tuple(origin), tuple(n)


def box_flags(flags: np.ndarray, origin, n, periodic: bool) -> np.ndarray:
    """The flags of a box's parent cells (uint8, n dims; a periodic box wraps)."""
    pn = flags.shape
    ix = [np.arange(origin[a], origin[a] + n[a]) % pn[a] if periodic else np.arange(origin[a], origin[a] + n[a])
          for a in range(3)]
    return np.ascontiguousarray(flags[np.ix_(*ix)].astype(np.uint8))


def sinusoid(N: int, m: int = 1, amp: float = 1.0, axis: int = 0) -> torch.Tensor:
    """amp * sin(2 pi m (i + 1/2) / N) along one axis (cell centres)."""
    i = (torch.arange(N, dtype=torch.float64) + 0.5)
    v = amp * torch.sin(2 * math.pi * m * i / N)
    shape = [1, 1, 1]
    shape[axis] = N
    return v.view(shape).expand(N, N, N).contiguous()
