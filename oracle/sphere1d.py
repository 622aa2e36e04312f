"""Spherically symmetric solutions for the static sphere test of Sect. 5.1 ("Potential solver").

TEST INFRASTRUCTURE ONLY.  The paper checks its grid solutions against the same equations written in
spherical coordinates and solved as a 1D boundary-value problem; this module is that 1D solve, in FP64,
independent of both the CUDA path and the 3D oracle:
  - Newtonian potential:  (1/r^2)(r^2 Phi')' = K (eta - eta_mean)               (Sect. 3.1)
  - symmetron:            (1/r^2)(r^2 chi')' = A [(s eta - 1) chi + chi^3]         (Sect. 4.1, Eq. (symmetron_dimensionles))
  - Hu-Sawicki f(R):      (1/r^2)(r^2 e^u u')' = K1 (eta - 1) - K2 e^{-u/(n+1)} + K3 (Sect. 4.2)
Finite volumes on M radial cells r_i = (i + 1/2) dr of [0, R_max]: zero flux at r = 0, the far-field value
held at r = R_max (a ghost cell), f(R) face coefficient b = (e^{u_i} + e^{u_i+1})/2 (the paper's face mean).
The density is the sphere profile of Sect. 5.1 with the straddling cell's eta its volume average.
Newton iterations with a tridiagonal Jacobian, step halving while the residual norm does not fall.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import solve_banded

H0_MPC = 1.0 / 2997.92458


def sphere_profile(r_edges: np.ndarray, R: float, eta_in: float, eta_out: float) -> np.ndarray:
    """Volume-averaged eta of each radial cell [r_edges[i], r_edges[i+1]] for a uniform sphere of radius R."""
    lo, hi = r_edges[:-1], r_edges[1:]
    inside = np.clip(np.minimum(hi, R) ** 3 - lo ** 3, 0.0, None) / (hi ** 3 - lo ** 3)
    return eta_out + (eta_in - eta_out) * inside


def sphere_densities(delta: float, R: float, B: float):
    """eta_in, eta_out of Sect. 5.1 (mean density 1 in a box of side B)."""
    eta_out = 1.0 / (1.0 + 4.0 * math.pi / 3.0 * delta * (R / B) ** 3)
    return (1.0 + delta) * eta_out, eta_out


class Radial:
    """The finite-volume radial Laplacian of M cells of width dr."""

    def __init__(self, M: int, R_max: float):
        self.M, self.dr = M, R_max / M
        self.r = (np.arange(M) + 0.5) * self.dr
        self.edges = np.arange(M + 1) * self.dr
        self.vol = (self.edges[1:] ** 3 - self.edges[:-1] ** 3) / 3.0  # per unit solid angle

    def div_flux(self, u: np.ndarray, u_far: float, b: np.ndarray | None = None):
        """(1/V_i) sum of face fluxes r_f^2 b_f (u_nb - u_i)/dr, and its derivatives d/du_i, d/du_{i+-1}
        for a constant b (b = None) or face coefficients from per-cell b (arithmetic mean)."""
        M, dr = self.M, self.dr
        ue = np.append(u, u_far)
        area = self.edges[1:] ** 2  # outer face of cell i
        if b is None:
            bf = np.ones(M)
        else:
            be = np.append(b, b[-1])
            bf = 0.5 * (be[:-1] + be[1:])
        flux_out = area * bf * (ue[1:] - ue[:-1]) / dr  # through the outer face of cell i
        flux_in = np.concatenate([[0.0], flux_out[:-1]])  # through the inner face (zero at r = 0)
        return (flux_out - flux_in) / self.vol, area, bf


def _newton(resid_jac, u0, tol=1e-12, max_it=200):
    u = u0.copy()
    F, ab = resid_jac(u)
    nrm = np.linalg.norm(F)
    for _ in range(max_it):
        du = solve_banded((1, 1), ab, -F)
        step = 1.0
        while True:
            un = u + step * du
            Fn, abn = resid_jac(un)
            nn = np.linalg.norm(Fn)
            if np.isfinite(nn) and (nn < nrm or step < 1e-6):
                break
            step *= 0.5
        u, F, ab, nrm_old, nrm = un, Fn, abn, nrm, nn
        if np.max(np.abs(step * du)) <= tol * max(1.0, np.max(np.abs(u))):
            return u
    raise RuntimeError("radial Newton did not converge")


def symmetron(eta: np.ndarray, rad: Radial, A: float, s: float, chi_far: float, chi0=None) -> np.ndarray:
    """chi(r) of (1/r^2)(r^2 chi')' = A [(s eta - 1) chi + chi^3], chi(R_max) = chi_far."""
    M, dr = rad.M, rad.dr

    def rj(u):
        L, area, bf = rad.div_flux(u, chi_far)
        F = L - A * ((s * eta - 1.0) * u + u ** 3)
        c_out = area * bf / dr / rad.vol
        c_in = np.concatenate([[0.0], (area * bf / dr)[:-1]]) / rad.vol
        diag = -c_out - c_in - A * ((s * eta - 1.0) + 3.0 * u ** 2)
        ab = np.zeros((3, M))
        ab[0, 1:] = c_out[:-1]
        ab[1] = diag
        ab[2, :-1] = c_in[1:]
        return F, ab

    u0 = np.full(M, chi_far) if chi0 is None else chi0
    return _newton(rj, u0)


def poisson(eta: np.ndarray, rad: Radial, K: float, eta_mean: float, phi_far: float) -> np.ndarray:
    """Phi(r) of (1/r^2)(r^2 Phi')' = K (eta - eta_mean), Phi(R_max) = phi_far (linear: one Newton step)."""
    M, dr = rad.M, rad.dr

    def rj(u):
        L, area, bf = rad.div_flux(u, phi_far)
        F = L - K * (eta - eta_mean)
        c_out = area * bf / dr / rad.vol
        c_in = np.concatenate([[0.0], (area * bf / dr)[:-1]]) / rad.vol
        ab = np.zeros((3, M))
        ab[0, 1:] = c_out[:-1]
        ab[1] = -c_out - c_in
        ab[2, :-1] = c_in[1:]
        return F, ab

    return _newton(rj, np.zeros(M))


def fofr(eta: np.ndarray, rad: Radial, K1: float, K2: float, K3: float, n: int, u_far: float) -> np.ndarray:
    """u(r) of (1/r^2)(r^2 e^u u')' = K1 (eta - 1) - K2 e^{-u/(n+1)} + K3, u(R_max) = u_far, from the
    cell-wise uniform-density solution (where S(u, eta) = 0)."""
    M, dr = rad.M, rad.dr
    np1 = n + 1.0

    def rj(u):
        b = np.exp(u)
        L, area, bf = rad.div_flux(u, u_far, b)
        S = K1 * (eta - 1.0) - K2 * np.exp(-u / np1) + K3
        F = L - S
        ue = np.append(u, u_far)
        be = np.append(b, math.exp(u_far))
        g = area / dr / rad.vol
        # d/du_i and d/du_{i+1} of the outer flux area b_f (u_{i+1} - u_i)/dr, b_f = (b_i + b_{i+1})/2
        d_out_i = g * (0.5 * be[:-1] * (ue[1:] - ue[:-1]) - bf)
        d_out_ip = g * (0.5 * be[1:] * (ue[1:] - ue[:-1]) + bf)
        # the inner face of cell i is the outer face of cell i-1, seen with the sign flipped and cell i's volume
        gi = np.concatenate([[0.0], (area / dr)[:-1]]) / rad.vol
        dui = np.concatenate([[0.0], (0.5 * be[1:-1] * (ue[1:-1] - ue[:-2]) + bf[:-1])])  # d(inner flux)/du_i
        duim = np.concatenate([[0.0], (0.5 * be[:-2] * (ue[1:-1] - ue[:-2]) - bf[:-1])])  # d(inner flux)/du_{i-1}
        diag = d_out_i - gi * dui - K2 / np1 * np.exp(-u / np1)
        ab = np.zeros((3, M))
        ab[0, 1:] = d_out_ip[:-1]
        ab[1] = diag
        ab[2, :-1] = -(gi * duim)[1:]
        return F, ab

    u0 = np1 * np.log(K2 / (K1 * (eta - 1.0) + K3))
    return _newton(rj, u0)


def fofr_constants(a: float, Omega_m: float, Omega_L: float, H0: float, n: int, fR0_abs: float):
    """K1, K2, K3 of Sect. 4.2's source."""
    r = Omega_L / Omega_m
    K1 = Omega_m * a * H0 * H0
    K2 = Omega_m * a ** 4 * H0 * H0 * (1 + 4 * r) * (fR0_abs * a * a) ** (1.0 / (n + 1))
    K3 = Omega_m * a * H0 * H0 * (1 + 4 * a ** 3 * r)
    return K1, K2, K3
