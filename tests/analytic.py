"""Closed-form solutions of the continuous Oldroyd-B equations used to pin the oracle.

Everything here is derived from the paper's continuum model (Eq. (stokes) with the
polymer force of Eq. (dtau), and the constitutive Eq. (oldroydb)), not from the
discrete scheme, so it is independent of the oracle's arithmetic.
"""
from __future__ import annotations

import math

import numpy as np


def poiseuille_u(y, g, eta, y0, y1):
    """Steady plane Poiseuille velocity between no-slip walls at y0 < y1, body force g."""
    y = np.asarray(y, dtype=np.float64)
    return g / (2.0 * eta) * (y - y0) * (y1 - y)


def poiseuille_shear_rate(y, g, eta, y0, y1):
    y = np.asarray(y, dtype=np.float64)
    return g / (2.0 * eta) * ((y1 - y) - (y - y0))


def oldroydb_simple_shear(eta_p, lam, gdot):
    """Steady Oldroyd-B stress of u_i = gdot * r_j: (tau_ij, tau_ii, tau_jj)."""
    return eta_p * gdot, 2.0 * eta_p * lam * gdot * gdot, 0.0


def oldroydb_uniaxial(eta_p, lam, edot):
    """Steady stress in uniaxial extension u = edot (x, -y/2, -z/2): (tau_xx, tau_yy=tau_zz)."""
    return 2.0 * eta_p * edot / (1.0 - 2.0 * lam * edot), -eta_p * edot / (1.0 + lam * edot)


def oldroydb_planar(eta_p, lam, edot):
    """Steady stress in planar extension u = edot (x, -y, 0): (tau_xx, tau_yy, tau_zz)."""
    return 2.0 * eta_p * edot / (1.0 - 2.0 * lam * edot), -2.0 * eta_p * edot / (1.0 + 2.0 * lam * edot), 0.0


def startup_poiseuille(t, y, *, g, rho, eta_n, eta_p, lam, L, nmodes=401):
    """Start-up of plane Poiseuille flow of an Oldroyd-B fluid from rest.

    Unidirectional flow u_x(y, t) between walls at y=0 and y=L.  The x-momentum and
    the xy constitutive equation are linear:
        rho du/dt = eta_n u'' + d tau_xy/dy + g,     lam d tau_xy/dt + tau_xy = eta_p u'.
    With u = sum a_n sin(k_n y), tau_xy = sum b_n cos(k_n y), k_n = n pi / L (odd n carry
    the forcing 4 g/(n pi)), each mode is a 2x2 linear ODE with constant forcing,
    solved here exactly through its eigen-decomposition.  Returns u[t, y].
    """
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    u = np.zeros((t.size, y.size))
    for n in range(1, nmodes + 1, 2):
        k = n * math.pi / L
        A = np.array([[-eta_n * k * k / rho, -k / rho], [eta_p * k / lam, -1.0 / lam]])
        b = np.array([4.0 * g / (n * math.pi * rho), 0.0])
        xs = -np.linalg.solve(A, b)  # steady state of the mode
        ev, V = np.linalg.eig(A)
        c0 = np.linalg.solve(V, -xs)  # x(0) = 0  ->  x = xs + V exp(ev t) c0
        tr = (V[0, :][None, :] * np.exp(np.outer(t, ev)) * c0[None, :]).sum(axis=1).real
        a_n = xs[0] + tr
        u += np.outer(a_n, np.sin(k * y))
    return u


def startup_newtonian_centre(t, *, g, rho, eta, L, nmodes=401):
    """Newtonian start-up centre velocity (same series with eta_p = 0)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    nu = eta / rho
    u = np.zeros(t.size)
    for n in range(1, nmodes + 1, 2):
        k = n * math.pi / L
        amp = 4.0 * g / (n * math.pi * eta * k * k)
        u += amp * (1.0 - np.exp(-nu * k * k * t)) * math.sin(k * L / 2)
    return u


def four_roll_mill_newtonian(F, k, eta):
    """Steady Stokes flow under the four-roll-mill force F0 (sin kx cos ky, -cos kx sin ky):
    the field is divergence free and an eigenfunction of the Laplacian (eigenvalue -2 k^2),
    so eta lap u + F = 0 with no pressure gradient gives u = F / (2 k^2 eta) (any frame)."""
    return np.asarray(F) / (2.0 * k * k * eta)
