"""Seeded synthetic inputs shaped like the paper's workloads (geometry, initial fields).

These generators hold none of the method's arithmetic: they only build flag fields,
random initial velocities and stresses, and the parameter sets of the benchmark
configurations.  Both the CUDA library and the CPU oracle are fed from here.
Arrays use the (…, nz, ny, nx) layout of the C ABI (x fastest).
"""
from __future__ import annotations

import math

import numpy as np

FLUID, NOSLIP, WALL0 = 0, 1, 2


def channel_flags(shape, wall_axis=1, top_flag=NOSLIP, bottom_flag=NOSLIP):
    """Channel with solid first and last layers along wall_axis (0=x, 1=y, 2=z)."""
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    ax = 2 - wall_axis
    idx = [slice(None)] * 3
    idx[ax] = 0
    fl[tuple(idx)] = bottom_flag
    idx[ax] = -1
    fl[tuple(idx)] = top_flag
    return fl


def sphere_mask(shape, centre, radius):
    """Cells whose centre (integer coordinates) lies within radius of centre."""
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2) <= radius * radius


def random_obstacles(shape, fraction, seed):
    """Seeded Bernoulli(fraction) no-slip obstacles."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    return (rng.random((nz, ny, nx)) < fraction).astype(np.uint8)


def random_velocity(shape, amplitude, seed):
    """u ~ U(-amplitude, amplitude) per component and cell."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    return rng.uniform(-amplitude, amplitude, (3, nz, ny, nx))


def random_stress(shape, amplitude, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    return amplitude * rng.standard_normal((6, nz, ny, nx))


# ---------------------------------------------------------------------------------
# the benchmark configurations
# ---------------------------------------------------------------------------------
def config_channel(nx=4, ny=32, nz=4):
    """Plain method, FP64: periodic channel with walls at y=0 and y=ny-1, g=1e-6 along x,
    rho0=1, eta=1/6, beta=0.5, lambda=3000, zero initial velocity and stress."""
    return {
        "shape": (nx, ny, nz),
        "params": dict(periodic=(1, 0, 1), eta=1.0 / 6.0, beta=0.5, lambda_p=3000.0, rho0=1.0,
                       body_force=(1e-6, 0.0, 0.0)),
        "flags": channel_flags((nx, ny, nz), 1),
        "wall_vel": (),
        "steps": 20000,
    }


def duct_centreline_factor(aspect=1.0, terms=60):
    """u_c = factor * g H^2 / eta for a square duct of side H (textbook Fourier series)."""
    s = 0.0
    for n in range(1, 2 * terms, 2):
        x = n * math.pi * aspect / 2.0
        sech = 0.0 if x > 700.0 else 1.0 / math.cosh(x)  # cosh overflows beyond ~710
        s += (-1) ** ((n - 1) // 2) / n ** 3 * (1.0 - sech)
    return 4.0 / math.pi ** 3 * s / 1.0


def config_sphere_duct(n=128, radius=12.0, beta=0.5, wi=0.5, g=5e-6, eta=1.0):
    """Fixed complex boundary: n^3 box periodic in x, no-slip walls in y and z, a fixed
    sphere (wall class 0, zero velocity) at the centre, body force g along x.  lambda is
    set from Wi = lambda u_ref / R with u_ref the empty-duct centreline velocity."""
    shape = (n, n, n)
    fl = np.zeros((n, n, n), np.uint8)
    fl[:, 0, :] = NOSLIP
    fl[:, -1, :] = NOSLIP
    fl[0, :, :] = NOSLIP
    fl[-1, :, :] = NOSLIP
    c = (n - 1) / 2.0
    fl[sphere_mask(shape, (c, c, c), radius)] = WALL0
    H = n - 2.0
    u_ref = duct_centreline_factor() * g * H * H / eta
    lam = wi * radius / u_ref
    return {
        "shape": shape,
        "params": dict(periodic=(1, 0, 0), eta=eta, beta=beta, lambda_p=lam, rho0=1.0, body_force=(g, 0.0, 0.0)),
        "flags": fl,
        "wall_vel": [(0.0, 0.0, 0.0)],
        "steps": 50000,
        "u_ref": u_ref,
    }


def config_throughput(n=512, seed=0, obstacle_fraction=0.01, beta=0.5, lam=1000.0, nz=None):
    """Throughput, single large domain: n^3 periodic box (n x n x nz when nz is given), 1 %
    seeded Bernoulli obstacles, u ~ U(-1e-3, 1e-3), zero stress, beta=0.5, lambda=1000,
    eta=1/6."""
    shape = (n, n, n if nz is None else nz)
    return {
        "shape": shape,
        "params": dict(periodic=(1, 1, 1), eta=1.0 / 6.0, beta=beta, lambda_p=lam, rho0=1.0,
                       body_force=(0.0, 0.0, 0.0)),
        "flags_fn": lambda: random_obstacles(shape, obstacle_fraction, seed),
        "u_fn": lambda: random_velocity(shape, 1e-3, seed + 1),
        "steps": 1000,
    }


# ---------------------------------------------------------------------------------
# two-dimensional workloads (D2Q9 / D2Q5)
# ---------------------------------------------------------------------------------
def cavity2d(L=194, u0=1e-4, beta=0.5, wi=0.5, eta_n=1.0):
    """Lid-driven cavity of Sec. "Lid-driven cavity": an L x L fluid cell inside solid
    walls (grid (L + 2)^2, halfway walls at 0.5 and L + 0.5), the top wall moving along x
    with the regularised profile 16 u0 xi^2 (1 - xi)^2, xi = (x - 0.5) / L clamped to
    [0, 1] and evaluated at the solid cell's centre.  eta_n is the Newtonian viscosity,
    eta_p = beta / (1 - beta) eta_n, Wi = lambda u0 / L."""
    n = L + 2
    fl = np.ones((n, n), np.uint8)
    fl[1:-1, 1:-1] = 0
    ub = np.zeros((2, n, n))
    xi = np.clip((np.arange(n) - 0.5) / L, 0.0, 1.0)
    ub[0, -1, :] = 16.0 * u0 * xi ** 2 * (1.0 - xi) ** 2
    eta = eta_n / (1.0 - beta)
    lam = max(wi * L / u0, 1.0)
    return {"shape": (n, n), "flags": fl, "ub": ub,
            "params": dict(periodic=(0, 0), eta=eta, beta=beta, lambda_p=lam, body_force=(0.0, 0.0))}


def four_roll_mill2d(N=214, u0=1e-3, beta=1.0 / 3.0, eta_n=1.5, wi=0.5, rotated=True):
    """Four-roll mill of Sec. "Four-roll mill" on an N x N periodic lattice.  The force
    density F0 (sin kx cos ky, -cos kx sin ky), F0 = 8 pi^2 eta_n u0 / L^2, k = 2 pi / L,
    drives four counter-rotating rolls (the printed second component carries no minus
    sign, which would make the field a pure gradient that drives no flow).  rotated: the
    lattice is turned by 45 degrees against the system, x = (x' + y') / sqrt 2,
    y = (y' - x') / sqrt 2, with L = N sqrt 2 so that the N x N lattice stays periodic;
    else L = N.  Returns the force field at the cell centres in lattice components
    (2, N, N), L, k and the parameters (Wi = 4 pi lambda u0 / L)."""
    L = N * math.sqrt(2.0) if rotated else float(N)
    k = 2.0 * math.pi / L
    yl, xl = np.meshgrid(np.arange(N, dtype=float), np.arange(N, dtype=float), indexing="ij")
    if rotated:
        x = (xl + yl) / math.sqrt(2.0)
        y = (yl - xl) / math.sqrt(2.0)
    else:
        x, y = xl, yl
    F0 = 8.0 * math.pi ** 2 * eta_n * u0 / L ** 2
    Fs = np.stack([F0 * np.sin(k * x) * np.cos(k * y), -F0 * np.cos(k * x) * np.sin(k * y)])
    if rotated:  # system components -> lattice components
        F = np.stack([(Fs[0] - Fs[1]) / math.sqrt(2.0), (Fs[0] + Fs[1]) / math.sqrt(2.0)])
    else:
        F = Fs
    eta = eta_n / (1.0 - beta)
    lam = max(wi * L / (4.0 * math.pi * u0), 1.0)
    return {"shape": (N, N), "force": F, "L": L, "k": k,
            "params": dict(periodic=(1, 1), eta=eta, beta=beta, lambda_p=lam, body_force=(0.0, 0.0))}
