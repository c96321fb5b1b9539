"""Brute-force evaluation of one time step, cell by cell, for tiny grids.

TEST INFRASTRUCTURE ONLY.  This is a second, independent statement of the coupled step of
Kuron et al. (arXiv:2009.12279), written directly from the equations in plain Python /
numpy, one cell and one link at a time, for grids of a few cells per side.  It shares no
code with the oracle (it never imports ``oracle/``) and is organised differently on
purpose: the lattice is generated from its definition, the collision and the forcing use
tensor contractions, streaming pulls instead of pushing, and the stress source is written
in matrix form.  ``tests/test_oracle_brute_force.py`` compares one oracle step with it
element by element.

Sub-steps and the passages they follow (the readings are those of the oracle's header):

1. polymer force F^p_j = sum over D3Q7 faces of +-tau_kj(face), face value the mean of the
   two cells or tau(r) towards a solid cell                 Eqs. (force), (interpolation),
                                                            (extrapolation)
2. rho = sum f, u = (sum f c + F/2) / rho, F = g + F^p      Eq. (macroscopic-velocity)
3. stress: d_k u_j from face values (boundary velocity at solid faces), donor-cell face
   fluxes (optionally with the transverse overlap factors), source
   S = tau G + (tau G)^T + (eta_p/lambda)(G + G^T) - tau/lambda (+ tau tr G, Giesekus
   -(alpha/eta_p) tau.tau), explicit Euler                   Eqs. (continuity)-(source)
4. TRT collision with Guo forcing                           Eqs. (lb), (lb-equilibrium), (guo)
5. streaming with link bounce-back, moving-wall term -6 w rho c.u_b, and momentum
   exchange c (2 f* - 6 w rho c.u_b) on links into wall classes and particles
                                                            Eq. (ubb), Sec. "Moving boundaries"
6. particle update, symplectic Euler                        Sec. "Moving boundaries"
7. re-voxelisation, fill/drain with stress redistribution  Sec. "Moving boundaries"
"""
from __future__ import annotations

import itertools
import math

import numpy as np

FLUID, NOSLIP, WALL0, PART0 = 0, 1, 2, 64


def d3q19():
    """Velocities c with components in {-1, 0, 1} and |c|^2 <= 2, weights by |c|^2
    (1/3, 1/18, 1/36), in lexicographic order of (cx, cy, cz)."""
    cs, ws = [], []
    for c in itertools.product((-1, 0, 1), repeat=3):
        s = c[0] ** 2 + c[1] ** 2 + c[2] ** 2
        if s <= 2:
            cs.append(c)
            ws.append({0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}[s])
    c = np.array(cs, dtype=np.int64)
    w = np.array(ws)
    opp = np.array([cs.index((-a, -b, -d)) for (a, b, d) in cs])
    return c, w, opp


C, W, OPP = d3q19()
MOVING = [i for i in range(19) if C[i].any()]  # the 18 non-rest velocities
FACES = [np.array(v) for v in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))]


class Particle:
    def __init__(self, X, R, rho_p, v=(0, 0, 0), w=(0, 0, 0), Fext=(0, 0, 0), Text=(0, 0, 0)):
        self.X = np.array(X, float)
        self.R = float(R)
        self.v = np.array(v, float)
        self.w = np.array(w, float)
        self.Fext = np.array(Fext, float)
        self.Text = np.array(Text, float)
        self.m = rho_p * 4.0 / 3.0 * math.pi * R ** 3
        self.I = 2.0 / 5.0 * self.m * R ** 2
        self.F = np.zeros(3)
        self.T = np.zeros(3)


class Grid:
    """State of a tiny solve: f[q][x, y, z], tau as 3x3 matrices per cell, flags."""

    def __init__(self, shape, periodic, eta, beta, lambda_p, rho0, g, magic, wall_vel, fv_flux, fv_source,
                 fv_ctu, fv_divu, giesekus_alpha):
        self.shape = tuple(shape)
        self.periodic = tuple(bool(p) for p in periodic)
        self.rho0 = rho0
        self.g = np.array(g, float)
        self.wall_vel = [np.array(v, float) for v in wall_vel]
        eta_n = (1.0 - beta) * eta
        self.omega_p = 1.0 / (3.0 * eta_n / rho0 + 0.5)
        self.omega_m = 1.0 / (magic / (1.0 / self.omega_p - 0.5) + 0.5)
        self.eta_p = beta * eta
        self.lam = lambda_p
        self.flux, self.source, self.ctu, self.divu = fv_flux, fv_source, fv_ctu, fv_divu
        self.alpha = giesekus_alpha
        self.particles: list[Particle] = []
        self.body_force = {}
        self.destroyed = self.created = 0
        self.dropped = np.zeros((3, 3))

    # -- geometry -------------------------------------------------------------------
    def cells(self):
        nx, ny, nz = self.shape
        return [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]

    def nb(self, r, d):
        """Neighbour r + d with periodic wrap, None outside a closed side."""
        q = []
        for a in range(3):
            v = r[a] + int(d[a])
            if not 0 <= v < self.shape[a]:
                if not self.periodic[a]:
                    return None
                v %= self.shape[a]
            q.append(v)
        return tuple(q)

    def fluid(self, flags, r):
        return r is not None and flags[r] == FLUID

    def image(self, r, X):
        """Minimum-image displacement of cell centre r from point X."""
        d = np.array(r, float) - X
        for a in range(3):
            if self.periodic[a]:
                L = self.shape[a]
                d[a] -= L * math.floor(d[a] / L + 0.5)
        return d

    def u_boundary(self, flags, r):
        """Velocity of the solid cell r: 0 (no-slip or outside), the wall class velocity
        (Eq. (ubb)), or the rigid-body velocity v + omega x (r - X) of a particle."""
        if r is None:
            return np.zeros(3)
        fl = int(flags[r])
        if WALL0 <= fl < PART0:
            k = fl - WALL0
            return self.wall_vel[k].copy() if k < len(self.wall_vel) else np.zeros(3)
        if fl >= PART0:
            P = self.particles[fl - PART0]
            return P.v + np.cross(P.w, self.image(r, P.X))
        return np.zeros(3)

    # -- per-cell formulas ----------------------------------------------------------
    @staticmethod
    def equilibrium(rho, u):
        cu = C @ u
        return W * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * (u @ u))

    def forcing(self, u, F):
        """Guo forcing split for TRT: w [3 (1 - w-/2) c.F + 9/2 (1 - w+/2) (uF + Fu):(cc - I/3)]."""
        out = np.zeros(19)
        S = np.outer(u, F) + np.outer(F, u)
        for i in range(19):
            Q = np.outer(C[i], C[i]) - np.eye(3) / 3.0
            out[i] = W[i] * (3.0 * (1.0 - self.omega_m / 2.0) * (C[i] @ F)
                             + 4.5 * (1.0 - self.omega_p / 2.0) * np.sum(S * Q))
        return out

    def collide(self, f, rho, u, F):
        feq = self.equilibrium(rho, u)
        sym = lambda a: 0.5 * (a + a[OPP])  # noqa: E731
        anti = lambda a: 0.5 * (a - a[OPP])  # noqa: E731
        return (f - self.omega_p * (sym(f) - sym(feq)) - self.omega_m * (anti(f) - anti(feq))
                + self.forcing(u, F))

    # -- one step ----------------------------------------------------------------------
    def step(self, f, tau, flags):
        """One time step.  f: dict cell -> 19 PDFs, tau: dict cell -> 3x3, flags: ndarray
        indexed by cell.  Returns new (f, tau, flags); fluid cells' entries are the
        meaningful ones."""
        cells = self.cells()
        fluid = [r for r in cells if self.fluid(flags, r)]

        # 1-2: polymer force and moments
        rho, u, F = {}, {}, {}
        for r in fluid:
            Fp = np.zeros(3)
            for e in FACES:
                k = int(np.nonzero(e)[0][0])
                s = float(e[k])
                n = self.nb(r, e)
                face = 0.5 * (tau[r] + tau[n]) if self.fluid(flags, n) else tau[r]
                Fp += s * face[k, :]
            F[r] = self.g + Fp
            rho[r] = float(np.sum(f[r]))
            u[r] = (C.T @ f[r] + 0.5 * F[r]) / rho[r]

        # 3: finite-volume stress update from tau^t, u^t
        tau_new = {r: np.zeros((3, 3)) for r in cells}
        for r in fluid:
            T = tau[r]
            G = np.zeros((3, 3))  # G[k, j] = d_k u_j
            for k in range(3):
                e = np.zeros(3, int)
                e[k] = 1
                up_n, um_n = self.nb(r, e), self.nb(r, -e)
                up = 0.5 * (u[r] + u[up_n]) if self.fluid(flags, up_n) else self.u_boundary(flags, up_n)
                um = 0.5 * (u[r] + u[um_n]) if self.fluid(flags, um_n) else self.u_boundary(flags, um_n)
                G[k, :] = up - um
            net = np.zeros((3, 3))
            if self.flux:
                for e in FACES:
                    k = int(np.nonzero(e)[0][0])
                    s = float(e[k])
                    n = self.nb(r, e)
                    if not self.fluid(flags, n):
                        continue  # no flux across a solid link
                    a, b = [m for m in range(3) if m != k]
                    out_rate = max(s * u[r][k], 0.0)
                    in_rate = max(-s * u[n][k], 0.0)
                    if self.ctu:
                        out_rate *= (1.0 - abs(u[r][a])) * (1.0 - abs(u[r][b]))
                        in_rate *= (1.0 - abs(u[n][a])) * (1.0 - abs(u[n][b]))
                    net += out_rate * T - in_rate * tau[n]
            S = np.zeros((3, 3))
            if self.source:
                TG = T @ G
                S = TG + TG.T + (self.eta_p / self.lam) * (G + G.T) - T / self.lam
                if self.alpha != 0.0:
                    S -= (self.alpha / self.eta_p) * (T @ T)
            if self.divu:
                S += T * np.trace(G)
            tau_new[r] = T - net + S

        # 4: collision
        fstar = {r: self.collide(f[r], rho[r], u[r], F[r]) for r in fluid}

        # 5: streaming (pull) with bounce-back; momentum exchange
        f_new = {r: np.array(f[r], float) for r in cells}
        for r in fluid:
            for i in range(19):
                src = self.nb(r, -C[i])
                if self.fluid(flags, src):
                    f_new[r][i] = fstar[src][i]
                else:
                    # f*_{-i}(r) ran into the solid cell r - c_i and comes back as f_i(r)
                    j = OPP[i]
                    ub = self.u_boundary(flags, src)
                    f_new[r][i] = fstar[r][j] - 6.0 * W[j] * rho[r] * (C[j] @ ub)
        self.body_force = {}
        for P in self.particles:
            P.F = np.zeros(3)
            P.T = np.zeros(3)
        for r in fluid:
            for i in MOVING:
                n = self.nb(r, C[i])
                if n is None or int(flags[n]) < WALL0:
                    continue
                ub = self.u_boundary(flags, n)
                Fl = C[i] * (2.0 * fstar[r][i] - 6.0 * W[i] * rho[r] * (C[i] @ ub))
                fl = int(flags[n])
                self.body_force[fl] = self.body_force.get(fl, np.zeros(3)) + Fl
                if fl >= PART0:
                    P = self.particles[fl - PART0]
                    P.F = P.F + Fl
                    P.T = P.T + np.cross(self.image(n, P.X), Fl)

        # 6: particles, symplectic Euler
        for P in self.particles:
            P.v = P.v + (P.F + P.Fext) / P.m
            P.w = P.w + (P.T + P.Text) / P.I
            P.X = P.X + P.v

        # 7: fill/drain
        if self.particles:
            f_new, tau_new, flags = self.fill_drain(f_new, tau_new, flags)
        return f_new, tau_new, flags

    def owner(self, r):
        for q, P in enumerate(self.particles):
            d = self.image(r, P.X)
            if d @ d <= P.R * P.R:
                return q
        return None

    def fill_drain(self, f, tau, flags):
        cells = self.cells()
        new = flags.copy()
        for r in cells:
            if flags[r] == FLUID or flags[r] >= PART0:
                q = self.owner(r)
                new[r] = FLUID if q is None else PART0 + q
        was = {r: flags[r] == FLUID for r in cells}
        now = {r: new[r] == FLUID for r in cells}
        stable = {r for r in cells if was[r] and now[r]}
        destroyed = [r for r in cells if was[r] and not now[r]]
        created = [r for r in cells if now[r] and not was[r]]

        def face_nbs(r):
            return [n for n in (self.nb(r, e) for e in FACES) if n is not None and n in stable]

        Nf = {r: len(face_nbs(r)) for r in destroyed + created}
        t_created = {r: sum((tau[n] for n in face_nbs(r)), np.zeros((3, 3))) / (Nf[r] + 1) for r in created}
        dP = [np.zeros(3) for _ in self.particles]
        dL = [np.zeros(3) for _ in self.particles]
        for r in destroyed:  # the deleted populations' momentum goes to the particle
            q = int(new[r]) - PART0
            Pm = C.T @ f[r]
            dP[q] = dP[q] + Pm
            dL[q] = dL[q] + np.cross(self.image(r, self.particles[q].X), Pm)
            if Nf[r] == 0:
                self.dropped += tau[r]
            self.destroyed += 1
        f_created = {}
        for r in created:  # new fluid at equilibrium with the surface velocity
            q = int(flags[r]) - PART0
            P = self.particles[q]
            dens = [float(np.sum(f[n])) for n in (self.nb(r, C[i]) for i in MOVING)
                    if n is not None and n in stable]
            rho_bar = sum(dens) / len(dens) if dens else self.rho0
            d = self.image(r, P.X)
            feq = self.equilibrium(rho_bar, P.v + np.cross(P.w, d))
            f_created[r] = feq
            Pm = C.T @ feq
            dP[q] = dP[q] - Pm
            dL[q] = dL[q] - np.cross(d, Pm)
            self.created += 1
        tau_out = dict(tau)
        for r in stable:  # each converted face neighbour shares its stress with its N_f cells
            t = tau[r].copy()
            for n in (self.nb(r, e) for e in FACES):
                if n in Nf and n in destroyed:
                    t = t + tau[n] / Nf[n]
                elif n in Nf and n in created:
                    t = t - t_created[n] / Nf[n]
            tau_out[r] = t
        for r in destroyed:
            tau_out[r] = np.zeros((3, 3))
        for r in created:
            tau_out[r] = t_created[r]
            f[r] = f_created[r]
        for q, P in enumerate(self.particles):
            P.v = P.v + dP[q] / P.m
            P.w = P.w + dL[q] / P.I
        return f, tau_out, new

    def place(self, P: Particle, flags, tau):
        """Add a particle: covered fluid cells become particle cells (no impulse)."""
        self.particles.append(P)
        q = len(self.particles) - 1
        for r in self.cells():
            d = self.image(r, P.X)
            if flags[r] == FLUID and d @ d <= P.R * P.R:
                flags[r] = PART0 + q
                tau[r] = np.zeros((3, 3))
