"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks one part of the oracle against something other than the oracle's
own formula: lattice isotropy, moment identities, exact balance laws, textbook
closed forms of Oldroyd-B flows and the analytic start-up transient.  A plausible
mistake (dropped term, wrong sign, transposed index) in any sub-step fails at least
one of them.
"""
import math

import numpy as np
import pytest

import analytic as A

RNG = np.random.default_rng(12279)


def _channel_flags(shape, wall_axis):
    nx, ny, nz = shape
    fl = np.zeros((nz, ny, nx), np.uint8)
    idx = [slice(None)] * 3
    ax = 2 - wall_axis  # numpy axis of the wall-normal direction
    idx[ax] = 0
    fl[tuple(idx)] = 1
    idx[ax] = -1
    fl[tuple(idx)] = 1
    return fl


def _line(arr, wall_axis):
    """1-D profile along wall_axis of a (nz, ny, nx) field in a 1-cell-thick channel."""
    return np.moveaxis(arr, 2 - wall_axis, 0).reshape(arr.shape[2 - wall_axis], -1)[:, 0]


# ----------------------------------------------------------------------------------
# lattice and local operators
# ----------------------------------------------------------------------------------
def test_lattice_isotropy(oracle_mod):
    """D3Q19 weights and velocities: moments up to fourth order are those of a Maxwellian
    with c_s^2 = 1/3 (Sec. "Lattice Boltzmann")."""
    c, w, opp = oracle_mod.lattice()
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3.0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(m4, iso, atol=1e-16)
    assert np.array_equal(c[opp], -c)
    assert (np.abs(c).sum(axis=1) <= 2).all() and len({tuple(v) for v in c}) == 19


def test_equilibrium_moments(oracle_mod):
    """Eq. (lb-equilibrium) in its second-order reading has moments rho, rho u, rho(uu + I/3)."""
    c, w, _ = oracle_mod.lattice()
    for _ in range(20):
        rho = 1.0 + 0.1 * RNG.standard_normal()
        u = 0.05 * RNG.standard_normal(3)
        feq = oracle_mod.equilibrium(rho, u)
        assert abs(feq.sum() - rho) < 1e-14
        assert np.allclose(feq @ c, rho * u, atol=1e-15)
        assert np.allclose(np.einsum("i,ia,ib->ab", feq, c, c), rho * (np.outer(u, u) + np.eye(3) / 3.0), atol=1e-15)


def test_forcing_moments(oracle_mod):
    """Guo forcing for TRT (Eq. (guo) reading): zeroth moment 0, first (1 - omega-/2) F,
    second (1 - omega+/2)(uF + Fu)."""
    c, _, _ = oracle_mod.lattice()
    for _ in range(20):
        u = 0.05 * RNG.standard_normal(3)
        F = 1e-3 * RNG.standard_normal(3)
        wp, wm = RNG.uniform(0.5, 1.9), RNG.uniform(0.5, 1.9)
        D = oracle_mod.forcing(u, F, wp, wm)
        assert abs(D.sum()) < 1e-18
        assert np.allclose(D @ c, (1 - wm / 2) * F, rtol=1e-13, atol=1e-19)
        assert np.allclose(np.einsum("i,ia,ib->ab", D, c, c), (1 - wp / 2) * (np.outer(u, F) + np.outer(F, u)),
                           rtol=1e-12, atol=1e-19)


def test_trt_collision_moments(oracle_mod):
    """TRT (Eq. (lb)): mass kept, momentum gains exactly F, even moments relax with omega+
    and odd moments with omega- towards the equilibrium ones, forcing added."""
    c, w, _ = oracle_mod.lattice()
    for _ in range(20):
        rho = 1.0 + 0.05 * RNG.standard_normal()
        u0 = 0.03 * RNG.standard_normal(3)
        f = oracle_mod.equilibrium(rho, u0) + 1e-3 * RNG.standard_normal(19) * w
        F = 1e-4 * RNG.standard_normal(3)
        wp, wm = RNG.uniform(0.6, 1.8), RNG.uniform(0.6, 1.8)
        fs = oracle_mod.collide(f, F, wp, wm)
        rho_ = f.sum()
        j = f @ c
        u = (j + 0.5 * F) / rho_
        assert abs(fs.sum() - rho_) < 1e-14
        assert np.allclose(fs @ c, j + F, atol=1e-16)
        Pi = np.einsum("i,ia,ib->ab", f, c, c)
        Pi_eq = rho_ * (np.outer(u, u) + np.eye(3) / 3.0)
        Pi_s = Pi - wp * (Pi - Pi_eq) + (1 - wp / 2) * (np.outer(u, F) + np.outer(F, u))
        assert np.allclose(np.einsum("i,ia,ib->ab", fs, c, c), Pi_s, atol=1e-15)
        # odd third moment sum_i f c_x c_y^2: equilibrium value rho u_x / 3, forcing (1-wm/2) F_x / 3
        Q = f @ (c[:, 0] * c[:, 1] ** 2)
        Q_s = Q - wm * (Q - rho_ * u[0] / 3.0) + (1 - wm / 2) * F[0] / 3.0
        assert abs(fs @ (c[:, 0] * c[:, 1] ** 2) - Q_s) < 1e-15


def test_rates_from_viscosity(oracle_mod):
    """omega+ from nu_n = (1/omega+ - 1/2)/3 and the magic product 3/16 (config-1 values)."""
    o = oracle_mod.Oracle((2, 2, 2), eta=1.0 / 6.0, beta=0.5, lambda_p=3000.0)
    r = o.rates()
    assert abs(r["omega_p"] - 4.0 / 3.0) < 1e-15
    assert abs((1 / r["omega_p"] - 0.5) * (1 / r["omega_m"] - 0.5) - 3.0 / 16.0) < 1e-15
    assert abs(r["omega_m"] - 0.8) < 1e-15
    assert abs(r["eta_p"] - 1.0 / 12.0) < 1e-16 and abs(r["inv_l"] - 1.0 / 3000.0) < 1e-18


@pytest.mark.parametrize("flow,grad", [(0, 1), (1, 0), (0, 2), (2, 0), (1, 2), (2, 1)])
def test_source_simple_shear_steady(oracle_mod, flow, grad):
    """The textbook steady Oldroyd-B simple-shear stress (tau_fg = eta_p gdot,
    tau_ff = 2 eta_p lam gdot^2, rest 0) zeroes the source of Eq. (source)."""
    eta_p, lam, gdot = 0.3, 700.0, 2e-4
    comp = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}
    G = np.zeros((3, 3))
    G[grad, flow] = gdot  # d_grad u_flow
    txy, txx, _ = A.oldroydb_simple_shear(eta_p, lam, gdot)
    tau = np.zeros(6)
    tau[comp[(flow, grad)]] = txy
    tau[comp[(flow, flow)]] = txx
    S = oracle_mod.source(tau, G, eta_p / lam, 1.0 / lam)
    assert np.abs(S).max() < 1e-12 * txx / lam
    # the lower-convected (wrong) steady state must not be a fixed point
    bad = np.zeros(6)
    bad[comp[(flow, grad)]] = txy
    bad[comp[(grad, grad)]] = -txx
    assert np.abs(oracle_mod.source(bad, G, eta_p / lam, 1.0 / lam)).max() > 1e-3 * txx / lam


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_source_extension_steady(oracle_mod, axis):
    """Steady uniaxial and planar extension stresses of Oldroyd-B zero the source."""
    eta_p, lam, ed = 0.2, 300.0, 4e-4
    perm = [axis, (axis + 1) % 3, (axis + 2) % 3]
    comp_diag = [0, 1, 2]
    # uniaxial: u_a = ed r_a, others -ed/2
    G = np.zeros((3, 3))
    G[perm[0], perm[0]] = ed
    G[perm[1], perm[1]] = -ed / 2
    G[perm[2], perm[2]] = -ed / 2
    txx, tyy = A.oldroydb_uniaxial(eta_p, lam, ed)
    tau = np.zeros(6)
    tau[comp_diag[perm[0]]] = txx
    tau[comp_diag[perm[1]]] = tyy
    tau[comp_diag[perm[2]]] = tyy
    assert np.abs(oracle_mod.source(tau, G, eta_p / lam, 1 / lam)).max() < 1e-12 * abs(txx) / lam
    # planar
    G = np.zeros((3, 3))
    G[perm[0], perm[0]] = ed
    G[perm[1], perm[1]] = -ed
    txx, tyy, tzz = A.oldroydb_planar(eta_p, lam, ed)
    tau = np.zeros(6)
    tau[comp_diag[perm[0]]] = txx
    tau[comp_diag[perm[1]]] = tyy
    assert np.abs(oracle_mod.source(tau, G, eta_p / lam, 1 / lam)).max() < 1e-12 * abs(txx) / lam


# ----------------------------------------------------------------------------------
# finite-volume pieces on fields
# ----------------------------------------------------------------------------------
def test_polymer_force_exact_on_quadratic_stress(oracle_mod):
    """Eq. (force) with linear face interpolation is the exact divergence sum_i d_i tau_ij
    of a quadratic stress field (interior cells away from the periodic seam)."""
    n = 12
    o = oracle_mod.Oracle((n, n, n), beta=0.5, lambda_p=100.0)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    X = [x.astype(float), y.astype(float), z.astype(float)]
    coef = RNG.standard_normal((6, 10)) * 1e-4
    def quad(cf):
        terms = [np.ones_like(X[0]), X[0], X[1], X[2], X[0] ** 2, X[1] ** 2, X[2] ** 2, X[0] * X[1], X[0] * X[2], X[1] * X[2]]
        return sum(a * t for a, t in zip(cf, terms))
    def dquad(cf, ax):
        d = [np.zeros_like(X[0]), np.ones_like(X[0]) * (ax == 0), np.ones_like(X[0]) * (ax == 1), np.ones_like(X[0]) * (ax == 2),
             2 * X[0] * (ax == 0), 2 * X[1] * (ax == 1), 2 * X[2] * (ax == 2),
             X[1] * (ax == 0) + X[0] * (ax == 1), X[2] * (ax == 0) + X[0] * (ax == 2), X[2] * (ax == 1) + X[1] * (ax == 2)]
        return sum(a * t for a, t in zip(cf, d))
    tau = np.stack([quad(coef[c]) for c in range(6)])
    o.write_tau(tau)
    Fp = o.polymer_force()
    comp = [[0, 3, 4], [3, 1, 5], [4, 5, 2]]
    inner = (slice(1, n - 1),) * 3
    for j in range(3):
        exact = sum(dquad(coef[comp[i][j]], i) for i in range(3))
        assert np.allclose(Fp[j][inner], exact[inner], rtol=1e-10, atol=1e-16)


def test_polymer_force_uniform_stress_is_zero_with_walls(oracle_mod):
    """A uniform stress exerts no force anywhere, also next to walls (constant
    extrapolation of Eq. (extrapolation))."""
    n = 10
    o = oracle_mod.Oracle((n, n, n), periodic=(1, 0, 0), beta=0.5, lambda_p=100.0)
    fl = np.zeros((n, n, n), np.uint8)
    fl[0], fl[-1], fl[:, 0], fl[:, -1] = 1, 1, 1, 1
    fl[4:6, 4:6, 3:6] = 1
    o.set_flags(fl)
    tau = np.broadcast_to(RNG.standard_normal(6)[:, None, None, None], (6, n, n, n)).copy()
    o.write_tau(tau)
    assert np.abs(o.polymer_force()).max() < 1e-15


def test_polymer_force_sums_to_zero_periodic(oracle_mod):
    """In a fully periodic box sum_r F^p(r) telescopes to zero."""
    n = 8
    o = oracle_mod.Oracle((n, n + 1, n + 2), beta=0.5, lambda_p=100.0)
    o.write_tau(RNG.standard_normal((6, n + 2, n + 1, n)))
    assert np.abs(o.polymer_force().sum(axis=(1, 2, 3))).max() < 1e-12


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_upwind_advection_is_multinomial(oracle_mod, sign):
    """Donor-cell advection (Sec. "Stability improvements") of a point stress by a
    uniform velocity spreads it as a multinomial distribution after k steps."""
    n = 16
    o = oracle_mod.Oracle((n, n, n), beta=0.0, lambda_p=0.0, fv_terms=oracle_mod.FV_FLUX)
    vel = sign * np.array([0.11, 0.07, 0.05])
    u = np.broadcast_to(vel[:, None, None, None], (3, n, n, n)).copy()
    tau = np.zeros((6, n, n, n))
    tau[:, 8, 8, 8] = np.arange(1.0, 7.0)
    k = 5
    for _ in range(k):
        o.write_tau(tau)
        tau = o.fv_update(u)
    expect = np.zeros((n, n, n))
    a = np.abs(vel)
    stay = 1.0 - a.sum()
    s = int(sign)
    for mx in range(k + 1):
        for my in range(k + 1 - mx):
            for mz in range(k + 1 - mx - my):
                m0 = k - mx - my - mz
                coef = math.factorial(k) / (math.factorial(mx) * math.factorial(my) * math.factorial(mz) * math.factorial(m0))
                expect[8 + s * mz, 8 + s * my, 8 + s * mx] += coef * a[0] ** mx * a[1] ** my * a[2] ** mz * stay ** m0
    for c in range(6):
        assert np.allclose(tau[c], (c + 1.0) * expect, atol=1e-15)


def _box_overlap(d, vel):
    """Volume of the unit cell displaced by vel (lattice units, one step) that lies in
    the cell at integer offset d: the product of the 1-D interval overlaps."""
    vol = 1.0
    for a in range(3):
        vol *= max(0.0, min(1.0 + vel[a], d[a] + 1.0) - max(vel[a], float(d[a])))
    return vol


@pytest.mark.parametrize("vel", [(0.11, 0.07, 0.05), (-0.09, 0.13, -0.06), (0.12, -0.04, 0.0)])
def test_ctu_advection_moves_face_overlap_volumes(oracle_mod, vel):
    """Corner-transport-upwind variant (Sec. "Stability improvements"): a point stress
    under a uniform velocity hands each face neighbour the volume by which the displaced
    cell overlaps it, computed here from the geometry of the displaced cube; the edge and
    corner overlaps stay behind.  After k steps the result is the multinomial of those
    per-step fractions."""
    n = 16
    o = oracle_mod.Oracle((n, n, n), beta=0.0, lambda_p=0.0, fv_terms=oracle_mod.FV_FLUX | oracle_mod.FV_CTU)
    vel = np.array(vel)
    u = np.broadcast_to(vel[:, None, None, None], (3, n, n, n)).copy()
    tau = np.zeros((6, n, n, n))
    tau[:, 8, 8, 8] = np.arange(1.0, 7.0)
    k = 4
    for _ in range(k):
        o.write_tau(tau)
        tau = o.fv_update(u)
    moves = []  # (offset, fraction) per face neighbour with a nonzero overlap
    for axis in range(3):
        for sg in (1, -1):
            d = [0, 0, 0]
            d[axis] = sg
            frac = _box_overlap(d, vel)
            if frac > 0.0:
                moves.append((np.array(d), frac))
    assert all(abs(f - abs(vel[np.flatnonzero(d)[0]]) * np.prod([1 - abs(vel[a]) for a in range(3) if d[a] == 0])) < 1e-15
               for d, f in moves)
    stay = 1.0 - sum(f for _, f in moves)
    expect = np.zeros((n, n, n))
    m = len(moves)
    for counts in np.ndindex(*([k + 1] * m)):
        if sum(counts) > k:
            continue
        c0 = k - sum(counts)
        coef = math.factorial(k) / math.prod(math.factorial(c) for c in (*counts, c0))
        p = stay**c0 * math.prod(f**c for (_, f), c in zip(moves, counts))
        pos = np.array([8, 8, 8]) + sum((c * d for (d, _), c in zip(moves, counts)), np.zeros(3, int))
        expect[pos[2], pos[1], pos[0]] += coef * p
    for c in range(6):
        assert np.abs(tau[c] - (c + 1.0) * expect).max() <= 1e-14 * (c + 1.0)


def test_ctu_reduces_to_donor_cell_without_transverse_velocity(oracle_mod):
    """With the velocity along one axis only the transverse overlap factors are 1, so the
    corner-transport-upwind update equals the donor-cell one bit for bit."""
    n = 10
    u = np.zeros((3, n, n, n))
    u[1] = 0.08 * RNG.standard_normal((n, n, n))
    tau = RNG.standard_normal((6, n, n, n))
    out = []
    for terms in (oracle_mod.FV_FLUX | oracle_mod.FV_SOURCE,
                  oracle_mod.FV_FLUX | oracle_mod.FV_SOURCE | oracle_mod.FV_CTU):
        o = oracle_mod.Oracle((n, n, n), beta=0.4, lambda_p=30.0, fv_terms=terms)
        o.write_tau(tau)
        out.append(o.fv_update(u))
    assert np.array_equal(out[0], out[1])
    o.write_tau(tau)
    u[0] = 0.05 * RNG.standard_normal((n, n, n))
    assert not np.array_equal(o.fv_update(u), out[1])


def test_divu_source_adds_stress_times_trace(oracle_mod):
    """The tau div(u) term of Eq. (source): on a linear velocity field u_j = A_jk r_k the
    central difference is exact, so switching the term on adds tau_ij tr(A) in the
    interior, and alone (no flux, no other source) it is the whole update."""
    n = 12
    Amat = 1e-3 * RNG.standard_normal((3, 3))
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.stack([x, y, z]).astype(float)
    u = np.einsum("jk,k...->j...", Amat, r)
    tau = RNG.standard_normal((6, n, n, n))
    inner = (slice(None), slice(1, n - 1), slice(1, n - 1), slice(1, n - 1))
    res = {}
    for terms in (oracle_mod.FV_SOURCE, oracle_mod.FV_SOURCE | oracle_mod.FV_DIVU, oracle_mod.FV_DIVU):
        o = oracle_mod.Oracle((n, n, n), eta=0.3, beta=0.5, lambda_p=40.0, fv_terms=terms)
        o.write_tau(tau)
        res[terms] = o.fv_update(u)
    tr = np.trace(Amat)
    d = res[oracle_mod.FV_SOURCE | oracle_mod.FV_DIVU] - res[oracle_mod.FV_SOURCE]
    assert np.allclose(d[inner], (tau * tr)[inner], rtol=1e-9, atol=1e-17)
    assert np.allclose(res[oracle_mod.FV_DIVU][inner], (tau * (1.0 + tr))[inner], rtol=1e-12, atol=0)


def _giesekus_steady_shear(eta_p, lam, alpha, gdot):
    """Steady simple shear u = (gdot y, 0, 0) of the Giesekus law
    tau + lam tau_(1) + (alpha lam / eta_p) tau.tau = eta_p (L + L^T), tau_(1) the upper
    convected derivative, L_ij = d u_i / d x_j: its xx, yy and xy components (zz, xz and
    yz vanish), solved by Newton's method from the Oldroyd-B state."""
    from scipy.optimize import fsolve

    a = alpha * lam / eta_p

    def eqs(t):
        txx, tyy, txy = t
        return [txx - 2 * lam * gdot * txy + a * (txx * txx + txy * txy),
                tyy + a * (txy * txy + tyy * tyy),
                txy - lam * gdot * tyy + a * txy * (txx + tyy) - eta_p * gdot]

    t0 = [2 * eta_p * lam * gdot * gdot, 0.0, eta_p * gdot]
    sol = fsolve(eqs, t0, xtol=1e-13)
    assert np.abs(eqs(sol)).max() <= 1e-15 * max(1.0, eta_p * gdot) * 10
    return sol


@pytest.mark.parametrize("alpha", [0.0, 0.2, 0.5])
def test_giesekus_steady_shear(oracle_mod, alpha):
    """Giesekus variant of the source (constitutive laws of Sec. "Oldroyd-B fluids"):
    iterating the stress update on a simple shear field (central difference exact, no
    flux) converges to the root of the steady constitutive equations written out above;
    alpha > 0 shear-thins (tau_xy < eta_p gdot) and gives a negative second normal
    stress difference, alpha = 0 is the Oldroyd-B state."""
    n = 8
    eta, beta, lam, gdot = 0.4, 0.5, 12.0, 0.1  # Wi = 1.2
    eta_p = beta * eta
    o = oracle_mod.Oracle((n, n, n), eta=eta, beta=beta, lambda_p=lam, fv_terms=oracle_mod.FV_SOURCE,
                          giesekus_alpha=alpha)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    u = np.zeros((3, n, n, n))
    u[0] = gdot * y
    tau = np.zeros((6, n, n, n))
    for _ in range(1200):
        o.write_tau(tau)
        tau = o.fv_update(u)
    inner = (slice(1, n - 1),) * 3
    txx, tyy, txy = _giesekus_steady_shear(eta_p, lam, alpha, gdot)
    expect = {0: txx, 1: tyy, 2: 0.0, 3: txy, 4: 0.0, 5: 0.0}
    for c, v in expect.items():
        assert np.allclose(tau[c][inner], v, rtol=1e-10, atol=1e-14), (c, tau[c][inner].ravel()[:3], v)
    if alpha == 0.0:
        assert np.isclose(txy, eta_p * gdot, rtol=1e-12) and np.isclose(txx, 2 * eta_p * lam * gdot**2, rtol=1e-12)
    else:
        assert txy < eta_p * gdot and tyy < 0.0


@pytest.mark.parametrize("ctu", [False, True])
def test_flux_conserves_stress_with_walls(oracle_mod, ctu):
    """With the source off, the FV update conserves sum tau over fluid cells exactly,
    also with obstacles (zero flux across solid links) and a non-uniform velocity, with
    and without the transverse overlap factors."""
    n = 12
    terms = oracle_mod.FV_FLUX | (oracle_mod.FV_CTU if ctu else 0)
    o = oracle_mod.Oracle((n, n, n), beta=0.0, lambda_p=0.0, fv_terms=terms)
    fl = (RNG.random((n, n, n)) < 0.15).astype(np.uint8)
    o.set_flags(fl)
    u = 0.05 * RNG.standard_normal((3, n, n, n))
    tau = RNG.standard_normal((6, n, n, n)) * (fl == 0)
    o.write_tau(tau)
    tn = o.fv_update(u)
    assert np.allclose(tn.sum(axis=(1, 2, 3)), tau.sum(axis=(1, 2, 3)), rtol=0, atol=1e-12)
    assert np.abs(tn[:, fl != 0]).max() == 0.0


def test_velocity_gradient_term_on_linear_flow(oracle_mod):
    """On a linear velocity field with zero stress one FV step gives
    tau' = (eta_p/lam)(d_i u_j + d_j u_i) dt, the central difference being exact."""
    n = 12
    lam, eta, beta = 50.0, 0.4, 0.5
    o = oracle_mod.Oracle((n, n, n), eta=eta, beta=beta, lambda_p=lam, fv_terms=oracle_mod.FV_SOURCE)
    Amat = 1e-4 * RNG.standard_normal((3, 3))  # u_j = sum_k A[j,k] r_k
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.stack([x, y, z]).astype(float)
    u = np.einsum("jk,k...->j...", Amat, r)
    o.write_tau(np.zeros((6, n, n, n)))
    tn = o.fv_update(u)
    ep_l = beta * eta / lam
    inner = (slice(1, n - 1),) * 3
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    for c, (i, j) in enumerate(pairs):
        expect = ep_l * (Amat[j, i] + Amat[i, j])
        assert np.allclose(tn[c][inner], expect, rtol=1e-12, atol=1e-20)


# ----------------------------------------------------------------------------------
# full steps: balance laws
# ----------------------------------------------------------------------------------
def _mom(f, c, mask=None):
    """Total momentum sum_r sum_i f_i c_i, optionally over a mask of cells."""
    j = np.tensordot(c.T.astype(float), f, axes=(1, 0))
    return j[:, mask].sum(axis=1) if mask is not None else j.reshape(3, -1).sum(axis=1)


def _random_state(o, n_shape, umax=1e-3, taumax=1e-5):
    nx, ny, nz = n_shape
    u = RNG.uniform(-umax, umax, (3, nz, ny, nx))
    rho = 1.0 + 1e-3 * RNG.standard_normal((nz, ny, nx))
    tau = taumax * RNG.standard_normal((6, nz, ny, nx))
    o.init_fields(rho=rho, u=u, tau=tau)


def test_mass_conserved_with_obstacles_and_tangential_wall(oracle_mod):
    """sum f is constant (roundoff only) with obstacles, polymer stress and a wall
    moving tangentially (Eq. (ubb))."""
    shape = (10, 12, 8)
    o = oracle_mod.Oracle(shape, periodic=(1, 0, 1), beta=0.5, lambda_p=200.0, g=(1e-5, 0, 2e-6),
                          wall_vel=[(1e-3, 0.0, -5e-4)])
    fl = (RNG.random((8, 12, 10)) < 0.05).astype(np.uint8)
    fl[:, 0, :] = 1
    fl[:, -1, :] = 2
    o.set_flags(fl)
    _random_state(o, shape)
    m0 = o.read_pdfs()[:, fl == 0].sum()
    o.step(200)
    m1 = o.read_pdfs()[:, fl == 0].sum()
    assert abs(m1 - m0) / m0 < 1e-13


def test_momentum_gain_equals_body_force_periodic(oracle_mod):
    """Fully periodic box: every step the total momentum grows by exactly N g (the
    collision adds F per cell and sum F^p vanishes)."""
    shape = (7, 6, 5)
    g = np.array([3e-6, -1e-6, 2e-6])
    o = oracle_mod.Oracle(shape, beta=0.7, lambda_p=50.0, g=g)
    _random_state(o, shape, taumax=1e-4)
    c, _, _ = oracle_mod.lattice()
    for _ in range(5):
        j0 = _mom(o.read_pdfs(), c)
        o.step(1)
        j1 = _mom(o.read_pdfs(), c)
        assert np.allclose(j1 - j0, np.prod(shape) * g, rtol=1e-9, atol=1e-16)


def test_momentum_exchange_balances_fluid_momentum(oracle_mod):
    """Newtonian fluid, closed box with a fixed obstacle class and a moving wall class:
    each step, fluid momentum change = N_fluid g - (momentum-exchange forces on the
    tracked bodies) - (no-slip wall share, none here).  Pins sign and size of the
    momentum-exchange formula (Sec. "Moving boundaries")."""
    shape = (12, 10, 9)
    g = np.array([2e-5, 1e-5, -1e-5])
    o = oracle_mod.Oracle(shape, periodic=(1, 0, 0), beta=0.0, lambda_p=0.0, g=g,
                          wall_vel=[(0, 0, 0), (2e-3, 0, 1e-3), (0, 0, 0)])
    fl = np.full((9, 10, 12), 0, np.uint8)
    fl[:, 0, :] = 3   # moving wall class 1 (tangential velocity)
    fl[:, -1, :] = 4  # fixed class 2
    fl[0, :, :] = 4
    fl[-1, :, :] = 4
    fl[3:6, 4:7, 5:8] = 2  # obstacle class 0
    o.set_flags(fl)
    _random_state(o, shape, taumax=0.0)
    c, _, _ = oracle_mod.lattice()
    nf = int((fl == 0).sum())
    for _ in range(4):
        j0 = _mom(o.read_pdfs(), c, fl == 0)
        o.step(1)
        j1 = _mom(o.read_pdfs(), c, fl == 0)
        bf = o.body_forces()
        assert np.allclose(j1 - j0, nf * g - bf[2] - bf[3] - bf[4], rtol=1e-10, atol=1e-16)
        assert np.abs(bf[2]).max() > 0 and np.abs(bf[3]).max() > 0


def test_newtonian_poiseuille_is_exact(oracle_mod):
    """TRT with the magic value 3/16 and halfway bounce-back reproduces the Newtonian
    Poiseuille parabola exactly (to roundoff after convergence); three orientations."""
    eta, g = 1.0 / 6.0, 1e-6
    for flow, wall in [(0, 1), (2, 0), (1, 2)]:
        shape = [1, 1, 1]
        shape[wall] = 24
        periodic = [1, 1, 1]
        periodic[wall] = 0
        gv = [0.0, 0.0, 0.0]
        gv[flow] = g
        o = oracle_mod.Oracle(tuple(shape), periodic=tuple(periodic), eta=eta, beta=0.0, lambda_p=0.0, g=gv)
        o.set_flags(_channel_flags(tuple(shape), wall))
        y = np.arange(24, dtype=float)
        ua = A.poiseuille_u(y, g, eta, 0.5, 22.5)
        u0 = np.zeros((3,) + tuple(reversed(shape)))
        u0[flow] = ua.reshape(tuple(reversed(shape)))
        o.init_fields(u=u0 * (_channel_flags(tuple(shape), wall) == 0))
        o.step(6000)
        _, u, _, _ = o.read_fields()
        prof = _line(u[flow], wall)[1:-1]
        assert np.abs(prof - ua[1:-1]).max() < 1e-10 * ua.max()
        for a in range(3):
            if a != flow:
                assert np.abs(u[a]).max() < 1e-10 * ua.max()


@pytest.mark.parametrize("flow,wall", [(0, 1), (2, 0), (1, 2)])
def test_oldroydb_poiseuille_steady(oracle_mod, flow, wall):
    """Steady Oldroyd-B channel flow: parabolic u with the total viscosity,
    tau_fw = eta_p gdot, N1 = tau_ff - tau_ww = 2 eta_p lam gdot^2, other components 0.
    Interior cells within 1 %, wall-adjacent cells within 5 % (Sec. "Steady shear flow")."""
    eta, beta, lam, g, W = 1.0 / 6.0, 0.5, 400.0, 1e-6, 24
    shape = [1, 1, 1]
    shape[wall] = W
    periodic = [1, 1, 1]
    periodic[wall] = 0
    gv = [0.0, 0.0, 0.0]
    gv[flow] = g
    o = oracle_mod.Oracle(tuple(shape), periodic=tuple(periodic), eta=eta, beta=beta, lambda_p=lam, g=gv)
    o.set_flags(_channel_flags(tuple(shape), wall))
    o.step(12000)
    _, u, tau, _ = o.read_fields()
    comp = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}
    y = np.arange(W, dtype=float)[1:-1]
    L0, L1 = 0.5, W - 1.5
    ua = A.poiseuille_u(y, g, eta, L0, L1)
    gd = A.poiseuille_shear_rate(y, g, eta, L0, L1)
    eta_p = beta * eta
    up = _line(u[flow], wall)[1:-1]
    t_fw = _line(tau[comp[(flow, wall)]], wall)[1:-1]
    n1 = (_line(tau[comp[(flow, flow)]], wall) - _line(tau[comp[(wall, wall)]], wall))[1:-1]
    assert np.abs(up - ua).max() < 0.01 * ua.max()
    inner = slice(1, -1)
    assert np.abs(t_fw - eta_p * gd)[inner].max() < 0.01 * np.abs(eta_p * gd).max()
    assert np.abs(t_fw - eta_p * gd).max() < 0.05 * np.abs(eta_p * gd).max()
    n1a = 2 * eta_p * lam * gd ** 2
    assert np.abs(n1 - n1a)[inner].max() < 0.01 * n1a.max()
    assert np.abs(n1 - n1a).max() < 0.05 * n1a.max()
    others = [c for c in range(6) if c not in (comp[(flow, wall)], comp[(flow, flow)])]
    assert max(np.abs(tau[c]).max() for c in others) < 1e-6 * n1a.max()


def test_startup_transient_matches_analytic(oracle_mod):
    """Config-1 flow (walls at y=0,31, g=1e-6, eta=1/6, beta=0.5, lam=3000): centre
    velocity over 20000 steps against the analytic Oldroyd-B start-up series
    (Sec. "Time-dependent Poiseuille flow"); within 1 % of the steady centre velocity."""
    eta, beta, lam, g = 1.0 / 6.0, 0.5, 3000.0, 1e-6
    o = oracle_mod.Oracle((1, 32, 1), periodic=(1, 0, 1), eta=eta, beta=beta, lambda_p=lam, g=(g, 0, 0))
    o.set_flags(_channel_flags((1, 32, 1), 1))
    ts, uc = [], []
    for _ in range(100):
        o.step(200)
        _, u, _, _ = o.read_fields()
        ts.append(o.time)
        uc.append(0.5 * (u[0, 0, 15, 0] + u[0, 0, 16, 0]))
    L = 30.0
    ua = A.startup_poiseuille(ts, [14.5, 15.5], g=g, rho=1.0, eta_n=(1 - beta) * eta, eta_p=beta * eta,
                              lam=lam, L=L).mean(axis=1)
    us = g * L * L / (8 * eta)
    assert np.abs(np.array(uc) - ua).max() < 0.01 * us
    assert max(uc) > 1.3 * us  # the elastic overshoot is there


def test_couette_first_normal_stress_difference(oracle_mod):
    """Steady Couette flow driven by a moving-wall class: N1 = 2 eta_p lam u0^2 / L^2
    within 0.2 % in the interior, 5 % at the wall cells (Sec. "Steady shear flow")."""
    eta, beta, lam, u0, W = 1.0 / 6.0, 0.6, 150.0, 1e-3, 30
    o = oracle_mod.Oracle((1, W, 1), periodic=(1, 0, 1), eta=eta, beta=beta, lambda_p=lam,
                          wall_vel=[(u0, 0.0, 0.0)])
    fl = _channel_flags((1, W, 1), 1)
    fl[:, -1, :] = 2
    o.set_flags(fl)
    o.step(16000)
    _, u, tau, _ = o.read_fields()
    L = W - 2.0
    n1 = (tau[0] - tau[1])[0, 1:-1, 0]
    n1a = 2 * beta * eta * lam * u0 ** 2 / L ** 2
    assert np.abs(n1 - n1a)[1:-1].max() < 0.002 * n1a
    assert np.abs(n1 - n1a).max() < 0.05 * n1a
    y = np.arange(1, W - 1) - 0.5
    assert np.abs(u[0, 0, 1:-1, 0] - u0 * y / L).max() < 1e-3 * u0


def test_fixed_sphere_drag_balances_body_force(oracle_mod):
    """Periodic box with a fixed sphere (Newtonian): the momentum-exchange drag equals
    the total body force N_fluid g at steady state, and the lateral force vanishes by
    symmetry."""
    n, R, g = 14, 3.2, 1e-5
    o = oracle_mod.Oracle((n, n, n), eta=1.0 / 6.0, beta=0.0, lambda_p=0.0, g=(g, 0, 0), wall_vel=[(0, 0, 0)])
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    c0 = (n - 1) / 2.0
    fl = (((x - c0) ** 2 + (y - c0) ** 2 + (z - c0) ** 2) <= R * R).astype(np.uint8) * 2
    o.set_flags(fl)
    o.step(2500)
    F = o.body_forces()[2]
    nf = int((fl == 0).sum())
    assert abs(F[0] - nf * g) < 2e-3 * nf * g
    assert abs(F[1]) < 1e-12 * nf * g and abs(F[2]) < 1e-12 * nf * g


# ----------------------------------------------------------------------------------
# moving boundaries
# ----------------------------------------------------------------------------------
def _particle_box(oracle_mod, n=16, beta=0.5, lam=100.0, g=(0, 0, 0)):
    o = oracle_mod.Oracle((n, n, n), periodic=(1, 1, 1), eta=1.0 / 6.0, beta=beta, lambda_p=lam, g=g)
    return o


def test_fill_drain_conserves_stress_and_momentum(oracle_mod):
    """Moving a particle by hand and converting cells (Sec. "Moving boundaries"):
    sum tau over fluid (+ dropped) is unchanged, fluid + particle linear and angular
    momentum are unchanged, and created cells carry the surface velocity."""
    n = 16
    o = _particle_box(oracle_mod, n)
    c, _, _ = oracle_mod.lattice()
    X0 = np.array([7.3, 7.6, 7.1])
    v, w = np.array([1e-3, -2e-3, 5e-4]), np.array([1e-4, 2e-4, -3e-4])
    pid = o.add_particle(X0, 3.7, 1.5, v=v, w=w)
    _random_state(o, (n, n, n), taumax=1e-4)
    o.step(3)
    f0 = o.read_pdfs()
    _, _, tau0, fl0 = o.read_fields()
    p0 = o.read_particle(pid)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    pos = np.stack([x, y, z]).astype(float)

    def totals(f, fl, P):
        fluid = fl == 0
        j = np.tensordot(c.T.astype(float), f, axes=(1, 0))
        J = j[:, fluid].sum(axis=1) + P["m"] * P["v"]
        Lf = np.cross(pos[:, fluid].T, j[:, fluid].T).sum(axis=0)
        L = Lf + np.cross(P["X"], P["m"] * P["v"]) + P["I"] * P["w"]
        return J, L

    X1 = X0 + np.array([1.4, -0.9, 0.6])
    # the hand move itself changes X x m v; measure the before-state about the new position
    J0, L0 = totals(f0, fl0, dict(p0, X=X1))
    o.set_particle(pid, X=X1)
    o.fill_drain()
    f1 = o.read_pdfs()
    _, _, tau1, fl1 = o.read_fields()
    p1 = o.read_particle(pid)
    d = o.diag()
    assert d["created"] > 5 and d["destroyed"] > 5
    assert np.allclose(tau1[:, fl1 == 0].sum(axis=1) + d["dropped_tau"], tau0[:, fl0 == 0].sum(axis=1), rtol=0, atol=1e-15)
    J1, L1 = totals(f1, fl1, p1)
    assert np.allclose(J1, J0, rtol=0, atol=1e-14)
    assert np.allclose(L1, L0, rtol=0, atol=1e-12)
    created = (fl0 != 0) & (fl1 == 0)
    rho_c = f1[:, created].sum(axis=0)
    u_c = np.tensordot(c.T.astype(float), f1[:, created], axes=(1, 0)) / rho_c
    d_c = pos[:, created] - p1["X"][:, None]
    ub = p0["v"][:, None] + np.cross(p0["w"], d_c.T).T
    assert np.allclose(u_c, ub, atol=1e-15)


def test_sedimenting_particle_total_momentum_balance(oracle_mod):
    """Newtonian fluid with a moving particle under an external force: every step the
    fluid + particle momentum grows by exactly N_fluid g + F_ext (momentum exchange and
    fill/drain only move momentum between the two)."""
    n = 16
    g = np.array([0.0, 0.0, -2e-6])
    Fext = np.array([0.0, 0.0, -2e-2])
    o = _particle_box(oracle_mod, n, beta=0.0, lam=0.0, g=g)
    pid = o.add_particle([7.5, 7.5, 9.2], 3.5, 1.2, v=[0, 0, -0.02], Fext=Fext)
    c, _, _ = oracle_mod.lattice()
    total_moves = 0
    for _ in range(30):
        f0 = o.read_pdfs()
        _, _, _, fl0 = o.read_fields()
        p0 = o.read_particle(pid)
        J0 = np.tensordot(c.T.astype(float), f0, axes=(1, 0))[:, fl0 == 0].sum(axis=1) + p0["m"] * p0["v"]
        o.step(1)
        f1 = o.read_pdfs()
        _, _, _, fl1 = o.read_fields()
        p1 = o.read_particle(pid)
        J1 = np.tensordot(c.T.astype(float), f1, axes=(1, 0))[:, fl1 == 0].sum(axis=1) + p1["m"] * p1["v"]
        assert np.allclose(J1 - J0, (fl0 == 0).sum() * g + Fext, rtol=1e-9, atol=1e-14)
        total_moves += int((fl0 != fl1).sum())
    assert total_moves > 0
    assert o.read_particle(pid)["v"][2] < 0


def test_particle_update_is_symplectic_euler(oracle_mod):
    """Sec. "Moving boundaries": velocities are advanced with the momentum-exchange plus
    external force first, the position with the new velocity; the fill/drain impulse is
    added to the velocity afterwards."""
    n = 16
    o = _particle_box(oracle_mod, n, beta=0.5, lam=80.0, g=(0, 0, 1e-6))
    Fext, Text = np.array([1e-3, 0.0, -3e-3]), np.array([0.0, 2e-3, 0.0])
    pid = o.add_particle([7.4, 7.5, 7.7], 3.3, 1.3, v=[0.01, 0, -0.01], w=[0, 0, 1e-3], Fext=Fext, Text=Text)
    prev = o.read_particle(pid)
    for _ in range(12):
        o.step(1)
        p = o.read_particle(pid)
        v_mid = prev["v"] + (p["F"] + Fext) / p["m"]
        assert np.allclose(p["X"], prev["X"] + v_mid, rtol=0, atol=1e-15)
        assert np.allclose(p["v"], v_mid + p["dP"] / p["m"], rtol=0, atol=1e-16)
        assert np.allclose(p["w"], prev["w"] + (p["T"] + Text + p["dL"]) / p["I"], rtol=0, atol=1e-16)
        prev = p


def test_created_cell_shares_uniform_stress_equally(oracle_mod):
    """A created cell takes 1/(N_f+1) of its N_f fluid neighbours' stress and they give it
    up in equal parts, so a uniform stress stays uniform over the created cell and a
    neighbour that no other conversion touches (Sec. "Moving boundaries")."""
    n = 16
    o = _particle_box(oracle_mod, n)
    X0 = np.array([7.5, 7.5, 7.5])
    pid = o.add_particle(X0, 4.2, 1.0)
    _, _, _, fl0 = o.read_fields()
    tau0 = np.array([3.0, 1.0, 2.0, 0.5, -0.25, 0.125])
    o.write_tau(np.broadcast_to(tau0[:, None, None, None], (6, n, n, n)) * (fl0 == 0))
    o.set_particle(pid, X=X0 + np.array([0.45, 0.0, 0.0]))
    o.fill_drain()
    _, _, tau1, fl1 = o.read_fields()
    created = (fl0 != 0) & (fl1 == 0)
    destroyed = (fl0 == 0) & (fl1 != 0)
    assert created.sum() > 0 and destroyed.sum() > 0
    touch = np.zeros((n, n, n), int)
    conv = created | destroyed
    shifts = [(0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)]
    for s in shifts:
        touch += np.roll(conv, s, axis=(0, 1, 2))
    checked = 0
    for c in zip(*np.nonzero(created)):
        for s in shifts:
            nb = tuple((np.array(c) + np.array(s)) % n)
            if fl0[nb] == 0 and fl1[nb] == 0 and touch[nb] == 1:
                assert np.allclose(tau1[(slice(None),) + nb], tau1[(slice(None),) + c], rtol=1e-14, atol=0)
                checked += 1
    assert checked > 0


def test_subbox_centre_equals_full_periodic_solve():
    """Locality that the full-size GPU parity test relies on: after T steps the centre of a
    periodic sub-box of side 2M + 1 (M = 2T + 2) cut around a cell equals that cell of the
    full periodic solve, obstacles and wrap-around included."""
    from gpu_helpers import oracle_kwargs, oracle_subbox_centre

    from oracle import oracle
    from paper_2009_12279_gb300 import workloads

    n, T = 40, 3
    M = 2 * T + 2
    side = 2 * M + 1
    cfg = workloads.config_throughput(n, obstacle_fraction=0.05)
    cfg["params"]["body_force"] = (1e-5, -2e-6, 0.0)
    flags = cfg["flags_fn"]()
    u = workloads.random_velocity((n, n, n), 1e-3, 5)
    tau = workloads.random_stress((n, n, n), 1e-5, 6)
    full = oracle.Oracle((n, n, n), **oracle_kwargs(cfg["params"]))
    full.set_flags(flags)
    full.init_fields(u=u, tau=tau)
    full.step(T)
    _, uf, tf, _ = full.read_fields()
    ff = full.read_pdfs()
    rng = np.random.default_rng(3)
    off = np.arange(-M, M + 1)
    cells = [(0, 0, 0), (n - 1, 5, 0)] + [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(6)]
    for x, y, z in cells:
        xi, yi, zi = (x + off) % n, (y + off) % n, (z + off) % n
        o = oracle.Oracle((side, side, side), **oracle_kwargs(cfg["params"]))
        o.set_flags(flags[np.ix_(zi, yi, xi)])
        o.init_fields(u=u[:, zi][:, :, yi][:, :, :, xi], tau=tau[:, zi][:, :, yi][:, :, :, xi])
        o.step(T)
        c = M + side * (M + side * M)
        r = x + n * (y + n * z)
        assert np.array_equal(o.read_pdfs().reshape(19, -1)[:, c], ff.reshape(19, -1)[:, r])
        _, uo, to, _ = o.read_fields()
        assert np.array_equal(uo.reshape(3, -1)[:, c], uf.reshape(3, -1)[:, r])
        assert np.array_equal(to.reshape(6, -1)[:, c], tf.reshape(6, -1)[:, r])
        o.close()
    # the helper the GPU test uses (zero initial stress) gives the same centre
    x, y, z = 7, 33, 20
    xi, yi, zi = (x + off) % n, (y + off) % n, (z + off) % n
    full2 = oracle.Oracle((n, n, n), **oracle_kwargs(cfg["params"]))
    full2.set_flags(flags)
    full2.init_fields(u=u)
    full2.step(T)
    got = oracle_subbox_centre(cfg["params"], flags[np.ix_(zi, yi, xi)], u[:, zi][:, :, yi][:, :, :, xi], T)
    r = x + n * (y + n * z)
    assert np.array_equal(got[:19], full2.read_pdfs().reshape(19, -1)[:, r])
    _, u2, _, _ = full2.read_fields()
    assert np.array_equal(got[20:23], u2.reshape(3, -1)[:, r])


# ---------------------------------------------------------------------------------
# FENE-P (conformation tensor with the Peterlin closure)
# ---------------------------------------------------------------------------------
def test_fene_conformation_and_stress_are_inverse(oracle_mod):
    """tau = (eta_p/lambda)(f A - I) with f = 1/(1 - tr A / L^2), and the closed-form
    inverse A = (I + lambda tau / eta_p) / f, f = 1 + (3 + lambda tr tau / eta_p) / L^2:
    round trips to rounding, f obeys its definition, and zero stress is the isotropic
    equilibrium A = I L^2 / (L^2 + 3)."""
    eta_p, lam, L2 = 0.12, 40.0, 60.0
    for _ in range(20):
        t = 1e-3 * RNG.standard_normal(6)
        A = oracle_mod.fene_conformation(t, eta_p, lam, L2)
        assert np.allclose(oracle_mod.fene_stress(A, eta_p, lam, L2), t, rtol=1e-12, atol=1e-17)
        f = 1.0 / (1.0 - A[:3].sum() / L2)
        assert np.allclose(f * A[:3] - 1.0, lam * t[:3] / eta_p, rtol=1e-12, atol=1e-15)
    A0 = oracle_mod.fene_conformation(np.zeros(6), eta_p, lam, L2)
    assert np.allclose(A0, [L2 / (L2 + 3.0)] * 3 + [0.0] * 3, rtol=1e-15, atol=0)


def _fene_steady_shear(lam, L2, gdot):
    """Steady homogeneous simple shear u_x = gdot y of the FENE-P conformation equations
    A_(1) = -(f A - I)/lambda, written out component by component (xx, yy = zz, xy; xz
    and yz vanish) and solved by Newton's method from the Oldroyd-B state."""
    from scipy.optimize import fsolve

    def eqs(a):
        axx, ayy, axy = a
        f = 1.0 / (1.0 - (axx + 2.0 * ayy) / L2)
        return [2.0 * gdot * axy - (f * axx - 1.0) / lam,
                -(f * ayy - 1.0) / lam,
                gdot * ayy - f * axy / lam]

    a0 = [1.0 + 2.0 * (lam * gdot) ** 2, 1.0, lam * gdot]
    sol = fsolve(eqs, a0, xtol=1e-13)
    assert np.abs(eqs(sol)).max() <= 1e-15
    return sol


@pytest.mark.parametrize("L2", [10.0, 50.0, 1e12])
def test_fene_steady_shear(oracle_mod, L2):
    """FENE-P in simple shear: iterating the conformation update (source only) converges
    to the root of the steady equations above; the stress read back shear-thins (tau_xy <
    eta_p gdot, N1 < 2 eta_p lambda gdot^2) for finite L^2, and L^2 -> infinity is the
    Oldroyd-B state."""
    n = 8
    eta, beta, lam, gdot = 0.4, 0.5, 12.0, 0.1  # Wi = 1.2
    eta_p = beta * eta
    o = oracle_mod.Oracle((n, n, n), eta=eta, beta=beta, lambda_p=lam, fv_terms=oracle_mod.FV_SOURCE, fene_L2=L2)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    u = np.zeros((3, n, n, n))
    u[0] = gdot * y
    A = np.zeros((6, n, n, n))
    A[:3] = L2 / (L2 + 3.0)  # zero stress
    for _ in range(1500):
        o.write_tau(A)
        A = o.fv_update(u)
    inner = (slice(1, n - 1),) * 3
    axx, ayy, axy = _fene_steady_shear(lam, L2, gdot)
    for c, v in {0: axx, 1: ayy, 2: ayy, 3: axy, 4: 0.0, 5: 0.0}.items():
        assert np.allclose(A[c][inner], v, rtol=1e-10, atol=1e-14), (c, A[c][inner].ravel()[:2], v)
    o.write_tau(A)
    _, _, tau, _ = o.read_fields()
    txy = tau[3][inner].mean()
    n1 = (tau[0] - tau[1])[inner].mean()
    if L2 > 1e6:
        assert np.isclose(txy, eta_p * gdot, rtol=1e-9) and np.isclose(n1, 2 * eta_p * lam * gdot**2, rtol=1e-9)
    else:
        assert txy < eta_p * gdot and n1 < 2 * eta_p * lam * gdot**2


def test_fene_large_extensibility_is_oldroyd_b(oracle_mod):
    """One source-only update of a random conformation field under a random velocity
    field: with L^2 = 1e15 the FENE-P update, mapped to stress by
    tau = (eta_p/lambda)(A - I), is the Oldroyd-B update of Eq. (source)."""
    n = 6
    eta, beta, lam = 0.3, 0.6, 25.0
    eta_p = beta * eta
    u = 0.02 * RNG.standard_normal((3, n, n, n))
    tau = 1e-3 * RNG.standard_normal((6, n, n, n))
    ob = oracle_mod.Oracle((n, n, n), eta=eta, beta=beta, lambda_p=lam, fv_terms=oracle_mod.FV_SOURCE)
    ob.write_tau(tau)
    t_ob = ob.fv_update(u)
    fe = oracle_mod.Oracle((n, n, n), eta=eta, beta=beta, lambda_p=lam, fv_terms=oracle_mod.FV_SOURCE, fene_L2=1e15)
    A = lam * tau / eta_p
    A[:3] += 1.0
    fe.write_tau(A)
    A1 = fe.fv_update(u)
    t_fe = eta_p / lam * A1
    t_fe[:3] -= eta_p / lam
    assert np.allclose(t_fe, t_ob, rtol=1e-9, atol=1e-12 * np.abs(t_ob).max())
