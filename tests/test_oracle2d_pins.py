"""The two-dimensional oracle (D2Q9 lattice Boltzmann, D2Q5 finite-volume stress)
pinned against what the mathematics fixes: the lattice moments, exact Newtonian
Poiseuille flow, the steady Oldroyd-B channel and Couette profiles, the steady Stokes
four-roll mill (on the lattice and on the 45-degree rotated lattice the paper uses),
exact mass conservation and the mirror symmetry of the regularised-lid cavity in the
Stokes limit."""
import numpy as np
import pytest

import analytic as A


@pytest.fixture(scope="module")
def orc():
    from oracle import oracle

    oracle.build()
    return oracle


def _channel(ny, nx=1):
    fl = np.zeros((ny, nx), np.uint8)
    fl[0] = fl[-1] = 1
    return fl


def test_d2q9_lattice_moments(orc):
    c, w, opp = orc.lattice2d()
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(2) / 3.0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(2)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(m4, iso, atol=1e-16)
    assert (c[opp] == -c).all()


def test_newtonian_poiseuille_is_exact(orc):
    ny, g, eta = 20, 1e-6, 1.0 / 6.0
    o = orc.Oracle2D((1, ny), periodic=(1, 0), eta=eta, beta=0.0, lambda_p=0.0, g=(g, 0.0))
    o.set_geometry(_channel(ny))
    o.step(8000)
    _, u, _ = o.read_fields()
    y = np.arange(1, ny - 1, dtype=float)
    ua = A.poiseuille_u(y, g, eta, 0.5, ny - 1.5)
    assert np.abs(u[0, 1:-1, 0] - ua).max() < 1e-10 * ua.max()
    assert np.abs(u[1]).max() < 1e-14


def test_oldroydb_channel_steady(orc):
    ny, g, eta, beta, lam = 24, 1e-6, 1.0 / 6.0, 0.5, 400.0
    o = orc.Oracle2D((1, ny), periodic=(1, 0), eta=eta, beta=beta, lambda_p=lam, g=(g, 0.0))
    o.set_geometry(_channel(ny))
    o.step(12000)
    _, u, tau = o.read_fields()
    y = np.arange(1, ny - 1, dtype=float)
    L0, L1 = 0.5, ny - 1.5
    ua = A.poiseuille_u(y, g, eta, L0, L1)
    gd = A.poiseuille_shear_rate(y, g, eta, L0, L1)
    eta_p = beta * eta
    txy, n1 = tau[2, 1:-1, 0], (tau[0] - tau[1])[1:-1, 0]
    inner = slice(1, -1)
    assert np.abs(u[0, 1:-1, 0] - ua).max() < 0.01 * ua.max()
    assert np.abs(txy - eta_p * gd)[inner].max() < 0.01 * np.abs(eta_p * gd).max()
    assert np.abs(txy - eta_p * gd).max() < 0.05 * np.abs(eta_p * gd).max()
    n1a = 2 * eta_p * lam * gd ** 2
    assert np.abs(n1 - n1a)[inner].max() < 0.01 * n1a.max()
    assert np.abs(n1 - n1a).max() < 0.05 * n1a.max()
    assert np.abs(tau[1]).max() < 1e-6 * n1a.max()  # tau_yy stays zero in shear


def test_couette_first_normal_stress_difference(orc):
    """Moving top wall (prescribed velocity of the solid row): N1 = 2 eta_p lambda u0^2 / L^2
    within 0.2 % in the interior (Sec. "Steady shear flow")."""
    eta, beta, lam, u0, W = 1.0 / 6.0, 0.6, 150.0, 1e-3, 30
    o = orc.Oracle2D((1, W), periodic=(1, 0), eta=eta, beta=beta, lambda_p=lam)
    ub = np.zeros((2, W, 1))
    ub[0, -1, 0] = u0
    o.set_geometry(_channel(W), ub)
    o.step(16000)
    _, u, tau = o.read_fields()
    L = W - 2.0
    n1 = (tau[0] - tau[1])[1:-1, 0]
    n1a = 2 * beta * eta * lam * u0 ** 2 / L ** 2
    assert np.abs(n1 - n1a)[1:-1].max() < 0.002 * n1a
    assert np.abs(n1 - n1a).max() < 0.05 * n1a
    y = np.arange(1, W - 1) - 0.5
    assert np.abs(u[0, 1:-1, 0] - u0 * y / L).max() < 1e-3 * u0


@pytest.mark.parametrize("rotated", [False, True])
def test_four_roll_mill_newtonian_steady_state(orc, rotated):
    """Stokes limit (tiny u0, beta = 0) of the four-roll mill: the steady velocity is the
    closed form F / (2 k^2 eta), also on the 45-degree rotated lattice (periodic with
    L = N sqrt 2).  The residual is the lattice's O(k^2) discretisation error."""
    from paper_2009_12279_gb300 import workloads

    N = 48
    cfg = workloads.four_roll_mill2d(N=N, u0=1e-6, beta=0.0, eta_n=1.0 / 6.0, rotated=rotated)
    prm = dict(cfg["params"], beta=0.0, lambda_p=0.0)
    o = orc.Oracle2D(cfg["shape"], **{k.replace("body_force", "g"): v for k, v in prm.items()})
    o.set_force(cfg["force"])
    o.step(6000)
    _, u, _ = o.read_fields()
    ua = A.four_roll_mill_newtonian(cfg["force"], cfg["k"], prm["eta"])
    err = np.abs(u - ua).max() / np.abs(ua).max()
    assert err < 0.01, err
    # the centre of the rolls' stagnation point is extensional: u vanishes there
    assert np.abs(u).max() > 0.9 * np.abs(ua).max()


def test_cavity_mass_and_mirror_symmetry_in_the_stokes_limit(orc):
    """Lid-driven cavity (Sec. "Lid-driven cavity").  A uniformly sliding lid conserves
    the fluid mass exactly (each fluid cell's diagonal links into the lid carry opposite
    moving-wall terms).  Under the regularised profile 16 u0 xi^2 (1 - xi)^2 the flow at
    vanishing Reynolds number is mirror symmetric about x = L/2 (u_x even, u_y odd)."""
    from paper_2009_12279_gb300 import workloads

    cfg = workloads.cavity2d(L=30, u0=1e-7, beta=0.5, wi=0.3, eta_n=1.0 / 6.0)
    prm = cfg["params"]
    kw = {k.replace("body_force", "g"): v for k, v in prm.items()}
    fl = cfg["flags"] == 0
    uniform = np.zeros_like(cfg["ub"])
    uniform[0, -1, :] = 1e-3
    om = orc.Oracle2D(cfg["shape"], **kw)
    om.set_geometry(cfg["flags"], uniform)
    m0 = om.read_pdfs()[:, fl].sum()
    om.step(200)
    assert abs(om.read_pdfs()[:, fl].sum() - m0) < 1e-13 * m0
    o = orc.Oracle2D(cfg["shape"], **kw)
    o.set_geometry(cfg["flags"], cfg["ub"])
    o.step(3000)
    _, u, tau = o.read_fields()
    ux, uy = u[0][1:-1, 1:-1], u[1][1:-1, 1:-1]
    scale = np.abs(u).max()
    assert scale > 0
    assert np.abs(ux - ux[:, ::-1]).max() < 1e-6 * scale
    assert np.abs(uy + uy[:, ::-1]).max() < 1e-6 * scale
    assert ux[-1].mean() > 0  # the fluid under the lid follows it
