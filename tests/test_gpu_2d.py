"""The two-dimensional path (include/lbve2d.h: D2Q9 lattice Boltzmann, D2Q5 stress)
through the C ABI against the 2-D oracle: FP64 to 1e-12, FP32 within 1e-5, on a ragged
box with obstacles, a non-uniform moving wall, a force field and random initial fields,
on the regularised-lid cavity (Sec. "Lid-driven cavity") and on the four-roll mill of the
45-degree rotated lattice (Sec. "Four-roll mill"), at reduced and at the paper's sizes."""
import numpy as np
import pytest

import analytic as A
from gpu_helpers import TOL_F32, TOL_F64, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _pair(shape, prm, precision, flags=None, ub=None, force=None, rho=None, u=None, tau=None):
    from oracle import oracle
    from paper_2009_12279_gb300 import Solver2D

    g = Solver2D(shape, precision=precision, **prm)
    o = oracle.Oracle2D(shape, **{k.replace("body_force", "g"): v for k, v in prm.items()})
    for s in (g, o):
        if flags is not None:
            s.set_geometry(flags, ub)
    if force is not None:
        g.set_force_field(force)
        o.set_force(force)
    if rho is not None or u is not None or tau is not None:
        g.init_fields(rho=rho, u=u, tau=tau)
        o.init_fields(rho=rho, u=u, tau=tau)
    return g, o


def _compare(g, o, flags):
    rg, ug, tg = g.read_fields()
    ro, uo, to = o.read_fields()
    fl = flags == 0 if flags is not None else np.ones(rg.shape, bool)
    return {"f": rel_l2(g.read_pdfs()[:, fl], o.read_pdfs()[:, fl]), "rho": float(np.abs(rg - ro)[fl].max()),
            "u": rel_l2(ug[:, fl], uo[:, fl]), "tau": rel_l2(tg[:, fl], to[:, fl])}


def _ragged_case():
    shape = (37, 26)
    nx, ny = shape
    rng = np.random.default_rng(41)
    fl = np.zeros((ny, nx), np.uint8)
    fl[0] = fl[-1] = 1
    fl[(rng.random((ny, nx)) < 0.04)] = 1
    ub = np.zeros((2, ny, nx))
    ub[0, -1] = 2e-3 * np.sin(np.linspace(0, np.pi, nx))  # non-uniform moving top wall
    ub[1, -1] = 1e-4
    ub[:, fl == 0] = 0.0
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    force = np.stack([1e-6 * np.cos(2 * np.pi * y / ny), 5e-7 * np.sin(2 * np.pi * x / nx)])
    u0 = rng.uniform(-2e-3, 2e-3, (2, ny, nx)) * (fl == 0)
    t0 = 1e-5 * rng.standard_normal((3, ny, nx)) * (fl == 0)
    rho0 = 1.0 + 1e-3 * rng.standard_normal((ny, nx))
    prm = dict(periodic=(1, 0), eta=1.0 / 6.0, beta=0.6, lambda_p=150.0, body_force=(3e-6, 0.0))
    return shape, prm, fl, ub, force, rho0, u0, t0


@pytest.mark.parametrize("precision,tol", [("f64", TOL_F64), ("f32", TOL_F32)])
def test_2d_ragged_box_matches_oracle(precision, tol, capsys):
    shape, prm, fl, ub, force, rho0, u0, t0 = _ragged_case()
    g, o = _pair(shape, prm, precision, fl, ub, force, rho0, u0, t0)
    for k in range(5):
        g.step(100 + k)
        o.step(100 + k)
    e = _compare(g, o, fl)
    with capsys.disabled():
        print(f"\n[2-D ragged box {precision}, {g.time} steps] {e}")
    assert g.time == o.time == 510
    assert max(e["u"], e["tau"]) <= tol, e
    if precision == "f64":
        assert e["f"] <= TOL_F64 and e["rho"] <= 1e-14


@pytest.mark.parametrize("precision,tol", [("f64", TOL_F64), ("f32", TOL_F32)])
@pytest.mark.parametrize("L,steps", [(48, 3000), (194, 200)])
def test_2d_cavity_matches_oracle(precision, tol, L, steps, capsys):
    """Regularised-lid cavity, beta 0.5, Wi 0.5 (reduced L = 48 over 3000 steps and the
    paper's L = 194 over 200)."""
    from paper_2009_12279_gb300 import workloads

    cfg = workloads.cavity2d(L=L, u0=1e-3 if L < 100 else 1e-4, beta=0.5, wi=0.5, eta_n=1.0 / 6.0 if L < 100 else 1.0)
    g, o = _pair(cfg["shape"], cfg["params"], precision, cfg["flags"], cfg["ub"])
    g.step(steps)
    o.step(steps)
    e = _compare(g, o, cfg["flags"])
    with capsys.disabled():
        print(f"\n[2-D cavity L {L} {precision}, {steps} steps] {e}")
    assert max(e["u"], e["tau"]) <= tol, e


@pytest.mark.parametrize("precision,tol", [("f64", TOL_F64), ("f32", TOL_F32)])
@pytest.mark.parametrize("N,steps", [(48, 3000), (214, 200)])
def test_2d_four_roll_mill_rotated_matches_oracle(precision, tol, N, steps, capsys):
    """Four-roll mill on the 45-degree rotated lattice, beta 1/3, Wi 0.5 (reduced N = 48
    over 3000 steps and the paper's 214 x 214 lattice, L = 214 sqrt 2, over 200)."""
    from paper_2009_12279_gb300 import workloads

    cfg = workloads.four_roll_mill2d(N=N, u0=1e-3, beta=1.0 / 3.0, eta_n=1.5 if N > 100 else 1.0 / 6.0, wi=0.5)
    g, o = _pair(cfg["shape"], cfg["params"], precision, force=cfg["force"])
    g.step(steps)
    o.step(steps)
    e = _compare(g, o, None)
    with capsys.disabled():
        print(f"\n[2-D four-roll mill N {N} rotated {precision}, {steps} steps] {e}")
    assert max(e["u"], e["tau"]) <= tol, e


def test_2d_four_roll_mill_stokes_limit_on_the_gpu(capsys):
    """The GPU path's own steady state against the closed form F / (2 k^2 eta) (Stokes
    limit, rotated lattice, FP32 storage)."""
    from paper_2009_12279_gb300 import Solver2D, workloads

    cfg = workloads.four_roll_mill2d(N=48, u0=1e-5, beta=0.0, eta_n=1.0 / 6.0)
    prm = dict(cfg["params"], beta=0.0, lambda_p=0.0)
    g = Solver2D(cfg["shape"], precision="f32", **prm)
    g.set_force_field(cfg["force"])
    g.step(6000)
    _, u, _ = g.read_fields()
    ua = A.four_roll_mill_newtonian(cfg["force"], cfg["k"], prm["eta"])
    err = np.abs(u - ua).max() / np.abs(ua).max()
    with capsys.disabled():
        print(f"\n[2-D four-roll mill, Stokes limit, FP32] max error against the closed form {err:.2e}")
    assert err < 0.01
