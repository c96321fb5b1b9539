"""Moving-boundary parity of the CUDA path with the FP64 oracle (Sec. "Moving boundaries"):
momentum exchange on particle links, symplectic particle update, re-voxelisation and
fill/drain with stress redistribution, in FP64 (relative L2 <= 1e-12) and FP32."""
import numpy as np
import pytest

from gpu_helpers import TOL_F32, TOL_F64, compare, pair, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _moving_sphere_case(n=16):
    from paper_2009_12279_gb300 import workloads

    shape = (n, n, n)
    prm = dict(periodic=(1, 1, 1), eta=1.0 / 6.0, beta=0.5, lambda_p=100.0, body_force=(0.0, 0.0, 1e-6))
    u0 = workloads.random_velocity(shape, 1e-3, 21)
    t0 = workloads.random_stress(shape, 1e-5, 22)
    part = dict(X=(7.4, 7.6, 7.3), R=3.6, rho_p=1.3, v=(0.02, -0.012, 0.008), w=(1e-3, -2e-3, 5e-4),
                Fext=(1e-3, 0.0, -2e-3), Text=(0.0, 1e-3, 0.0))
    return shape, prm, u0, t0, part


def _add(obj, part):
    return obj.add_particle(part["X"], part["R"], part["rho_p"], v=part["v"], w=part["w"], Fext=part["Fext"],
                            Text=part["Text"])


def _particle_err(pg, po):
    return max(rel_l2(pg[k], po[k]) for k in ("X", "v", "w"))


@pytest.mark.parametrize("precision,tol", [("f64", TOL_F64), ("f32", TOL_F32)])
def test_moving_sphere_parity(precision, tol):
    shape, prm, u0, t0, part = _moving_sphere_case()
    g, o = pair(shape, prm, precision=precision)
    _add(g, part)
    _add(o, part)
    g.init_fields(u=u0, tau=t0)
    o.init_fields(u=u0, tau=t0)
    moved = 0
    for _ in range(6):
        g.step(25)
        o.step(25)
        pg, po = g.read_particle(0), o.read_particle(0)
        assert _particle_err(pg, po) <= tol, (pg, po)
    e = compare(g, o)
    assert max(e["u"], e["tau"]) <= tol, e
    if precision == "f64":
        assert e["f"] <= tol
    cg, co = g.conversions(), o.diag()
    assert cg["created"] == co["created"] and cg["destroyed"] == co["destroyed"]
    assert co["created"] > 5 and co["destroyed"] > 5
    bg, bo = g.body_forces()[64], o.body_forces()[64]
    assert np.linalg.norm(bg - bo) <= max(tol, 1e-9) * np.linalg.norm(bo) * 10


def test_sedimenting_sphere_closed_box_curve():
    """Closed box (config-3 shape, reduced): the velocity-versus-time curve of the FP32 and
    BF16-storage runs against the FP64 oracle; FP64 GPU must match to 1e-12."""
    from paper_2009_12279_gb300 import workloads

    shape = (20, 20, 36)
    nx, ny, nz = shape
    fl = np.ones((nz, ny, nx), np.uint8)
    fl[1:-1, 1:-1, 1:-1] = 0
    R, rho_p = 4.0, 1.2
    vol = 4.0 / 3.0 * np.pi * R ** 3
    Fz = -(rho_p - 1.0) * vol * 6e-5
    prm = dict(periodic=(0, 0, 0), eta=1.0 / 6.0, beta=0.5, lambda_p=400.0)
    part = dict(X=((nx - 1) / 2, (ny - 1) / 2, nz - 3 * R), R=R, rho_p=rho_p, v=(0, 0, 0), w=(0, 0, 0),
                Fext=(0, 0, Fz), Text=(0, 0, 0))
    o = None
    curves = {}
    for prec in ("f64", "f32", "bf16"):
        g, oo = pair(shape, prm, fl, precision=prec)
        _add(g, part)
        if o is None:
            o = oo
            _add(o, part)
        vs = []
        for _ in range(12):
            g.step(25)
            vs.append(g.read_particle(0)["v"][2])
        curves[prec] = np.array(vs)
    vo = []
    for _ in range(12):
        o.step(25)
        vo.append(o.read_particle(0)["v"][2])
    vo = np.array(vo)
    assert vo[-1] < 0
    assert np.abs(curves["f64"] - vo).max() <= TOL_F64 * np.abs(vo).max()
    assert np.abs(curves["f32"] - vo).max() <= 1e-4 * np.abs(vo).max()
    err_bf16 = np.abs(curves["bf16"] - vo).max() / np.abs(vo).max()
    print(f"\n[sedimentation] max |v - v_oracle| / max|v|: f32 "
          f"{np.abs(curves['f32'] - vo).max() / np.abs(vo).max():.2e}, bf16 {err_bf16:.2e}")
    assert err_bf16 < 0.2


def test_total_momentum_balance_on_device():
    """Newtonian fluid + particle: each step the fluid + particle momentum grows by
    N_fluid g + F_ext (FP64 sums on the device)."""
    from paper_2009_12279_gb300 import Solver

    n = 16
    g = np.array([0.0, 0.0, -2e-6])
    Fext = np.array([0.0, 0.0, -2e-2])
    s = Solver((n, n, n), precision="f64", beta=0.0, lambda_p=0.0, body_force=g)
    s.add_particle([7.5, 7.5, 9.2], 3.5, 1.2, v=[0, 0, -0.02], Fext=Fext)
    for _ in range(20):
        r0, p0 = s.reduce(), s.read_particle(0)
        s.step(1)
        r1, p1 = s.reduce(), s.read_particle(0)
        J0 = r0["momentum"] + p0["m"] * p0["v"]
        J1 = r1["momentum"] + p1["m"] * p1["v"]
        assert np.allclose(J1 - J0, r0["fluid_cells"] * g + Fext, rtol=1e-9, atol=1e-13)


def test_add_particle_validation():
    from paper_2009_12279_gb300 import LbveError, Solver

    s = Solver((12, 12, 12), precision="f32")
    with pytest.raises(LbveError):
        s.add_particle([6, 6, 6], 4.0, 1.0)  # 2R + 6 > 12
    with pytest.raises(LbveError):
        s.add_particle([6, 6, 6], 2.0, -1.0)
    pid = s.add_particle([6, 6, 6], 2.5, 1.0)
    assert pid == 0
    _, _, _, fl = s.read_fields()
    assert (fl == 64).sum() > 0


def _three_spheres_case():
    """Several moving spheres in one solve: a ragged box, walls in y (bottom resting, top a
    moving lid class), periodic in x and z; the spheres differ in size, density and motion,
    one of them straddles the periodic x boundary, none come within reach of another."""
    from paper_2009_12279_gb300 import workloads

    shape = (44, 22, 19)
    fl = workloads.channel_flags(shape, 1, top_flag=workloads.WALL0)
    prm = dict(periodic=(1, 0, 1), eta=1.0 / 6.0, beta=0.4, lambda_p=80.0, body_force=(2e-6, 0.0, 0.0))
    u0 = workloads.random_velocity(shape, 1e-3, 31) * (fl == 0)
    t0 = workloads.random_stress(shape, 1e-5, 32) * (fl == 0)
    parts = [dict(X=(14.3, 10.4, 9.1), R=3.2, rho_p=1.3, v=(0.02, 0.004, -0.01), w=(1e-3, 0.0, -2e-3),
                  Fext=(1e-3, 0.0, 0.0), Text=(0.0, 0.0, 1e-3)),
             dict(X=(28.6, 11.2, 4.8), R=2.7, rho_p=2.0, v=(-0.015, -0.006, 0.012), w=(0.0, 2e-3, 0.0),
                  Fext=(0.0, -1e-3, 0.0), Text=(0.0, 0.0, 0.0)),
             dict(X=(43.2, 10.8, 13.3), R=3.0, rho_p=1.1, v=(0.025, 0.0, 0.006), w=(-1e-3, 1e-3, 1e-3),
                  Fext=(0.0, 0.0, 5e-4), Text=(1e-3, 0.0, 0.0))]
    return shape, prm, fl, u0, t0, parts


@pytest.mark.parametrize("precision,tol", [("f64", TOL_F64), ("f32", TOL_F32)])
def test_three_moving_spheres_parity(precision, tol):
    shape, prm, fl, u0, t0, parts = _three_spheres_case()
    wall = [(3e-3, 0.0, 1e-3)]
    g, o = pair(shape, prm, fl, wall, precision=precision)
    for p in parts:
        assert _add(g, p) == _add(o, p)
    flags0 = g.read_fields()[3]
    assert (flags0[:, :, 0] == 66).any() and (flags0[:, :, -1] == 66).any()  # sphere 2 wraps in x
    g.init_fields(u=u0, tau=t0)
    o.init_fields(u=u0, tau=t0)
    for _ in range(6):
        g.step(25)
        o.step(25)
        for k in range(len(parts)):
            pg, po = g.read_particle(k), o.read_particle(k)
            assert _particle_err(pg, po) <= tol, (k, pg, po)
    e = compare(g, o)
    assert max(e["u"], e["tau"]) <= tol, e
    if precision == "f64":
        assert e["f"] <= tol
    cg, co = g.conversions(), o.diag()
    assert cg["created"] == co["created"] and cg["destroyed"] == co["destroyed"]
    assert co["created"] > 15 and co["destroyed"] > 15
    bg, bo = g.body_forces(), o.body_forces()
    for k in [2] + [64 + p for p in range(len(parts))]:
        assert np.linalg.norm(bg[k] - bo[k]) <= max(tol, 1e-9) * np.linalg.norm(bo[k]) * 10, (k, bg[k], bo[k])
