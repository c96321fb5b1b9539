"""Checkpoint and restore (lbve_save / lbve_restore) through the C ABI: a solve saved at a
step boundary and restored into a fresh context continues bitwise like the solve that
was never interrupted, in every storage precision, with a moving sphere that converts
cells, a moving-wall class with body forces, and an odd step count at the save (the
in-place layout of odd steps)."""
import numpy as np
import pytest

from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _case():
    from paper_2009_12279_gb300 import workloads

    shape = (18, 16, 17)
    fl = workloads.channel_flags(shape, 1, top_flag=workloads.WALL0)
    fl[2:5, 3:5, 2:4] = workloads.NOSLIP
    prm = dict(periodic=(1, 0, 1), eta=1.0 / 6.0, beta=0.5, lambda_p=120.0, body_force=(2e-6, 0.0, 1e-6))
    wall = [(1e-3, 0.0, 5e-4)]
    u0 = workloads.random_velocity(shape, 1e-3, 31) * (fl == 0)
    t0 = workloads.random_stress(shape, 1e-5, 32) * (fl == 0)
    part = dict(X=(8.3, 7.6, 8.4), R=3.4, rho_p=1.3, v=(0.02, 0.01, -0.015), w=(1e-3, -2e-3, 5e-4))
    return shape, prm, fl, wall, u0, t0, part


def _build(precision):
    from paper_2009_12279_gb300 import Solver

    shape, prm, fl, wall, u0, t0, part = _case()
    s = Solver(shape, precision=precision, **prm)
    s.set_geometry(fl, wall)
    s.add_particle(part["X"], part["R"], part["rho_p"], v=part["v"], w=part["w"])
    s.init_fields(u=u0, tau=t0)
    return s


def _state(s):
    rho, u, tau, fl = s.read_fields()
    p = s.read_particle(0)
    return {"f": s.read_pdfs(), "rho": rho, "u": u, "tau": tau, "flags": fl,
            "particle": np.concatenate([p[k] for k in ("X", "v", "w", "F", "T")]),
            "conv": np.array(list(s.conversions()["dropped_tau"]) + [s.conversions()["destroyed"],
                                                                      s.conversions()["created"]]),
            "body": s.body_forces()[[2, 64]], "t": s.time}


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16", "f16"])
def test_restore_then_step_equals_uninterrupted(precision):
    a = _build(precision)
    a.step(37)
    rec = a.save()
    at_save = _state(a)
    a.step(45)
    want = _state(a)

    b = _build(precision)
    b.step(3)  # a different state before the restore
    b.restore(rec)
    got_at_save = _state(b)
    for k in at_save:
        assert np.array_equal(np.asarray(got_at_save[k]), np.asarray(at_save[k]), equal_nan=True), ("at save", k)
    b.step(45)
    got = _state(b)
    for k in want:
        assert np.array_equal(np.asarray(got[k]), np.asarray(want[k])), (precision, k)
    assert want["conv"][-2] + want["conv"][-1] > 0  # the sphere converted cells after the save
    a.close()
    b.close()


def test_restore_rejects_another_geometry_or_particle_count():
    from paper_2009_12279_gb300 import LbveError, Solver, lbve

    shape, prm, fl, wall, u0, t0, part = _case()
    a = _build("f32")
    a.step(4)
    rec = a.save()
    other = Solver(shape, precision="f32", **prm)
    fl2 = fl.copy()
    fl2[8, 8, 8] = 1  # one more no-slip cell
    other.set_geometry(fl2, wall)
    other.add_particle(part["X"], part["R"], part["rho_p"])
    with pytest.raises(LbveError) as e:
        other.restore(rec)
    assert e.value.status == lbve.STATUS.index("LBVE_EINVAL")
    nopart = Solver(shape, precision="f32", **prm)
    nopart.set_geometry(fl, wall)
    with pytest.raises(LbveError, match="particles"):
        nopart.restore(rec)
    f64 = Solver(shape, precision="f64", **prm)
    with pytest.raises(LbveError, match="precision"):
        f64.restore(rec)
    for s in (a, other, nopart, f64):
        s.close()
