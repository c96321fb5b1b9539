"""FENE-P (Peterlin closure on the conformation tensor) through the C ABI against the
oracle: the polymer force takes the stress of each cell's conformation, the
finite-volume update transports the conformation with the FENE-P source, and fields are
given and read as stress.  FP64 to 1e-12 (bitwise in practice), FP32 within 1e-5, on a
ragged box with obstacles, a moving-wall class and random initial stress, and on the
config-1 channel, where finite extensibility must shear-thin the steady stress."""
import numpy as np
import pytest

from gpu_helpers import TOL_F32, TOL_F64, compare, pair, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _obstacles(L2):
    from paper_2009_12279_gb300 import workloads

    shape = (37, 20, 18)
    nx, ny, nz = shape
    fl = workloads.channel_flags(shape, 1, top_flag=workloads.WALL0 + 1)
    rng = np.random.default_rng(5)
    fl[(rng.random((nz, ny, nx)) < 0.03) & (fl == 0)] = workloads.NOSLIP
    fl[5:9, 6:10, 10:15] = workloads.WALL0
    wall = [(0.0, 0.0, 0.0), (2e-3, 0.0, -1e-3)]
    u0 = workloads.random_velocity(shape, 2e-3, 6) * (fl == 0)
    t0 = workloads.random_stress(shape, 1e-4, 7) * (fl == 0)
    prm = dict(periodic=(1, 0, 1), eta=1.0 / 6.0, beta=0.6, lambda_p=150.0, body_force=(1e-5, 0.0, 3e-6),
               fene_L2=L2)
    return shape, prm, fl, wall, u0, t0


@pytest.mark.parametrize("precision,tol", [("f64", TOL_F64), ("f32", TOL_F32)])
@pytest.mark.parametrize("L2", [20.0, 200.0])
def test_fene_obstacles_match_oracle(precision, tol, L2, capsys):
    shape, prm, fl, wall, u0, t0 = _obstacles(L2)
    g, o = pair(shape, prm, fl, wall, u=u0, tau=t0, precision=precision)
    g.step(301)
    o.step(301)
    e = compare(g, o)
    with capsys.disabled():
        print(f"\n[FENE-P L^2 {L2} {precision}, 301 steps] {e}")
    assert max(e["u"], e["tau"]) <= tol, e
    if precision == "f64":
        assert e["f"] <= TOL_F64
    bg, bo = g.body_forces(), o.body_forces()
    assert np.linalg.norm(bg[2] - bo[2]) <= max(tol, 1e-12) * 10 * np.linalg.norm(bo[2])


def test_fene_channel_shear_thins(capsys):
    """Config-1 channel with L^2 = 10 against Oldroyd-B after 6000 steps (FP64, both
    against the oracle): finite extensibility lowers the first normal stress difference."""
    from paper_2009_12279_gb300 import workloads

    cfg = workloads.config_channel()
    res = {}
    for L2 in (0.0, 10.0):
        prm = dict(cfg["params"], fene_L2=L2)
        g, o = pair(cfg["shape"], prm, cfg["flags"], precision="f64")
        g.step(6000)
        o.step(6000)
        e = compare(g, o)
        assert max(e["f"], e["u"], e["tau"]) <= TOL_F64, e
        _, _, tau, _ = g.read_fields()
        res[L2] = (tau[0] - tau[1]).max()
    with capsys.disabled():
        print(f"\n[FENE-P channel, 6000 steps] max N1 Oldroyd-B {res[0.0]:.4e}, FENE-P L^2 = 10 {res[10.0]:.4e}")
    assert 0.0 < res[10.0] < res[0.0]


def test_fene_combinations_are_rejected():
    from paper_2009_12279_gb300 import LbveError, Pool, Solver, lbve

    with pytest.raises(LbveError, match="Giesekus"):
        Solver((8, 8, 8), precision="f32", fene_L2=10.0, giesekus_alpha=0.2)
    with pytest.raises(LbveError, match="split schedule"):
        Solver((8, 8, 8), precision="f32", fene_L2=10.0, schedule=lbve.SCHED_FUSED)
    s = Solver((16, 16, 16), precision="f32", fene_L2=10.0)
    with pytest.raises(LbveError, match="FENE-P"):
        s.add_particle((8, 8, 8), 3.0, 1.2)
    pool = Pool("f32", budget_bytes=10**9)
    with pytest.raises(LbveError, match="FENE-P"):
        pool.admit(s)
    s.close()
    pool.close()
