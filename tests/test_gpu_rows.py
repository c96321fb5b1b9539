"""The row-pipelined stream-collide (lbve_stream_collide_kernel == LBVE_LB_ROWS): whole
x-rows of PDFs, masks and stress moved into shared memory by bulk asynchronous copies on
mbarriers; and the two-cell stress kernel (lbve_stress_kernel == LBVE_FV_PAIRS), two
neighbouring cells per thread in the lanes of paired FP32 instructions.  FP64 must equal the oracle bitwise (relative L2 <= 1e-12 required), and every
storage mode must equal the per-cell and tiled kernels (schedule SPLIT) bitwise: the
arithmetic per cell is the same, only where the operands come from differs.  Schedule
PIPELINED takes the two kernels on these small grids (AUTO keeps them for large ones).  Cases cover the periodic
wrap of rows in x, y and z, closed sides, strips of 1 to 8 rows, moving walls, tracked
bodies, a moving sphere converting cells, odd and even step counts and the bench's row
length (512)."""
import numpy as np
import pytest

from gpu_helpers import TOL_F64, compare, pair, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _case(shape, periodic, seed, moving=True):
    """Random no-slip obstacles, walls on the closed sides (a moving wall class on the top
    of y when y is closed), a tracked obstacle class, random rho, u and tau."""
    from paper_2009_12279_gb300 import workloads

    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    fl = np.zeros((nz, ny, nx), np.uint8)
    if not periodic[1]:
        fl[:, 0, :] = workloads.NOSLIP
        fl[:, -1, :] = workloads.WALL0 + 1 if moving else workloads.NOSLIP
    if not periodic[2]:
        fl[0] = workloads.NOSLIP
        fl[-1] = workloads.NOSLIP
    fl[(rng.random((nz, ny, nx)) < 0.04) & (fl == 0)] = workloads.NOSLIP
    z0, y0, x0 = nz // 2, ny // 2, nx // 3
    fl[max(z0 - 1, 0):z0 + 1, max(y0 - 1, 0):y0 + 1, x0:x0 + 4] = workloads.WALL0
    wall = [(0.0, 0.0, 0.0), (2e-3, 0.0, -1e-3)]
    fluid = fl == 0
    u0 = workloads.random_velocity(shape, 2e-3, seed + 1) * fluid
    t0 = workloads.random_stress(shape, 1e-5, seed + 2) * fluid
    rho0 = 1.0 + 1e-3 * rng.standard_normal((nz, ny, nx))
    prm = dict(periodic=periodic, eta=1.0 / 6.0, beta=0.6, lambda_p=150.0, body_force=(1e-5, 2e-6, 3e-6))
    return fl, wall, rho0, u0, t0, prm


CASES = [
    ((64, 9, 7), (1, 1, 1)),     # strips of 8 and 1 rows, every side wraps
    ((96, 12, 10), (1, 0, 0)),   # closed y (moving lid) and z sides
    ((64, 3, 5), (1, 1, 1)),     # a single strip of 3 rows: every row wraps in y
    ((128, 5, 4), (1, 0, 1)),
]


@pytest.mark.parametrize("shape,periodic", CASES)
def test_rows_fp64_equal_oracle(shape, periodic):
    fl, wall, rho0, u0, t0, prm = _case(shape, periodic, 11)
    g, o = pair(shape, prm, fl, wall, rho=rho0, u=u0, tau=t0, precision="f64", schedule=3)
    assert g.stream_collide_kernel == "rows"
    for n in (1, 60, 40):  # odd and even AA parities, 101 steps
        g.step(n)
        o.step(n)
    e = compare(g, o)
    print(f"\n[rows f64 {shape} periodic {periodic}, 101 steps] {e}")
    assert max(e["f"], e["u"], e["tau"]) <= TOL_F64, e
    bg, bo = g.body_forces(), o.body_forces()
    assert np.linalg.norm(bg[2] - bo[2]) <= TOL_F64 * np.linalg.norm(bo[2])


def test_rows_fp64_moving_sphere_equal_oracle():
    from paper_2009_12279_gb300 import workloads

    shape = (64, 18, 18)
    prm = dict(periodic=(1, 1, 1), eta=1.0 / 6.0, beta=0.5, lambda_p=100.0, body_force=(0.0, 0.0, 1e-6))
    u0 = workloads.random_velocity(shape, 1e-3, 31)
    t0 = workloads.random_stress(shape, 1e-5, 32)
    part = dict(X=(62.4, 8.6, 8.3), R=3.6, rho_p=1.3, v=(0.02, -0.012, 0.008), w=(1e-3, -2e-3, 5e-4),
                Fext=(1e-3, 0.0, -2e-3), Text=(0.0, 1e-3, 0.0))
    g, o = pair(shape, prm, precision="f64", schedule=3)
    for obj in (g, o):
        obj.add_particle(part["X"], part["R"], part["rho_p"], v=part["v"], w=part["w"], Fext=part["Fext"],
                         Text=part["Text"])
        obj.init_fields(u=u0, tau=t0)
    assert g.stream_collide_kernel == "rows"
    g.step(151)
    o.step(151)
    e = compare(g, o)
    pg, po = g.read_particle(0), o.read_particle(0)
    print(f"\n[rows f64 moving sphere across the x wrap, 151 steps] {e}; conversions {o.diag()}")
    assert max(e["f"], e["u"], e["tau"]) <= TOL_F64, e
    for k in ("X", "v", "w"):
        assert np.allclose(pg[k], po[k], rtol=0, atol=1e-13), (k, pg[k], po[k])
    assert o.diag()["created"] > 5 and o.diag()["destroyed"] > 5


def _run(shape, prm, fl, wall, rho0, u0, t0, precision, schedule, steps, particle=None):
    from paper_2009_12279_gb300 import Solver

    s = Solver(shape, precision=precision, schedule=schedule, **prm)
    s.set_geometry(fl, wall)
    if particle is not None:
        s.add_particle(particle[0], particle[1], particle[2], v=particle[3])
    s.init_fields(rho=rho0, u=u0, tau=t0)
    for n in steps:
        s.step(n)
    out = (s.read_pdfs(), *s.read_fields()[:3], s.body_forces())
    kind = (s.stream_collide_kernel, s.stress_kernel)
    s.close()
    return out, kind


@pytest.mark.parametrize("precision", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("shape,periodic,sphere", [((64, 9, 7), (1, 1, 1), False), ((128, 12, 10), (1, 0, 0), False),
                                                   ((64, 16, 16), (1, 1, 1), True)])
def test_rows_equal_cells_bitwise(precision, shape, periodic, sphere):
    from paper_2009_12279_gb300 import lbve

    fl, wall, rho0, u0, t0, prm = _case(shape, periodic, 5)
    # a moving sphere across the periodic x boundary (moving-boundary bounces, conversions)
    part = ((shape[0] - 1.5, shape[1] / 2, shape[2] / 2), 2.6, 1.2, (0.02, 0.01, -0.01)) if sphere else None
    if part is not None:
        cx, cy, cz = part[0]
        zz, yy, xx = np.meshgrid(np.arange(shape[2]), np.arange(shape[1]), np.arange(shape[0]), indexing="ij")
        d2 = np.minimum(abs(xx - cx), shape[0] - abs(xx - cx)) ** 2 + (yy - cy) ** 2 + (zz - cz) ** 2
        fl[(d2 <= 4.0 ** 2) & (fl != 0)] = 0  # room for the sphere
    steps = (1, 16, 20)
    a, ka = _run(shape, prm, fl, wall, rho0, u0, t0, precision, lbve.SCHED_PIPELINED, steps, part)
    b, kb = _run(shape, prm, fl, wall, rho0, u0, t0, precision, lbve.SCHED_SPLIT, steps, part)
    assert ka == ("rows", "tiles" if precision == "f64" else "pairs") and kb == ("cells", "tiles")
    for name, x, y in zip(("pdfs", "rho", "u", "tau", "body forces"), a, b):
        assert np.array_equal(x, y), name


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_rows_equal_cells_bitwise_512_rows(precision):
    """The bench's row length (512 cells, the largest the row pipeline takes)."""
    from paper_2009_12279_gb300 import lbve, workloads

    shape = (512, 40, 6)
    fl = workloads.random_obstacles(shape, 0.01, 7)
    u0 = workloads.random_velocity(shape, 1e-3, 8) * (fl == 0)
    t0 = workloads.random_stress(shape, 1e-5, 9) * (fl == 0)
    prm = dict(periodic=(1, 1, 1), eta=1.0 / 6.0, beta=0.5, lambda_p=1000.0, body_force=(0.0, 0.0, 0.0))
    a, ka = _run(shape, prm, fl, [], None, u0, t0, precision, lbve.SCHED_PIPELINED, (3, 4))
    b, kb = _run(shape, prm, fl, [], None, u0, t0, precision, lbve.SCHED_SPLIT, (3, 4))
    assert ka == ("rows", "pairs") and kb == ("cells", "tiles")
    for name, x, y in zip(("pdfs", "rho", "u", "tau"), a, b):
        assert np.array_equal(x, y), name


def test_rows_not_taken_where_the_grid_does_not_allow_it():
    from paper_2009_12279_gb300 import Solver, lbve

    for shape, kw in (((37, 8, 8), {}), ((48, 8, 8), {}),
                      ((64, 8, 8), dict(schedule=lbve.SCHED_SPLIT)), ((64, 8, 8), dict(fene_L2=50.0)),
                      ((576, 2, 2), {}), ((512, 4, 4), dict(precision="f64")), ((64, 8, 8), dict(schedule=0))):
        kw.setdefault("precision", "f32")
        kw.setdefault("schedule", lbve.SCHED_PIPELINED)
        s = Solver(shape, **kw)
        assert s.stream_collide_kernel == "cells", (shape, kw)
        s.close()
    for shape, prec in (((384, 4, 4), "f64"), ((96, 4, 4), "bf16"), ((64, 4, 4), "f16"), ((512, 2, 2), "f32")):
        s = Solver(shape, precision=prec, schedule=lbve.SCHED_PIPELINED)
        assert s.stream_collide_kernel == "rows", (shape, prec)
        s.close()
    # schedule AUTO: the row pipeline from 2^22 cells, the two-cell stress update from 2^21
    for shape, kinds in (((256, 128, 128), ("rows", "pairs")), ((128, 128, 128), ("cells", "pairs")),
                         ((128, 128, 64), ("cells", "tiles"))):
        s = Solver(shape, precision="bf16")
        assert (s.stream_collide_kernel, s.stress_kernel) == kinds, shape
        s.close()


@pytest.mark.parametrize("shape,periodic", [((64, 12, 10), (1, 0, 0)), ((128, 9, 7), (1, 1, 1))])
def test_rows_fp32_match_oracle(shape, periodic):
    """FP32 through the row pipeline and the two-cell stress kernel against the FP64 oracle
    (relative L2 <= 1e-5)."""
    from gpu_helpers import TOL_F32

    fl, wall, rho0, u0, t0, prm = _case(shape, periodic, 17)
    g, o = pair(shape, prm, fl, wall, rho=rho0, u=u0, tau=t0, precision="f32", schedule=3)
    assert (g.stream_collide_kernel, g.stress_kernel) == ("rows", "pairs")
    for n in (1, 150, 150):
        g.step(n)
        o.step(n)
    e = compare(g, o)
    print(f"\n[rows f32 {shape} periodic {periodic}, 301 steps] {e}")
    assert max(e["u"], e["tau"]) <= TOL_F32, e



@pytest.mark.parametrize("precision", ["f32", "bf16"])
@pytest.mark.parametrize("shape,periodic", [((36, 21, 19), (1, 0, 1)), ((68, 9, 12), (0, 1, 1)),
                                            ((4, 6, 5), (1, 1, 1))])
def test_stress_pairs_equal_tiles_bitwise_ragged(precision, shape, periodic):
    """Ragged 64 x 8 columns (nx a multiple of 4, not of 64) and closed sides: the two-cell
    stress kernel against the tiled one (the stream-collide is the per-cell kernel here)."""
    from paper_2009_12279_gb300 import lbve

    fl, wall, rho0, u0, t0, prm = _case(shape, periodic, 23)
    if not periodic[0]:
        fl[:, :, 0] = 1
        fl[:, :, -1] = 1
    a, ka = _run(shape, prm, fl, wall, rho0, u0, t0, precision, lbve.SCHED_PIPELINED, (1, 6, 6))
    b, kb = _run(shape, prm, fl, wall, rho0, u0, t0, precision, lbve.SCHED_SPLIT, (1, 6, 6))
    assert ka == ("cells", "pairs") and kb == ("cells", "tiles")
    for name, x, y in zip(("pdfs", "rho", "u", "tau", "body forces"), a, b):
        assert np.array_equal(x, y), name


def test_stress_pairs_only_for_the_plain_update():
    from paper_2009_12279_gb300 import Solver, lbve

    for shape, kw in (((64, 8, 8), dict(fv_terms=lbve.FV_FLUX | lbve.FV_SOURCE | lbve.FV_CTU)),
                      ((64, 8, 8), dict(giesekus_alpha=0.2)), ((64, 8, 8), dict(fv_terms=lbve.FV_FLUX)),
                      ((64, 8, 8), dict(precision="f64")), ((38, 8, 8), {}),
                      ((64, 8, 8), dict(schedule=lbve.SCHED_SPLIT))):
        kw.setdefault("precision", "f32")
        kw.setdefault("schedule", lbve.SCHED_PIPELINED)
        s = Solver(shape, **kw)
        assert s.stress_kernel == "tiles", (shape, kw)
        s.close()
    s = Solver((36, 8, 8), precision="bf16", schedule=lbve.SCHED_PIPELINED)
    assert s.stress_kernel == "pairs"
    s.close()
