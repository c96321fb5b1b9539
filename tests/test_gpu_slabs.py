"""z-slab decomposition of one domain (lbve_set_z_range, lbve_step_phase, halo pack and
unpack) on one GPU: the decomposed run equals the undecomposed one bitwise in every
storage precision (the 16-bit rounding keys follow the domain's cells), for periodic and
closed z, uneven slabs, obstacles and a moving-wall class straddling slab faces, over
odd and even step counts; body forces of the slabs add up to the domain's."""
import numpy as np
import pytest

from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _case(periodic_z, nx=20):
    from paper_2009_12279_gb300 import workloads

    shape = (nx, 18, 30)
    nx, ny, nz = shape
    rng = np.random.default_rng(61)
    fl = np.zeros((nz, ny, nx), np.uint8)
    fl[:, 0, :] = workloads.NOSLIP
    fl[:, -1, :] = workloads.WALL0 + 1  # a moving lid
    fl[(rng.random((nz, ny, nx)) < 0.04) & (fl == 0)] = workloads.NOSLIP
    fl[6:10, 5:9, 4:9] = workloads.WALL0  # a tracked block across the faces at z = 7 / 8
    if not periodic_z:
        fl[0] = workloads.NOSLIP
        fl[-1] = workloads.NOSLIP
    wall = [(0.0, 0.0, 0.0), (2e-3, 0.0, -1e-3)]
    u0 = rng.uniform(-2e-3, 2e-3, (3, nz, ny, nx)) * (fl == 0)
    t0 = 1e-5 * rng.standard_normal((6, nz, ny, nx)) * (fl == 0)
    prm = dict(periodic=(1, 0, 1 if periodic_z else 0), eta=1.0 / 6.0, beta=0.6, lambda_p=150.0,
               body_force=(1e-5, 0.0, 3e-6))
    return shape, prm, fl, wall, u0, t0


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("periodic_z,nslabs,nx", [(True, 2, 20), (True, 4, 20), (False, 3, 20), (True, 1, 20),
                                                  (True, 2, 64), (False, 3, 64)])
def test_decomposed_run_equals_the_undecomposed_one(precision, periodic_z, nslabs, nx):
    """nx = 64 runs the row-pipelined kernels (z-ranges of the slabs included)."""
    from paper_2009_12279_gb300 import Solver
    from paper_2009_12279_gb300.slabs import SlabDomain

    shape, prm, fl, wall, u0, t0 = _case(periodic_z, nx)
    if nx == 64:
        prm["schedule"] = 3  # LBVE_SCHED_PIPELINED: the row pipeline and the two-cell stress kernel
    whole = Solver(shape, precision=precision, **prm)
    whole.set_geometry(fl, wall)
    whole.init_fields(u=u0, tau=t0)
    dom = SlabDomain(shape, nslabs, flags=fl, wall_vel=wall, precision=precision, **prm)
    dom.init_fields(u=u0, tau=t0)
    for n in (7, 6):
        whole.step(n)
        dom.step(n)
        assert dom.time == whole.time
        assert np.array_equal(dom.read_pdfs(), whole.read_pdfs()), (precision, dom.time, "pdfs")
        rw, uw, tw, fw = whole.read_fields()
        rd, ud, td, fd = dom.read_fields()
        assert np.array_equal(fd, fw)
        for name, a, b in (("rho", rd, rw), ("u", ud, uw), ("tau", td, tw)):
            assert np.array_equal(a, b), (precision, dom.time, name)
    bw, bd = whole.body_forces(), dom.body_forces()
    assert np.abs(bw[2]).max() > 0
    # the fields are bitwise equal; a body force is summed per slab and then over the slabs,
    # another order of the same FP64 link contributions (the moving lid's normal force is a
    # sum of thousands of O(1) terms), so it agrees to rounding only
    assert np.allclose(bd[[2, 3]], bw[[2, 3]], rtol=1e-10, atol=1e-16), (bd[[2, 3]] - bw[[2, 3]])
    whole.close()
    dom.close()


def test_slab_calls_are_validated():
    from paper_2009_12279_gb300 import LbveError, Solver, lbve

    s = Solver((8, 8, 10), precision="f32", periodic=(1, 1, 0))
    with pytest.raises(LbveError, match="ghost plane"):
        s.set_z_range(0, 9, 0)
    with pytest.raises(LbveError, match="not a z-slab"):
        s.halo_pack(lbve.HALO_U, 0, 1)
    s.set_z_range(1, 9, 0)
    with pytest.raises(LbveError, match="phase 1 without"):
        s.step_phase(1)
    s.step_phase(0)
    with pytest.raises(LbveError, match="awaits"):
        s.step(1)
    s.step_phase(1)
    assert s.time == 1
    p = Solver((8, 8, 10), precision="f32", periodic=(1, 1, 1))
    with pytest.raises(LbveError, match="not periodic in z"):
        p.set_z_range(1, 9, 0)
    for x in (s, p):
        x.close()
