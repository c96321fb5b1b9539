"""Instability reporting (LBVE_EUNSTABLE) through the C ABI.

The stream-collide flags a fluid cell with rho <= 0, |u|^2 >= 1/3 or a NaN; lbve_step
refuses to continue once the flag has reached the host, lbve_synchronize reports it, the
state stays readable, and re-initialising the fields clears it.  A pool refuses to step
while a member is flagged; removing that member lets the others continue.  The faults are
plain data (a NaN population, a supersonic velocity) written from the host.
"""
import numpy as np
import pytest

from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _solver(precision="f32", shape=(16, 12, 10)):
    from paper_2009_12279_gb300 import Solver, workloads

    s = Solver(shape, precision=precision, periodic=(1, 0, 1), eta=1.0 / 6.0, beta=0.5, lambda_p=100.0,
               body_force=(1e-6, 0.0, 0.0))
    s.set_geometry(workloads.channel_flags(shape, 1))
    return s


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16"])
def test_nan_population_is_reported_and_cleared(precision):
    from paper_2009_12279_gb300 import LbveError, lbve

    s = _solver(precision)
    s.step(3)
    s.synchronize()
    assert not s.is_unstable()
    f = s.read_pdfs()
    f[5, 4, 6, 7] = np.nan  # one population of one fluid cell
    s.write_pdfs(f)
    s.step(1)
    with pytest.raises(LbveError) as e:
        s.synchronize()
    assert e.value.status == lbve.EUNSTABLE
    assert s.is_unstable()
    t = s.time
    with pytest.raises(LbveError) as e:
        s.step(1)
    assert e.value.status == lbve.EUNSTABLE and s.time == t  # refused without stepping
    rho, _, _, _ = s.read_fields()  # the state stays readable
    assert np.isnan(rho).any()
    s.init_fields()
    assert not s.is_unstable()
    s.step(5)
    s.synchronize()
    s.close()


def test_supersonic_velocity_is_reported():
    from paper_2009_12279_gb300 import LbveError, lbve

    s = _solver("f32")
    shape = (16, 12, 10)
    u = np.zeros((3,) + shape[::-1])
    u[0, 5, 6, 8] = 0.7  # |u|^2 = 0.49 > 1/3
    s.init_fields(u=u)
    s.step(1)
    with pytest.raises(LbveError) as e:
        s.synchronize()
    assert e.value.status == lbve.EUNSTABLE
    s.close()


def test_healthy_fast_flow_is_not_flagged():
    """|u| = 0.5 of the sound speed everywhere: no flag (the limit is the sound speed)."""
    s = _solver("f32")
    shape = (16, 12, 10)
    u = np.zeros((3,) + shape[::-1])
    u[0] = 0.5 / np.sqrt(3.0)
    s.init_fields(u=u)
    s.step(4)
    s.synchronize()
    assert not s.is_unstable()
    s.close()


def test_pool_refuses_to_step_with_a_flagged_member():
    from paper_2009_12279_gb300 import LbveError, Pool, lbve

    pool = Pool("f32", budget_bytes=10**9)
    good, bad, alone = _solver("f32"), _solver("f32"), _solver("f32")
    pool.admit(good)
    pool.admit(bad)
    pool.step(2)
    alone.step(2)
    pool.remove(bad)  # a member's fields cannot be rewritten while it is in the pool
    fb = bad.read_pdfs()
    fb[3, 5, 5, 5] = np.nan
    bad.write_pdfs(fb)
    pool.admit(bad)
    pool.step(1)
    alone.step(1)
    import torch

    torch.cuda.synchronize()
    assert bad.is_unstable() and not good.is_unstable()
    with pytest.raises(LbveError) as e:
        pool.step(1)
    assert e.value.status == lbve.EUNSTABLE
    pool.remove(bad)
    pool.step(4)
    alone.step(4)
    assert np.array_equal(good.read_pdfs(), alone.read_pdfs())  # the mix did not touch it
    for s in (good, bad, alone):
        s.close()
    pool.close()
