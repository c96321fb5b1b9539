"""Schedule autotuning (lbve_autotune, lbve_pool_autotune).  Launch shapes do not change
results, so the tuners time their candidates on the solves' own steps; these tests check
that a tuned solve is bitwise the same as an untuned one stepped as often, that FP64
still matches the oracle, and that the choices are valid."""
import numpy as np
import pytest

from gpu_helpers import TOL_F64, compare, pair, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _case():
    from test_gpu_parity import _obstacle_case

    return _obstacle_case((44, 20, 18), seed=13)


def test_autotune_is_result_neutral_fp32():
    from paper_2009_12279_gb300 import Solver

    shape, prm, fl, wall, rho0, u0, t0 = _case()
    a = Solver(shape, precision="f32", **prm)
    b = Solver(shape, precision="f32", **prm)  # created before the tuning: default schedule
    for s in (a, b):
        s.set_geometry(fl, wall)
        s.init_fields(rho=rho0, u=u0, tau=t0)
    r = a.autotune(steps=3)
    assert r["candidates"] >= 2 and r["steps_taken"] == r["candidates"] * 6
    assert r["block_x"] in (32, 64, 128) and r["fv_zchunk"] >= 1
    assert r["ms_per_step"] <= r["ms_per_step_default"] * (1 + 1e-12)
    b.step(r["steps_taken"])
    a.step(25)
    b.step(25)
    assert a.time == b.time
    assert np.array_equal(a.read_pdfs(), b.read_pdfs())
    for x, y in zip(a.read_fields(), b.read_fields()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.body_forces(), b.body_forces())
    # the choice is recorded for the shape: a second call applies it without measuring
    r2 = a.autotune(steps=3)
    assert r2["candidates"] == 0 and (r2["block_x"], r2["fv_zchunk"]) == (r["block_x"], r["fv_zchunk"])


def test_autotuned_fp64_matches_oracle():
    shape, prm, fl, wall, rho0, u0, t0 = _case()
    g, o = pair(shape, prm, fl, wall, rho=rho0, u=u0, tau=t0, precision="f64")
    r = g.autotune(steps=2)
    o.step(r["steps_taken"])
    g.step(40)
    o.step(40)
    e = compare(g, o)
    assert max(e["f"], e["u"], e["tau"]) <= TOL_F64, e


def test_autotune_rejects_pool_members_and_fused():
    from paper_2009_12279_gb300 import LbveError, Solver, lbve

    shape, prm, fl, wall, rho0, u0, t0 = _case()
    s = Solver(shape, precision="f32", schedule=lbve.SCHED_FUSED, **prm)
    with pytest.raises(LbveError, match="LBVE_ESTATE"):
        s.autotune(steps=2)
    m = Solver(shape, precision="f32", **prm)
    pool = lbve.Pool("f32", budget_bytes=10**10)
    pool.admit(m)
    with pytest.raises(LbveError, match="LBVE_ESTATE"):
        m.autotune(steps=2)
    pool.close()


@pytest.mark.parametrize("precision", ["bf16", "f32"])
def test_pool_autotune_is_result_neutral(precision):
    """Members tuned in the pool end bitwise equal to the same solves stepped alone."""
    import torch

    from paper_2009_12279_gb300 import lbve, serve
    from test_gpu_pool import _members

    reqs = _members(precision)
    stream = torch.cuda.Stream()
    pool = lbve.Pool(precision, budget_bytes=10**10, stream=stream.cuda_stream)
    solvers = [serve.build_solver(r, precision, stream.cuda_stream) for r in reqs]
    for s in solvers:
        pool.admit(s)
    pool.step(5)
    r = pool.autotune(steps=2)
    nxs = sorted({rq.shape[0] for rq in reqs})
    assert sorted(c["nx"] for c in r["classes"]) == nxs
    for c in r["classes"]:
        assert c["lb_tx"] in (16, 32, 64, 128) and c["fv_tx"] in (16, 32, 64)
    assert r["ms_per_step_after"] <= r["ms_per_step_before"] * (1 + 1e-12)
    pool.step(30)
    total = solvers[0].time
    assert all(s.time == total for s in solvers)
    for rq, s in zip(reqs, solvers):
        alone = serve.build_solver(rq, precision, stream.cuda_stream)
        alone.step(total)
        assert np.array_equal(alone.read_pdfs(), s.read_pdfs()), rq.kind
        for x, y in zip(alone.read_fields(), s.read_fields()):
            assert np.array_equal(x, y)
        assert np.array_equal(alone.body_forces(), s.body_forces())
        alone.close()
    pool.close()
