"""Finite-volume variants through the C ABI: the corner-transport-upwind transverse
overlap on the face fluxes (LBVE_FV_CTU, Sec. "Stability improvements"), the tau div(u)
source term (LBVE_FV_DIVU, Eq. (source)) and the Giesekus source term (giesekus_alpha),
against the oracle with the same settings, in the split and fused schedules and as pool
members."""
import numpy as np
import pytest

from gpu_helpers import TOL_F32, TOL_F64, compare, pair, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

FLUX, SOURCE, CTU, DIVU = 1, 2, 4, 8
VARIANTS = [FLUX | SOURCE | CTU, FLUX | SOURCE | DIVU, FLUX | SOURCE | CTU | DIVU]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _case():
    from test_gpu_parity import _obstacle_case

    return _obstacle_case((37, 20, 18), seed=23)


@pytest.mark.parametrize("schedule", [1, 2])
@pytest.mark.parametrize("terms", VARIANTS)
def test_fp64_variants_match_oracle(terms, schedule):
    shape, prm, fl, wall, rho0, u0, t0 = _case()
    g, o = pair(shape, dict(prm, fv_terms=terms), fl, wall, rho=rho0, u=u0, tau=t0, precision="f64",
                schedule=schedule)
    _, base = pair(shape, dict(prm, fv_terms=FLUX | SOURCE), fl, wall, rho=rho0, u=u0, tau=t0, precision="f64")
    for n in (1, 60, 139):
        g.step(n)
        o.step(n)
    base.step(200)
    e = compare(g, o)
    assert max(e["f"], e["u"], e["tau"]) <= TOL_F64, e
    # the variant changes the result far beyond the tolerance (the bits reach the kernels)
    _, _, to, _ = o.read_fields()
    _, _, tb, _ = base.read_fields()
    assert rel_l2(to, tb) > 1e4 * TOL_F64


@pytest.mark.parametrize("schedule", [1, 2])
def test_fp64_giesekus_matches_oracle(schedule):
    """Giesekus source term (alpha = 0.3), alone and with the CTU and div(u) variants."""
    shape, prm, fl, wall, rho0, u0, t0 = _case()
    for terms in (FLUX | SOURCE, FLUX | SOURCE | CTU | DIVU):
        p = dict(prm, fv_terms=terms, giesekus_alpha=0.3)
        g, o = pair(shape, p, fl, wall, rho=rho0, u=u0, tau=t0, precision="f64", schedule=schedule)
        _, base = pair(shape, dict(prm, fv_terms=terms), fl, wall, rho=rho0, u=u0, tau=t0, precision="f64")
        for n in (1, 60, 139):
            g.step(n)
            o.step(n)
        base.step(200)
        e = compare(g, o)
        assert max(e["f"], e["u"], e["tau"]) <= TOL_F64, (terms, e)
        _, _, to, _ = o.read_fields()
        _, _, tb, _ = base.read_fields()
        assert rel_l2(to, tb) > 1e4 * TOL_F64


def test_giesekus_alpha_is_validated():
    from paper_2009_12279_gb300 import LbveError, Solver

    shape, prm, *_ = _case()
    for bad in (-0.1, 0.6):
        with pytest.raises((LbveError, ValueError)):
            Solver(shape, precision="f32", giesekus_alpha=bad, **prm)


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_reduced_precision_variants(precision, capsys):
    shape, prm, fl, wall, rho0, u0, t0 = _case()
    terms = FLUX | SOURCE | CTU | DIVU
    g, o = pair(shape, dict(prm, fv_terms=terms, giesekus_alpha=0.3), fl, wall, rho=rho0, u=u0, tau=t0,
                precision=precision)
    g.step(300)
    o.step(300)
    e = compare(g, o)
    with capsys.disabled():
        print(f"\n[{precision} CTU + div(u) + Giesekus 0.3, 300 steps] {e}")
    tol = TOL_F32 if precision == "f32" else 5e-2
    assert max(e["u"], e["tau"]) <= tol, e


def test_pool_with_a_variant_member_equals_alone():
    """A variant member makes its stress-tile group run the variant build of the batched
    kernel; the other members of the group must still compute exactly as alone."""
    from paper_2009_12279_gb300 import lbve, serve
    from test_gpu_pool import _members

    precision = "f32"
    reqs = _members(precision)
    reqs[3].params = dict(reqs[3].params, fv_terms=FLUX | SOURCE | CTU | DIVU)
    reqs[0].params = dict(reqs[0].params, fv_terms=FLUX | SOURCE | CTU)
    reqs[1].params = dict(reqs[1].params, giesekus_alpha=0.25)
    alone = []
    for r in reqs:
        s = serve.build_solver(r, precision)
        s.step(120)
        alone.append((s.read_pdfs(), s.read_fields(), s.body_forces()))
        s.close()
    pool = lbve.Pool(precision, budget_bytes=10**10)
    solvers = [serve.build_solver(r, precision) for r in reqs]
    for s in solvers:
        pool.admit(s)
    pool.step(60)
    pool.step(60)
    for r, s, (pdf, fields, bf) in zip(reqs, solvers, alone):
        assert np.array_equal(s.read_pdfs(), pdf), f"request {r.rid} ({r.kind}) differs in the mix"
        for a, b in zip(s.read_fields(), fields):
            assert np.array_equal(a, b)
        assert np.array_equal(s.body_forces(), bf)
    pool.close()
