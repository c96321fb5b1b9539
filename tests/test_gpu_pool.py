"""Batched pools and continuous-batching serving on the GPU: every solve's result is the
same alone (lbve_step) and in the mix (lbve_pool_step), whatever else is resident and
whenever it was admitted; admission respects the device-memory budget."""
import numpy as np
import pytest

from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _members(precision):
    """Heterogeneous solves: channel, sphere duct (tracked wall class), closed box with a
    sedimenting sphere (particle), ragged periodic box with obstacles."""
    from paper_2009_12279_gb300 import serve, workloads

    rng = np.random.default_rng(7)
    reqs = [serve.make_request(0, rng, bases=(16,), elongations=(2,), kind="channel"),
            serve.make_request(1, rng, bases=(16,), elongations=(1,), kind="sphere_duct"),
            serve.make_request(2, rng, bases=(32,), elongations=(1,), kind="sedimenting")]
    shape = (37, 21, 19)
    r3 = serve.make_request(3, rng, bases=(16,), elongations=(1,), kind="channel")
    r3.shape = shape
    r3.flags = workloads.random_obstacles(shape, 0.03, 3)
    r3.params = dict(periodic=(1, 1, 1), eta=1.0 / 6.0, beta=0.4, lambda_p=300.0, body_force=(2e-5, 1e-5, 0.0))
    reqs.append(r3)
    for r in reqs:
        if r.particle is not None:
            r.particle["Fext"] = (0.0, 0.0, -5e-2)  # moves a few cells within the test
    return reqs


def _state(s):
    rho, u, tau, fl = s.read_fields()
    return s.read_pdfs(), u, tau, fl


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_pool_results_equal_alone(precision):
    from paper_2009_12279_gb300 import lbve, serve

    reqs = _members(precision)
    alone = []
    for r in reqs:
        s = serve.build_solver(r, precision)
        late = r.rid == 3
        s.step(150 if late else 200)
        alone.append((_state(s), s.read_particle(0) if r.particle else None, s.body_forces()))
        s.close()
    pool = lbve.Pool(precision, budget_bytes=10**10)
    solvers = [serve.build_solver(r, precision) for r in reqs]
    for s in solvers[:3]:
        pool.admit(s)
    pool.step(25)
    pool.step(25)
    pool.admit(solvers[3])  # admitted late: its step parity differs from the others'
    pool.step(75)
    pool.step(75)
    for r, s, (ref, pref, bref) in zip(reqs, solvers, alone):
        got = _state(s)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), f"request {r.rid} ({r.kind}) differs in the mix"
        if pref is not None:
            p = s.read_particle(0)
            for k in ("X", "v", "w"):
                assert np.array_equal(p[k], pref[k])
            assert np.array_equal(s.read_fields()[3], ref[3])
        assert np.array_equal(s.body_forces(), bref)


def test_graphs_do_not_change_results():
    """On a capturable stream the step sequence is replayed from a CUDA graph."""
    import torch

    from paper_2009_12279_gb300 import lbve, serve

    reqs = _members("f32")
    out = []
    stream = torch.cuda.Stream()
    for graphs in (True, False):
        pool = lbve.Pool("f32", budget_bytes=10**10, graphs=graphs, stream=stream.cuda_stream)
        solvers = [serve.build_solver(r, "f32", stream.cuda_stream) for r in reqs]
        for s in solvers:
            pool.admit(s)
        for _ in range(3):
            pool.step(33)  # odd step count: both call parities are captured and replayed
        out.append([_state(s) for s in solvers])
        pool.close()
    for a, b in zip(out[0], out[1]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_budget_and_membership_rules():
    from paper_2009_12279_gb300 import LbveError, lbve, serve

    reqs = _members("bf16")
    solvers = [serve.build_solver(r, "bf16") for r in reqs[:2]]
    need = [lbve.device_bytes(s.params) for s in solvers]
    pool = lbve.Pool("bf16", budget_bytes=need[0] + need[1] // 2)
    assert pool.fits(solvers[0].params)
    pool.admit(solvers[0])
    assert not pool.fits(solvers[1].params)
    with pytest.raises(LbveError, match="LBVE_ENOMEM"):
        pool.admit(solvers[1])
    assert pool.bytes_in_use == need[0] and len(pool) == 1
    with pytest.raises(LbveError, match="LBVE_ESTATE"):
        solvers[0].step(1)  # a member only advances through the pool
    f32 = serve.build_solver(reqs[0], "f32")
    with pytest.raises(LbveError, match="LBVE_ESTATE"):
        pool.admit(f32)  # precision differs
    pool.remove(solvers[0])
    assert pool.bytes_in_use == 0 and len(pool) == 0
    solvers[0].step(1)


def test_residuals_same_alone_and_in_pool():
    from paper_2009_12279_gb300 import lbve, serve

    reqs = _members("f32")
    ref = []
    for r in reqs:
        s = serve.build_solver(r, "f32")
        s.step(100)
        s.residual()
        s.step(100)
        ref.append(s.residual())
        s.close()
    pool = lbve.Pool("f32", budget_bytes=10**10)
    solvers = [serve.build_solver(r, "f32") for r in reqs]
    for s in solvers:
        pool.admit(s)
    pool.step(100)
    pool.residuals()
    pool.step(100)
    got = pool.residuals()
    for (r0, n0), (r1, n1) in zip(ref, got):
        assert r0 == r1 and n0 == n1


def test_serving_each_result_same_alone_and_in_the_mix():
    """A short continuous-batching run (requests arriving while others are resident)
    against the same requests served one at a time with the same precision."""
    from paper_2009_12279_gb300 import serve

    reqs = serve.make_requests(8, seed=11, mean_interarrival=0.02, bases=(16,), elongations=(1, 2), max_steps_cap=400)
    srv = serve.Server("bf16", budget_bytes=10**10, check_every=100)
    mix, fmix = srv.run(reqs, keep_fields=True)
    srv.close()
    solo, fsolo = serve.run_one_at_a_time(reqs, precision="bf16", keep_fields=True)
    smix = {r.rid: (r.status, r.steps, r.residual) for r in mix}
    ssolo = {r.rid: (r.status, r.steps, r.residual) for r in solo}
    assert smix == ssolo
    for rid, fields in fsolo.items():
        for a, b in zip(fields, fmix[rid]):
            assert np.array_equal(a, b)
    summary = serve.summarize(mix, max(r.finished for r in mix))
    assert summary["solves"] + summary["unstable"] == 8
    assert summary["solves"] >= 6 and summary["p99_latency_s"] >= summary["p50_latency_s"] > 0
