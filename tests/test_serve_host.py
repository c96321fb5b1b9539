"""Host-side checks of the serving scheduler (no GPU): request stream, admission against
the budget, FIFO order, rejection, cancellation and eviction of unstable solves (faults
injected on the host), and replica sharding over two gloo ranks."""
import math
import os

import numpy as np
import pytest

from paper_2009_12279_gb300 import replicas, serve


def test_request_stream_matches_the_serving_workload():
    reqs = serve.make_requests(300, seed=5, mean_interarrival=0.01)
    again = serve.make_requests(300, seed=5, mean_interarrival=0.01)
    assert [r.shape for r in reqs] == [r.shape for r in again]
    assert {r.kind for r in reqs} == set(serve.KINDS)
    arr = [r.arrival for r in reqs]
    assert all(b > a for a, b in zip(arr, arr[1:]))
    for r in reqs:
        nx, ny, nz = r.shape
        assert 16 <= ny == nz <= 64 and ny <= nx <= 256 and nx * ny * nz <= 256 * 64 * 64
        assert 0.1 <= r.params["beta"] <= 0.9
        eta_n = (1.0 - r.params["beta"]) * r.params["eta"]
        assert eta_n >= 1.0 / 60.0 - 1e-12
        if r.kind == "sedimenting":
            assert abs(eta_n - 1.0 / 6.0) < 1e-12  # the paper's sphere runs keep eta_n
        assert 10.0 <= r.params["lambda_p"] <= 1e5
        assert 0 < r.max_steps <= 50000
        fl = r.flags
        for a, per in enumerate(r.params["periodic"]):
            if not per:
                assert (np.moveaxis(fl, 2 - a, 0)[0] != 0).all() and (np.moveaxis(fl, 2 - a, 0)[-1] != 0).all()
    gaps = np.diff([0.0] + arr)
    assert abs(gaps.mean() - 0.01) < 0.003  # exponential inter-arrival with the requested mean


def test_percentiles():
    v = list(range(1, 101))
    assert serve.percentile(v, 50) == pytest.approx(50.5)
    assert serve.percentile(v, 99) == pytest.approx(99.01)
    assert math.isnan(serve.percentile([], 50))


class FakeSolver:
    def __init__(self, req):
        self.req = req
        self.closed = False

    def close(self):
        self.closed = True

    def is_unstable(self):
        return getattr(self.req, "flagged", False)


class FakePool:
    """Budget bookkeeping like lbve_pool; residual r = 1/steps (converges), NaN for
    requests marked unstable."""

    def __init__(self, budget):
        self.budget, self.used, self.members, self.steps = budget, 0, [], {}
        self.peak = 0
        self.admit_order = []

    def fits(self, prm):
        return self.used + prm <= self.budget

    def admit(self, s):
        self.used += s.req.bytes
        assert self.used <= self.budget
        self.peak = max(self.peak, self.used)
        self.members.append(s)
        self.steps[s.req.rid] = 0
        self.admit_order.append(s.req.rid)

    def remove(self, s):
        self.members.remove(s)
        self.used -= s.req.bytes

    def step(self, n):
        from paper_2009_12279_gb300 import lbve

        if any(s.is_unstable() for s in self.members):  # as lbve_pool_step: refuse, no step
            raise lbve.LbveError(lbve.EUNSTABLE, "member unstable")
        for s in self.members:
            self.steps[s.req.rid] += n

    def residuals(self):
        out = []
        for s in self.members:
            k = self.steps[s.req.rid]
            out.append((float("nan"), 1.0) if getattr(s.req, "unstable", False) else (100.0 / k ** 2, 1.0))
        return np.array(out)

    @property
    def bytes_in_use(self):
        return self.used

    def close(self):
        pass


def _fake_requests(n, bytes_each, seed=1):
    reqs = serve.make_requests(n, seed=seed, mean_interarrival=0.0, bases=(16,), elongations=(1,))
    for r, b in zip(reqs, bytes_each):
        r.bytes = b
        r.arrival = 0.0
        r.tol = 1e-6
        r.max_steps = 10**6
    return reqs


def _server(budget):
    pool = FakePool(budget)
    srv = serve.Server(pool=pool, solver_factory=lambda req, prec, stream: FakeSolver(req),
                       params_factory=lambda req, prec: req.bytes, check_every=100)
    return srv, pool


def test_admission_respects_budget_and_fifo():
    reqs = _fake_requests(12, [30, 50, 20, 40, 10, 60, 25, 35, 15, 45, 5, 55])
    srv, pool = _server(100)
    results, _ = srv.run(reqs)
    assert sorted(r.rid for r in results) == list(range(12))
    assert all(r.status == "converged" for r in results)
    assert pool.peak <= 100
    assert pool.admit_order == sorted(pool.admit_order)  # FIFO


def test_faults_injected_on_the_host():
    reqs = _fake_requests(5, [10, 10, 500, 10, 10])
    reqs[1].unstable = True        # a solve that blows up: evicted, the rest continue
    reqs[3].cancel_at = 0.0        # a cancelled request
    srv, pool = _server(100)       # request 2 can never fit: rejected, not waited for
    results, _ = srv.run(reqs)
    st = {r.rid: r.status for r in results}
    assert st == {0: "converged", 1: "unstable", 2: "rejected", 3: "cancelled", 4: "converged"}
    assert pool.used == 0


def test_instability_status_of_the_pool_evicts_the_flagged_member():
    """lbve_pool_step refuses to step while a member's instability flag is set (rho <= 0,
    |u| at the sound speed, NaN): the server evicts exactly the flagged members and the
    others continue to convergence."""
    reqs = _fake_requests(4, [10, 10, 10, 10])
    reqs[2].flagged = True
    srv, pool = _server(100)
    results, _ = srv.run(reqs)
    st = {r.rid: r.status for r in results}
    assert st == {0: "converged", 1: "converged", 2: "unstable", 3: "converged"}
    assert pool.used == 0


class FloorPool(FakePool):
    """A 16-bit pool: the residual per step levels off at `floor` (stochastic rounding);
    the polish pool's members keep falling (residual 100 / k^2 per step check)."""

    def __init__(self, budget, floor):
        super().__init__(budget)
        self.floor = floor

    def residuals(self):
        out = []
        for s in self.members:
            k = self.steps[s.req.rid]
            out.append((max(100.0 / k ** 2, self.floor * 100), 1.0))
        return np.array(out)


def test_polish_moves_floored_solves_to_the_second_pool():
    """With polish on, a 16-bit solve that reaches its storage floor (above the tolerance)
    moves to the polish pool and retires there at the tolerance; without polish it
    retires at the floor."""
    reqs = _fake_requests(3, [10, 10, 10])
    for r in reqs:
        r.tol = 1e-6
    moved = []

    def polish_factory(req, prec, stream, src):
        moved.append((req.rid, prec))
        return FakeSolver(req)

    main, polish = FloorPool(100, serve.RESIDUAL_FLOOR["bf16"]), FakePool(100)
    srv = serve.Server("bf16", pool=main, polish="f32", polish_pool=polish, polish_factory=polish_factory,
                       solver_factory=lambda req, prec, stream: FakeSolver(req),
                       params_factory=lambda req, prec: req.bytes, check_every=100)
    results, _ = srv.run(reqs)
    assert sorted(rid for rid, _ in moved) == [0, 1, 2] and all(p == "f32" for _, p in moved)
    assert all(r.status == "converged" for r in results)
    assert all(r.residual <= 1e-6 for r in results)  # retired at the tolerance, not at the floor
    assert main.used == 0 and polish.used == 0 and srv.stats["polished"] == 3
    main2 = FloorPool(100, serve.RESIDUAL_FLOOR["bf16"])
    srv2 = serve.Server("bf16", pool=main2, solver_factory=lambda req, prec, stream: FakeSolver(req),
                        params_factory=lambda req, prec: req.bytes, check_every=100)
    results2, _ = srv2.run(_fake_requests(3, [10, 10, 10]))
    assert all(r.status == "converged" and r.residual > 1e-6 for r in results2)


def test_polish_pool_residuals_follow_the_polish_pool_order():
    """Solves migrate in an order other than their arrival (here the last arrival first):
    each must still be judged by its own residual in the polish pool, so every solve
    spends the same number of steps there."""

    class StaggeredFloor(FloorPool):
        def residuals(self):
            out = []
            for s in self.members:
                k = self.steps[s.req.rid]
                c = 100.0 * (1 + 4 * (2 - s.req.rid))  # later arrivals reach the floor sooner
                out.append((max(c / k ** 2, self.floor * 100), 1.0))
            return np.array(out)

    reqs = _fake_requests(3, [10, 10, 10])
    for r in reqs:
        r.tol = 1e-6
    main, polish = StaggeredFloor(100, serve.RESIDUAL_FLOOR["bf16"]), FakePool(100)
    srv = serve.Server("bf16", pool=main, polish="f32", polish_pool=polish,
                       polish_factory=lambda req, prec, stream, src: FakeSolver(req),
                       solver_factory=lambda req, prec, stream: FakeSolver(req),
                       params_factory=lambda req, prec: req.bytes, check_every=100)
    results, _ = srv.run(reqs)
    assert all(r.status == "converged" for r in results)
    in_polish = {rid: polish.steps[rid] for rid in range(3)}
    assert len(set(in_polish.values())) == 1, in_polish
    assert polish.admit_order != sorted(polish.admit_order)  # they did migrate out of order


def test_bad_request_is_rejected_without_stopping_the_server():
    reqs = _fake_requests(3, [10, 10, 10])

    def factory(req, prec, stream):
        if req.rid == 1:
            raise ValueError("invalid parameters")
        return FakeSolver(req)

    pool = FakePool(100)
    srv = serve.Server(pool=pool, solver_factory=factory, params_factory=lambda r, p: r.bytes)
    results, _ = srv.run(reqs)
    assert {r.rid: r.status for r in results} == {0: "converged", 1: "rejected", 2: "converged"}


def test_shard_covers_every_item_once():
    items = list(range(37))
    got = sorted(i for rank in range(4) for i in replicas.shard(items, rank, 4))
    assert got == items
    with pytest.raises(ValueError):
        replicas.shard(items, 4, 4)


def _gloo_worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = replicas.shard(list(range(10)), rank, world)
    t, w = replicas.reduce_timing(dist, elapsed_s=1.0 + rank, work=float(len(mine)))
    out.put((rank, t, w))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_reduction_over_two_gloo_ranks():
    import multiprocessing as mp
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gloo_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, w in res:
        assert t == 2.0 and w == 10.0  # max of per-rank times, sum of per-rank work


def test_convergence_respects_the_storage_residual_floor():
    """Stochastically rounded 16-bit storage cannot go below its residual floor: a BF16 or
    FP16 solve converges at max(tol, floor), an FP32 solve at tol."""
    steps = {}
    for prec in ("f32", "f16", "bf16"):
        reqs = _fake_requests(1, [10])
        pool = FakePool(100)
        srv = serve.Server(prec, pool=pool, solver_factory=lambda req, p, stream: FakeSolver(req),
                           params_factory=lambda req, p: req.bytes, check_every=100)
        results, _ = srv.run(reqs)
        assert results[0].status == "converged"
        steps[prec] = results[0].steps
    # the fake residual per step is 1 / k^2 after k steps
    for prec, n in steps.items():
        tol = max(1e-6, serve.RESIDUAL_FLOOR[prec])
        assert 1.0 / n ** 2 <= tol < 1.0 / (n - 100) ** 2
    assert steps["bf16"] < steps["f16"] < steps["f32"]


# ---------------------------------------------------------------------------------
# z-slab decomposition: host logic (partition, ghost planes, neighbour exchange)
# ---------------------------------------------------------------------------------
def test_slab_partition_and_ghost_planes():
    from paper_2009_12279_gb300 import slabs

    r = slabs.split_planes(30, 4)
    assert r == [(0, 8), (8, 16), (16, 23), (23, 30)]
    assert slabs.ghost_planes(0, 8, 30, True) == [29] + list(range(0, 8)) + [8]
    assert slabs.ghost_planes(23, 30, 30, False) == [22] + list(range(23, 30)) + [None]
    assert slabs.neighbours(0, 4, True) == (3, 1) and slabs.neighbours(3, 4, False) == (2, None)
    assert slabs.neighbours(0, 1, True) == (0, 0)
    a = np.arange(5 * 2 * 3).reshape(5, 2, 3)
    loc = slabs.slab_array(a, [4, 0, 1, None], 0, fill=-1)
    assert (loc[0] == a[4]).all() and (loc[2] == a[1]).all() and (loc[3] == -1).all()
    with pytest.raises(ValueError):
        slabs.split_planes(3, 4)


def _slab_worker(rank, world, port, periodic, out):
    import torch
    import torch.distributed as dist

    from paper_2009_12279_gb300 import slabs

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = {}

    def pack(what, side, buf):  # this rank's face data: (rank, field, side) stamped
        buf.fill_(0)
        buf[0], buf[1], buf[2] = rank, what, side

    def unpack(what, side, buf):
        got[(what, side)] = tuple(int(v) for v in buf[:3])

    send = [torch.zeros(8, dtype=torch.int64) for _ in range(2)]
    recv = [torch.zeros(8, dtype=torch.int64) for _ in range(2)]
    for what in (0, 1, 2):
        slabs.exchange_with_neighbours(what, rank, world, periodic, pack, unpack, send, recv)
    out.put((rank, got))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, True), (2, False), (3, True)])
def test_halo_exchange_between_gloo_ranks(world, periodic):
    """Each rank's low side receives what the rank below packed for its high side and vice
    versa; no exchange across a closed domain's ends; two periodic ranks (both neighbours
    the same rank) keep the two directions apart."""
    import multiprocessing as mp
    import socket

    from paper_2009_12279_gb300 import slabs

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_slab_worker, args=(r, world, port, periodic, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got in res.items():
        lo, hi = slabs.neighbours(rank, world, periodic)
        for what in (0, 1, 2):
            if lo is None:
                assert (what, 0) not in got
            else:
                assert got[(what, 0)] == (lo, what, 1)  # the lower rank's high-side pack
            if hi is None:
                assert (what, 1) not in got
            else:
                assert got[(what, 1)] == (hi, what, 0)  # the upper rank's low-side pack
