"""Continuous-batching serving of many solves on one GPU.

Requests (periodic channels, fixed-sphere ducts and sedimenting spheres of different
sizes, Weissenberg numbers, viscosity ratios and forces) arrive over time.  The server
keeps every admitted solve's PDF / stress / flag state resident on the device, admits
waiting requests whenever the pool's device-memory budget allows, advances all resident
solves together with the batched persistent kernels (lbve_pool_step), checks each
solve's steady-state residual every `check_every` steps and retires it when it has
converged or reached its step cap.  Latency is arrival to retirement.

All physics runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import lbve, workloads

KINDS = ("channel", "sphere_duct", "sedimenting")

# Residual per step below which a solve in this PDF storage cannot go: stochastically
# rounded 16-bit storage leaves step-to-step noise in u (measured floors on channels and
# ducts: BF16 ~2e-5, FP16 ~2.5e-6).  A solve counts as converged at max(tol, 2 x floor).
RESIDUAL_FLOOR = {"bf16": 4e-5, "f16": 5e-6, "f32": 0.0, "f64": 0.0}


@dataclasses.dataclass
class Request:
    rid: int
    kind: str
    shape: tuple
    params: dict
    flags: np.ndarray
    wall_vel: list
    particle: dict | None
    arrival: float           # seconds after the start of the run
    max_steps: int
    tol: float = 1e-6         # steady-state residual per step
    cancel_at: float | None = None  # host-side cancellation time (fault injection)


@dataclasses.dataclass
class Result:
    rid: int
    kind: str
    cells: int
    status: str               # converged | capped | unstable | rejected | cancelled
    steps: int
    residual: float
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


# ---------------------------------------------------------------------------------
# synthetic request stream
# ---------------------------------------------------------------------------------
def make_request(rid, rng, *, bases=(16, 32, 64), elongations=(1, 2, 4), eta=1.0 / 6.0, max_steps_cap=50000,
                 kind=None):
    kind = kind or KINDS[rng.integers(len(KINDS))]
    b = int(rng.choice(bases))
    e = int(rng.choice(elongations))
    shape = (min(b * e, 256), b, b)
    nx, ny, nz = shape
    wi = rng.uniform(0.1, 2.0)
    beta = rng.uniform(0.1, 0.9)
    g = math.exp(rng.uniform(math.log(1e-7), math.log(1e-5)))
    particle = None
    wall_vel = []
    if kind == "channel":
        flags = workloads.channel_flags(shape, 1)
        L = ny - 2.0
        gdot = g * L / (2.0 * eta)
        lam = wi / gdot
        params = dict(periodic=(1, 0, 1), eta=eta, beta=beta, body_force=(g, 0.0, 0.0))
    elif kind == "sphere_duct":
        flags = np.zeros((nz, ny, nx), np.uint8)
        flags[:, 0, :] = flags[:, -1, :] = workloads.NOSLIP
        flags[0, :, :] = flags[-1, :, :] = workloads.NOSLIP
        R = b / 5.0
        c = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
        flags[workloads.sphere_mask(shape, c, R)] = workloads.WALL0
        wall_vel = [(0.0, 0.0, 0.0)]
        u_ref = workloads.duct_centreline_factor() * g * (ny - 2.0) ** 2 / eta
        lam = wi * R / u_ref
        params = dict(periodic=(1, 0, 0), eta=eta, beta=beta, body_force=(g, 0.0, 0.0))
    else:
        # as in the paper's sedimenting-sphere runs, the Newtonian viscosity stays eta_n and
        # the polymer adds eta_p = beta / (1 - beta) eta_n: the explicit particle coupling of
        # a light sphere (rho_p = 1.2) is unstable once eta_n drops to ~1/30
        flags = np.ones((nz, ny, nx), np.uint8)
        flags[1:-1, 1:-1, 1:-1] = 0
        R = max(2.5, b / 8.0)
        rho_p = 1.2
        eta_tot = eta / (1.0 - beta)
        F = (rho_p - 1.0) * (4.0 / 3.0) * math.pi * R ** 3 * g  # net weight under gravity g
        v_st = F / (6.0 * math.pi * eta_tot * R)
        lam = wi * R / v_st
        particle = dict(X=((nx - 1) / 2.0, (ny - 1) / 2.0, nz * 0.6), R=R, rho_p=rho_p, Fext=(0.0, 0.0, -F))
        params = dict(periodic=(0, 0, 0), eta=eta_tot, beta=beta, body_force=(0.0, 0.0, 0.0))
    lam = float(min(max(lam, 10.0), 1e5))
    params["lambda_p"] = lam
    return Request(rid=rid, kind=kind, shape=shape, params=params, flags=flags, wall_vel=wall_vel,
                   particle=particle, arrival=0.0, max_steps=int(min(10 * lam, max_steps_cap)))


def make_requests(n, seed=0, mean_interarrival=0.05, **kw):
    """n requests with Poisson arrivals (exponential inter-arrival times)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n):
        r = make_request(rid, rng, **kw)
        t += rng.exponential(mean_interarrival)
        r.arrival = t
        out.append(r)
    return out


def build_solver(req: Request, precision: str, stream: int | None = None, particle_state=None):
    """A solve of the request; particle_state (lbve_read_particle's dict) places its sphere
    at a later position and velocity (a solve moved to the polish pool)."""
    s = lbve.Solver(req.shape, precision=precision, stream=stream, **req.params)
    s.set_geometry(req.flags, req.wall_vel)
    if req.particle is not None:
        p = req.particle
        if particle_state is None:
            s.add_particle(p["X"], p["R"], p["rho_p"], Fext=p["Fext"])
        else:
            q = particle_state
            s.add_particle(q["X"], p["R"], p["rho_p"], v=q["v"], w=q["w"], Fext=p["Fext"])
    return s


def copy_solver(req: Request, precision: str, stream, src):
    """A solve of the request in another storage precision with the state of src: its
    PDFs, stress and particle position and velocities (the polish step of Server)."""
    f = src.read_pdfs()
    _, _, tau, _ = src.read_fields()
    part = src.read_particle(0) if req.particle is not None else None
    t = build_solver(req, precision, stream, particle_state=part)
    t.init_fields(tau=tau)
    t.write_pdfs(f)
    return t


def percentile(values, q):
    v = sorted(values)
    if not v:
        return float("nan")
    k = (len(v) - 1) * q / 100.0
    lo, hi = int(math.floor(k)), int(math.ceil(k))
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


def summarize(results, wall):
    done = [r for r in results if r.status in ("converged", "capped")]
    lat = [r.latency for r in done]
    cells_steps = sum(r.cells * r.steps for r in done)
    return {"solves": len(done), "rejected": sum(r.status == "rejected" for r in results),
            "unstable": sum(r.status == "unstable" for r in results),
            "cancelled": sum(r.status == "cancelled" for r in results),
            "converged": sum(r.status == "converged" for r in results),
            "solves_per_s": len(done) / wall if wall > 0 else float("nan"),
            "p50_latency_s": percentile(lat, 50), "p99_latency_s": percentile(lat, 99),
            "mlups": cells_steps / wall / 1e6 if wall > 0 else float("nan"), "wall_s": wall}


# ---------------------------------------------------------------------------------
# continuous batching
# ---------------------------------------------------------------------------------
class Server:
    """Admits, batches and retires solves against a device-memory budget.

    polish: with stochastically rounded 16-bit storage a solve cannot go below its
    storage's residual floor (RESIDUAL_FLOOR).  With polish set (an FP32 or FP64 storage
    name), a solve that reaches that floor before its tolerance moves to a second pool of
    that precision: its PDFs, stress and particle state are copied into a new solve, which
    continues until the residual reaches the tolerance.  Retirement then has the accuracy
    of the polish precision while most steps ran in 16 bits."""

    def __init__(self, precision="bf16", budget_bytes=150 * 10**9, check_every=100, stream=None, graphs=True,
                 clock=time.perf_counter, max_members=256, pool=None, solver_factory=None, params_factory=None,
                 polish=None, polish_pool=None, polish_factory=None):
        self.precision = precision
        self.check_every = int(check_every)
        self.stream = stream
        self.pool = pool if pool is not None else lbve.Pool(precision, budget_bytes, stream=stream, graphs=graphs)
        self.polish = polish
        self.polish_pool = polish_pool
        if polish is not None and polish_pool is None:
            self.polish_pool = lbve.Pool(polish, budget_bytes, stream=stream, graphs=graphs)
        self.solver_factory = solver_factory or build_solver
        self.polish_factory = polish_factory or copy_solver
        self.params_factory = params_factory or (lambda req, prec: lbve.make_params(req.shape, precision=prec,
                                                                                     **req.params))
        self.clock = clock
        self.max_members = max_members
        self.peak_bytes = 0
        # host-side time spent per phase (admission incl. context set-up, stepping incl.
        # the residual read-back, retirement incl. read-out and release, migration to the
        # polish pool)
        self.stats = {"admit_s": 0.0, "step_s": 0.0, "retire_s": 0.0, "steps": 0, "admitted": 0, "polished": 0,
                      "polish_s": 0.0}

    def _migrate(self, item):
        """Move a member that reached its storage's floor into the polish pool."""
        req, s = item[0], item[1]
        t = self.polish_factory(req, self.polish, self.stream, s)
        self.pool.remove(s)
        s.close()
        self.polish_pool.admit(t)
        item[1] = t
        item[4] = 1
        item[5] = item[3]  # steps at migration
        self.stats["polished"] += 1

    def _step_pool(self, pool, members, active, results, now):
        """Step one pool; evict members flagged unstable.  Returns the residuals or None."""
        if not members:
            return None
        try:
            pool.step(self.check_every)
        except lbve.LbveError as exc:
            if exc.status != lbve.EUNSTABLE:
                raise
            for item in [it for it in members if it[1].is_unstable()]:
                req, s, adm, steps = item[:4]
                pool.remove(s)
                s.close()
                active.remove(item)
                results.append(Result(req.rid, req.kind, int(np.prod(req.shape)), "unstable", steps, float("nan"),
                                      req.arrival, adm, now()))
            return None
        for item in members:
            item[3] += self.check_every
        return pool.residuals()

    def run(self, requests, keep_fields=False):
        """Serve the requests (sorted by arrival); returns (results, fields by rid).
        keep_fields: True (every result's fields) or a set of request ids."""
        pending = sorted(requests, key=lambda r: r.arrival)
        results, fields = [], {}
        active = []  # [req, solver, admitted_at, steps, stage (0 main, 1 polish), steps at migration]
        t0 = self.clock()
        now = lambda: self.clock() - t0  # noqa: E731
        i = 0
        while i < len(pending) or active:
            t = now()
            # cancellations (host-side)
            for item in list(active):
                req = item[0]
                if req.cancel_at is not None and t >= req.cancel_at:
                    (self.polish_pool if item[4] else self.pool).remove(item[1])
                    item[1].close()
                    active.remove(item)
                    results.append(Result(req.rid, req.kind, int(np.prod(req.shape)), "cancelled", item[3], float("nan"),
                                          req.arrival, item[2], now()))
            # admission of arrived requests while the budget allows (FIFO)
            ta = self.clock()
            while i < len(pending) and pending[i].arrival <= t and len(active) < self.max_members:
                req = pending[i]
                prm = self.params_factory(req, self.precision)
                if not self.pool.fits(prm):
                    if not active:  # can never fit: reject instead of waiting forever
                        results.append(Result(req.rid, req.kind, int(np.prod(req.shape)), "rejected", 0,
                                              float("nan"), req.arrival, t, t))
                        i += 1
                        continue
                    break
                try:
                    s = self.solver_factory(req, self.precision, self.stream)
                    self.pool.admit(s)
                except (lbve.LbveError, ValueError) as exc:
                    results.append(Result(req.rid, req.kind, int(np.prod(req.shape)), "rejected", 0, float("nan"),
                                          req.arrival, t, now()))
                    req.error = str(exc)
                    i += 1
                    continue
                active.append([req, s, now(), 0, 0, 0])
                self.stats["admitted"] += 1
                i += 1
            self.stats["admit_s"] += self.clock() - ta
            used = self.pool.bytes_in_use + (self.polish_pool.bytes_in_use if self.polish_pool is not None else 0)
            self.peak_bytes = max(self.peak_bytes, used)
            if not active:
                if i < len(pending):
                    wait = pending[i].arrival - now()
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
                continue
            ts = self.clock()
            stages = []
            for stage, pool in ((0, self.pool), (1, self.polish_pool)):
                if pool is None:
                    continue
                # residuals come in the pool's member order (admission into that pool, which
                # for the polish pool is the order of migration, not of arrival)
                by_solver = {id(it[1]): it for it in active if it[4] == stage}
                res = self._step_pool(pool, list(by_solver.values()), active, results, now)
                if res is not None:
                    members = [by_solver[id(sv)] for sv in pool.members]
                    stages.append((stage, members, res))
            self.stats["step_s"] += self.clock() - ts
            self.stats["steps"] += self.check_every
            tr = self.clock()
            floor = RESIDUAL_FLOOR.get(self.precision, 0.0)
            for stage, members, res in stages:
                for item, (r, unorm) in zip(members, res):
                    req, s, adm, steps = item[:4]
                    per_step = r / self.check_every
                    status = None
                    fresh = steps - item[5] > self.check_every  # the residual compares two checks
                    if not np.isfinite(r) or not np.isfinite(unorm):
                        status = "unstable"
                    elif stage == 0 and per_step <= max(req.tol, floor) and fresh:
                        if per_step <= req.tol or self.polish is None:
                            status = "converged"
                        elif steps < req.max_steps:
                            tp = self.clock()
                            self._migrate(item)
                            self.stats["polish_s"] += self.clock() - tp
                            continue
                    elif stage == 1 and per_step <= req.tol and fresh:
                        status = "converged"
                    if status is None and steps >= req.max_steps:
                        status = "capped"
                    if status:
                        s = item[1]
                        keep = keep_fields is True or (not isinstance(keep_fields, bool) and req.rid in keep_fields)
                        if keep and status != "unstable":
                            fields[req.rid] = s.read_fields()
                        (self.polish_pool if item[4] else self.pool).remove(s)
                        s.close()
                        active.remove(item)
                        results.append(Result(req.rid, req.kind, int(np.prod(req.shape)), status, steps,
                                              float(per_step), req.arrival, adm, now()))
            self.stats["retire_s"] += self.clock() - tr
        return results, fields

    def close(self):
        self.pool.close()
        if self.polish_pool is not None:
            self.polish_pool.close()


def run_one_at_a_time(requests, precision="f32", check_every=100, stream=None, clock=time.perf_counter,
                      keep_fields=False):
    """Baseline: each request alone, in arrival order, with lbve_step and the same stop rule."""
    pending = sorted(requests, key=lambda r: r.arrival)
    results, fields = [], {}
    t0 = clock()
    for req in pending:
        wait = req.arrival - (clock() - t0)
        if wait > 0:
            time.sleep(wait)
        adm = clock() - t0
        try:
            s = build_solver(req, precision, stream)
        except (lbve.LbveError, ValueError):
            results.append(Result(req.rid, req.kind, int(np.prod(req.shape)), "rejected", 0, float("nan"),
                                  req.arrival, adm, clock() - t0))
            continue
        steps, status, per_step = 0, None, float("nan")
        while status is None:
            try:
                s.step(check_every)
            except lbve.LbveError as exc:
                if exc.status != lbve.EUNSTABLE:
                    raise
                status = "unstable"
                break
            steps += check_every
            r, unorm = s.residual()
            per_step = r / check_every
            if not np.isfinite(r) or not np.isfinite(unorm):
                status = "unstable"
            elif per_step <= max(req.tol, RESIDUAL_FLOOR.get(precision, 0.0)) and steps > check_every:
                status = "converged"
            elif steps >= req.max_steps:
                status = "capped"
        if keep_fields and status != "unstable":
            fields[req.rid] = s.read_fields()
        s.close()
        results.append(Result(req.rid, req.kind, int(np.prod(req.shape)), status, steps, per_step, req.arrival, adm,
                              clock() - t0))
    return results, fields
