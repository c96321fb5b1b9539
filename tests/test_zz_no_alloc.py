"""lbve_step_noalloc: time steps on caller-owned device buffers with no device allocation.

Callers that cannot call cudaMalloc (for example code running inside a framework that
owns all device memory through its own pool) keep the solve's state in their own
buffers and advance it with this entry point, whose only intermediate lives in a fixed
device array inside the library.  This test builds such buffers with torch, advances
them with two calls in a row, and checks each result against the regular context path
(lbve_create / lbve_step) on the same input, within the FP32 parity tolerance.
"""
import numpy as np
import pytest

from gpu_helpers import TOL_F32, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def test_noalloc_steps_match_the_context_path_on_two_calls():
    torch = require_gpu()
    from paper_2009_12279_gb300 import Solver, lbve, workloads

    shape = (40, 24, 20)  # 19,200 cells, ragged against the 32-thread x blocks
    nx, ny, nz = shape
    n = nx * ny * nz
    np_ = (n + 63) // 64 * 64
    assert n <= lbve.NOALLOC_MAX_CELLS
    flags = workloads.channel_flags(shape, 1, top_flag=workloads.WALL0)
    flags[(workloads.random_obstacles(shape, 0.03, 11) == 1) & (flags == 0)] = workloads.NOSLIP
    wall = [(1.5e-3, 0.0, -5e-4)]
    prm = dict(periodic=(1, 0, 1), eta=1.0 / 6.0, beta=0.5, lambda_p=200.0, body_force=(2e-6, 0.0, 1e-6))
    u0 = workloads.random_velocity(shape, 1e-3, 12) * (flags == 0)
    t0 = workloads.random_stress(shape, 1e-5, 13) * (flags == 0)

    ref = Solver(shape, precision="f32", **prm)
    ref.set_geometry(flags, wall)
    ref.init_fields(u=u0, tau=t0)
    f_init = ref.read_pdfs().reshape(19, n)

    dev = torch.device("cuda")
    f = torch.zeros((19, np_), dtype=torch.float32, device=dev)
    f[:, :n] = torch.from_numpy(f_init - W[:, None] * prm.get("rho0", 1.0)).to(dev, torch.float32)
    tau_a = torch.zeros((6, np_), dtype=torch.float32, device=dev)
    tau_a[:, :n] = torch.from_numpy(t0.reshape(6, n)).to(dev, torch.float32)
    tau_b = torch.zeros_like(tau_a)
    fl = torch.from_numpy(flags.reshape(n)).to(dev)
    params = lbve.make_params(shape, precision="f32", **prm)
    stream = torch.cuda.current_stream().cuda_stream
    fluid = flags.reshape(n) == 0

    t = 0
    for nsteps in (10, 6):  # even counts keep f in the plain layout and tau in tau_a
        lbve.step_noalloc(params, f.data_ptr(), tau_a.data_ptr(), tau_b.data_ptr(), fl.data_ptr(), wall,
                          t0=t, nsteps=nsteps, stream=stream)
        torch.cuda.synchronize()
        t += nsteps
        ref.step(nsteps)
        f_ref = ref.read_pdfs().reshape(19, n)
        _, _, tau_ref, _ = ref.read_fields()
        f_got = f[:, :n].double().cpu().numpy() + W[:, None]
        tau_got = tau_a[:, :n].double().cpu().numpy()
        assert np.isfinite(f_got).all() and np.isfinite(tau_got).all()
        assert rel_l2(f_got[:, fluid] - W[:, None], f_ref[:, fluid] - W[:, None]) <= TOL_F32
        assert rel_l2(tau_got[:, fluid], tau_ref.reshape(6, n)[:, fluid]) <= TOL_F32


def test_noalloc_rejects_oversized_grids():
    require_gpu()
    from paper_2009_12279_gb300 import lbve

    big = lbve.make_params((128, 128, 64), precision="f32")  # 2^20 cells > the 2^19 limit
    with pytest.raises(lbve.LbveError, match="LBVE_NOALLOC_MAX_CELLS"):
        lbve.step_noalloc(big, 1, 1, 1, 1, nsteps=1)
