"""lbve_step_noalloc: time steps on caller-owned device buffers with no device allocation.

Callers that cannot call cudaMalloc (for example code running inside a framework that
owns all device memory through its own pool, or a process that forbids allocation once
it has started serving) keep the solve's state in their own buffers and advance it with
this entry point, whose intermediates live in fixed device arrays inside the library.

These tests build such buffers with torch, advance them with two calls in a row, and
compare each result with the regular context path (lbve_create / lbve_step) on the same
input.  Both run the same kernels on the same values, so the stored PDFs and stresses must
be bitwise equal, in every storage precision, for even and odd step counts (the in-place
odd layout and the stress in the second buffer), and with particle flags in the caller's
field, which this entry point treats as resting walls.

The file is collected last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu

W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 0], [-1, -1, 0],
              [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1],
              [0, 1, -1], [0, -1, 1]])
OPP = np.array([0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17])
PART_FLAG = 64  # first particle flag value of the flag field


def _torch_dtype(torch, precision):
    return {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[precision]


def _unpermute(raw, shape, parity):
    """PDFs f_i(r) from raw storage (19, nz, ny, nx): at an odd time, f_i(r) sits in slot
    -i of cell r - c_i (the in-place layout), with periodic wrap in every direction."""
    if parity == 0:
        return raw
    out = np.empty_like(raw)
    for i in range(19):
        # out[i][r] = raw[opp(i)][r - c_i]  ->  roll by +c_i along each axis
        out[i] = np.roll(raw[OPP[i]], shift=(C[i, 2], C[i, 1], C[i, 0]), axis=(0, 1, 2))
    return out


def _case(with_particle_flags):
    from paper_2009_12279_gb300 import workloads

    shape = (40, 24, 20)  # 19,200 cells, ragged against the 64-wide stream-collide blocks
    flags = workloads.channel_flags(shape, 1, top_flag=workloads.WALL0)
    flags[(workloads.random_obstacles(shape, 0.03, 11) == 1) & (flags == 0)] = workloads.NOSLIP
    ref_flags = flags.copy()
    if with_particle_flags:
        # a small block of cells flagged as a particle: this entry point has no particle
        # table and treats them as a resting wall, i.e. as no-slip cells in the context
        flags[8:11, 9:12, 14:18] = PART_FLAG
        ref_flags[8:11, 9:12, 14:18] = workloads.NOSLIP
    wall = [(1.5e-3, 0.0, -5e-4)]
    prm = dict(periodic=(1, 0, 1), eta=1.0 / 6.0, beta=0.5, lambda_p=200.0, body_force=(2e-6, 0.0, 1e-6))
    u0 = workloads.random_velocity(shape, 1e-3, 12) * (ref_flags == 0)
    t0 = workloads.random_stress(shape, 1e-5, 13) * (ref_flags == 0)
    return shape, flags, ref_flags, wall, prm, u0, t0


@pytest.mark.parametrize("precision", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("calls", [(10, 6), (7, 5)], ids=["even", "odd"])
@pytest.mark.parametrize("particle_flags", [False, True], ids=["walls", "particle_flags"])
def test_noalloc_steps_equal_the_context_path_bitwise(precision, calls, particle_flags):
    torch = require_gpu()
    from paper_2009_12279_gb300 import Solver, lbve

    shape, flags, ref_flags, wall, prm, u0, t0 = _case(particle_flags)
    nx, ny, nz = shape
    n = nx * ny * nz
    np_ = (n + 63) // 64 * 64
    assert n <= lbve.NOALLOC_MAX_CELLS

    ref = Solver(shape, precision=precision, **prm)
    ref.set_geometry(ref_flags, wall)
    ref.init_fields(u=u0, tau=t0)
    params = ref.params
    # the context's stored PDFs at t = 0 are the caller's initial state: read them back as
    # f_i = w_i rho0 + stored (exact in FP64) and store the deviation again on the device
    f0 = ref.read_pdfs().reshape(19, n)
    _, _, tau_init, _ = ref.read_fields()
    shifted = precision != "f64"
    scale = 2.0 ** 15 if precision == "f16" else 1.0

    dev = torch.device("cuda")
    sdt = _torch_dtype(torch, precision)
    rdt = torch.float64 if precision == "f64" else torch.float32
    base = W[:, None] * prm.get("rho0", 1.0) if shifted else 0.0
    stored0 = torch.from_numpy((f0 - base) * scale)  # exact: the context stored these values
    f = torch.zeros((19, np_), dtype=sdt, device=dev)
    f[:, :n] = stored0.to(dev).to(sdt)
    tau_x = torch.zeros((6, np_), dtype=rdt, device=dev)
    tau_x[:, :n] = torch.from_numpy(tau_init.reshape(6, n)).to(dev).to(rdt)
    tau_y = torch.zeros_like(tau_x)
    fl = torch.from_numpy(np.ascontiguousarray(flags.reshape(n))).to(dev)
    stream = torch.cuda.current_stream().cuda_stream
    fluid = ref_flags.reshape(n) == 0

    # the initial copy is exact: the caller's buffer holds the context's stored values
    assert np.array_equal(f[:, :n].double().cpu().numpy() / scale + base, f0)

    t = 0
    for nsteps in calls:
        lbve.step_noalloc(params, f.data_ptr(), tau_x.data_ptr(), tau_y.data_ptr(), fl.data_ptr(), wall,
                          t0=t, nsteps=nsteps, stream=stream)
        torch.cuda.synchronize()
        t += nsteps
        if nsteps % 2:
            tau_x, tau_y = tau_y, tau_x  # the stress at t now sits in the second buffer
        ref.step(nsteps)
        raw = f[:, :n].double().cpu().numpy().reshape(19, nz, ny, nx) / scale
        got = (_unpermute(raw, shape, t & 1).reshape(19, n) + base)
        want = ref.read_pdfs().reshape(19, n)
        _, _, tau_ref, _ = ref.read_fields()
        tau_got = tau_x[:, :n].double().cpu().numpy()
        assert np.isfinite(got).all() and np.isfinite(tau_got).all()
        bad = np.argwhere(got[:, fluid] != want[:, fluid])
        assert bad.size == 0, (precision, t, bad[:5], got[:, fluid][tuple(bad[0])], want[:, fluid][tuple(bad[0])])
        assert np.array_equal(tau_got[:, fluid], tau_ref.reshape(6, n)[:, fluid]), (precision, t)
    ref.close()


def test_noalloc_rejects_oversized_grids():
    require_gpu()
    from paper_2009_12279_gb300 import lbve

    big = lbve.make_params((128, 128, 64), precision="f32")  # 2^20 cells > the 2^19 limit
    with pytest.raises(lbve.LbveError, match="LBVE_NOALLOC_MAX_CELLS"):
        lbve.step_noalloc(big, 1, 1, 1, 1, nsteps=1)
