"""Parity at the full size of the throughput workload, in the launch configuration that
bench.py times: a 512^3 periodic box with 1 % seeded obstacles and the bench's own
device-drawn initial velocity, stepped by the default (split) schedule.

The oracle cannot step 134 M cells, but it does not need to: after T steps a cell depends
only on cells within 2T of it (the stream-collide reaches one cell, the stress update
reads face neighbours' velocity, which in turn depends on their face neighbours' stress).
For each sampled cell the oracle steps a periodic sub-box of side 2M + 1 (M > 2T) cut from
the same initial fields and flags; whatever the sub-box's wrong, wrapped border does
cannot reach its centre within T steps, so the centre is the exact FP64 result.  The
CUDA side is read through lbve_probe (19 PDFs, rho, u, tau of the listed cells).
"""
import numpy as np
import pytest

from gpu_helpers import TOL_F32, TOL_F64, oracle_subbox_centre, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

N = 512
T = 4            # steps: both AA parities, twice
M = 2 * T + 2    # sub-box margin around the sampled cell
W_D3Q19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


@pytest.fixture(scope="module")
def setup():
    torch = require_gpu()
    from paper_2009_12279_gb300 import workloads

    cfg = workloads.config_throughput(N)
    flags = cfg["flags_fn"]()  # (z, y, x)
    # the sampled cells: random ones, fluid cells next to obstacles, cells on the periodic faces
    rng = np.random.default_rng(2024)
    cells = [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(16)]
    solid = np.argwhere(flags != 0)
    for z, y, x in solid[rng.choice(len(solid), 16, replace=False)]:
        for dz, dy, dx in ((0, 0, 1), (0, 1, 0), (1, 0, 0), (0, 1, 1)):
            zq, yq, xq = (z + dz) % N, (y + dy) % N, (x + dx) % N
            if flags[zq, yq, xq] == 0:
                cells.append((int(xq), int(yq), int(zq)))
                break
    for k in range(16):
        c = [int(v) for v in rng.integers(0, N, 3)]
        c[k % 3] = 0 if k % 2 else N - 1
        cells.append(tuple(c))
    return torch, cfg, flags, cells


def _device_velocity(torch):
    """The bench's initial velocity: U(-1e-3, 1e-3) per component, torch Philox seed 1."""
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    return (torch.rand((3, N, N, N), generator=g, device="cuda", dtype=torch.float64) * 2.0 - 1.0) * 1e-3


def _run(precision, setup):
    torch, cfg, flags, cells = setup
    from paper_2009_12279_gb300 import Solver

    u = _device_velocity(torch)
    # sub-boxes of the initial velocity and flags around every sampled cell (periodic wrap)
    off = np.arange(-M, M + 1)
    subs = []
    for x, y, z in cells:
        xi, yi, zi = (x + off) % N, (y + off) % N, (z + off) % N
        tx = torch.as_tensor(xi, device="cuda")
        ty = torch.as_tensor(yi, device="cuda")
        tz = torch.as_tensor(zi, device="cuda")
        us = u.index_select(1, tz).index_select(2, ty).index_select(3, tx).cpu().numpy()
        fs = flags[np.ix_(zi, yi, xi)]
        subs.append((us, fs))
    s = Solver(cfg["shape"], precision=precision, **cfg["params"])
    s.set_geometry(flags)
    s.init_fields_device(0, u.data_ptr(), 0)
    s.synchronize()
    del u
    torch.cuda.empty_cache()
    s.step(T)
    idx = [x + N * (y + N * z) for x, y, z in cells]
    got = s.probe(idx)
    s.close()
    ref = np.array([oracle_subbox_centre(cfg["params"], fs, us, T) for us, fs in subs])
    return got, ref, cells, flags


def _errors(got, ref, cells, flags):
    fluid = np.array([flags[z, y, x] == 0 for x, y, z in cells])
    assert fluid.sum() >= 40
    g, r = got[fluid], ref[fluid]
    return {
        "f_dev": rel_l2(g[:, :19] - W_D3Q19, r[:, :19] - W_D3Q19),
        "rho": float(np.abs(g[:, 19] - r[:, 19]).max()),
        "u": rel_l2(g[:, 20:23], r[:, 20:23]),
        "tau": rel_l2(g[:, 23:29], r[:, 23:29]),
    }


def test_fp32_full_size_sampled_cells_match_oracle(setup, capsys):
    got, ref, cells, flags = _run("f32", setup)
    e = _errors(got, ref, cells, flags)
    with capsys.disabled():
        print(f"\n[512^3 f32, {len(cells)} sampled cells, {T} steps] {e}")
    assert max(e["f_dev"], e["u"], e["tau"]) <= TOL_F32, e
    assert e["rho"] <= 1e-6, e


def test_fp64_full_size_sampled_cells_match_oracle(setup, capsys):
    got, ref, cells, flags = _run("f64", setup)
    e = _errors(got, ref, cells, flags)
    with capsys.disabled():
        print(f"\n[512^3 f64, {len(cells)} sampled cells, {T} steps] {e}")
    assert max(e["f_dev"], e["u"], e["tau"]) <= TOL_F64, e
    assert e["rho"] <= 1e-14, e
