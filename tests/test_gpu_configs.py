"""The fixed-sphere duct (128^3) and the sedimentation box (64 x 64 x 256) at their full
sizes, through the C ABI.

Short runs are compared with the oracle directly: FP64 to 1e-12 (fields, drag on the
fixed sphere, particle state), FP32 within 1e-5.  The sedimentation curve over the long
run is then compared between the GPU's FP64 mode, which the short run has just shown to
be the oracle's arithmetic, and the FP32 and BF16-storage modes: the oracle itself would
need hours for it on the host cores.
"""
import numpy as np
import pytest

from gpu_helpers import TOL_F32, TOL_F64, compare, pair, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _duct():
    from paper_2009_12279_gb300 import workloads

    return workloads.config_sphere_duct(128, radius=12.0, beta=0.5, wi=0.5)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_sphere_duct_full_size_matches_oracle(precision, capsys):
    cfg = _duct()
    g, o = pair(cfg["shape"], cfg["params"], cfg["flags"], cfg["wall_vel"], precision=precision)
    T = 16
    g.step(T)
    o.step(T)
    e = compare(g, o)
    drag_g, drag_o = g.body_forces()[2], o.body_forces()[2]  # wall class 0 (flag 2): the sphere
    with capsys.disabled():
        print(f"\n[sphere duct 128^3 {precision}, {T} steps] {e}; drag x oracle {drag_o[0]:.6e} gpu {drag_g[0]:.6e}")
    assert drag_o[0] > 0.0  # the sphere is pushed along the flow
    if precision == "f64":
        assert max(e["f"], e["u"], e["tau"]) <= TOL_F64, e
        assert np.linalg.norm(drag_g - drag_o) <= TOL_F64 * np.linalg.norm(drag_o)
    else:
        assert max(e["u"], e["tau"]) <= TOL_F32, e
        assert np.linalg.norm(drag_g - drag_o) <= TOL_F32 * np.linalg.norm(drag_o)


def _sediment():
    """Closed 64 x 64 x 256 box, R = 8 sphere at (31.5, 31.5, 256 - 3R), rho_p = 1.2,
    gravity from Re = 2 rho v_St R / eta = 0.1, eta = 1/6, beta = 0.5, Wi = lambda v_St / R
    = 0.25."""
    nx, ny, nz = 64, 64, 256
    fl = np.ones((nz, ny, nx), np.uint8)
    fl[1:-1, 1:-1, 1:-1] = 0
    R, rho_p, eta = 8.0, 1.2, 1.0 / 6.0
    v_st = 0.1 * eta / (2.0 * R)
    vol = 4.0 / 3.0 * np.pi * R**3
    F = 6.0 * np.pi * eta * R * v_st  # Stokes drag at v_St balances the net gravity force
    lam = 0.25 * R / v_st
    prm = dict(periodic=(0, 0, 0), eta=eta, beta=0.5, lambda_p=lam)
    part = dict(X=((nx - 1) / 2.0, (ny - 1) / 2.0, nz - 3 * R), R=R, rho_p=rho_p, Fext=(0.0, 0.0, -F))
    assert abs(F / ((rho_p - 1.0) * vol) - 6.1e-5) < 0.2e-5  # g of the configuration
    return (nx, ny, nz), prm, fl, part


def _add(obj, part):
    return obj.add_particle(part["X"], part["R"], part["rho_p"], v=(0, 0, 0), w=(0, 0, 0), Fext=part["Fext"],
                            Text=(0, 0, 0))


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_sedimentation_full_size_matches_oracle(precision, capsys):
    shape, prm, fl, part = _sediment()
    g, o = pair(shape, prm, fl, precision=precision)
    _add(g, part)
    _add(o, part)
    T = 24
    g.step(T)
    o.step(T)
    e = compare(g, o)
    pg, po = g.read_particle(0), o.read_particle(0)
    perr = max(rel_l2(pg[k], po[k]) for k in ("X", "v"))
    with capsys.disabled():
        print(f"\n[sedimentation 64x64x256 {precision}, {T} steps] {e}; particle X, v {perr:.2e}; "
              f"v_z {po['v'][2]:.4e}")
    assert po["v"][2] < 0.0
    if precision == "f64":
        assert max(e["f"], e["u"], e["tau"]) <= TOL_F64, e
        assert perr <= TOL_F64
    else:
        assert max(e["u"], e["tau"]) <= TOL_F32, e
        assert perr <= TOL_F32


def test_sedimentation_full_size_curve(capsys):
    """20,000 steps, v_z every 100: FP32 and BF16 storage against the FP64 mode.  The
    curve carries a spike at every cell conversion (the fill/drain impulse); a rounding
    difference that moves one conversion by a step shifts a spike, so single samples can
    differ by ~1e-3 of the peak velocity while the curve itself agrees.  Compared are the
    1000-step running means, the final velocity and the conversion counts."""
    from paper_2009_12279_gb300 import Solver

    shape, prm, fl, part = _sediment()
    curves, convs = {}, {}
    for prec in ("f64", "f32", "bf16"):
        s = Solver(shape, precision=prec, **prm)
        s.set_geometry(fl)
        _add(s, part)
        vs = []
        for _ in range(200):
            s.step(100)
            vs.append(s.read_particle(0)["v"][2])
        curves[prec] = np.array(vs)
        c = s.conversions()
        convs[prec] = c["created"] + c["destroyed"]
        s.close()
        assert c["created"] > 0 and c["destroyed"] > 0, prec  # the sphere moved across cells
    ref = curves["f64"]
    scale = np.abs(ref).max()

    def mean10(a):
        return np.convolve(a, np.ones(10) / 10.0, mode="valid")

    err = {}
    for prec in ("f32", "bf16"):
        err[prec] = (np.abs(curves[prec] - ref).max() / scale, np.abs(mean10(curves[prec]) - mean10(ref)).max() / scale,
                     abs(curves[prec][-1] - ref[-1]) / scale)
    with capsys.disabled():
        print(f"\n[sedimentation curve 64x64x256, 20000 steps] v_z(end) f64 {ref[-1]:.5e}, conversions {convs}; "
              + "; ".join(f"{p}: samples {a:.2e}, running mean {b:.2e}, final {c:.2e}" for p, (a, b, c) in err.items()))
    assert ref[-1] < 0.0 and np.all(np.isfinite(ref))
    assert convs["f32"] == convs["f64"]
    assert err["f32"][1] <= 5e-4 and err["f32"][2] <= 1e-4
    assert err["bf16"][1] <= 2e-3 and err["bf16"][2] <= 1e-3


def test_sphere_duct_drag_over_the_full_run(capsys):
    """The duct's 50,000 steps in FP32 and BF16 storage, the drag on the fixed sphere
    every 2000 steps; the FP64 mode (the oracle's arithmetic, as the short run above
    shows) runs the first 4000 steps only, FP64 arithmetic being slow on this part (the
    whole run in FP64 took ~6 min).  No cell converts, so the drag histories are smooth
    and compared sample by sample: FP32 and BF16 against FP64 where it ran, BF16 against
    FP32 over the whole run, all relative to the steady drag."""
    from paper_2009_12279_gb300 import Solver

    cfg = _duct()
    hist = {}
    for prec, steps in (("f64", 4000), ("f32", cfg["steps"]), ("bf16", cfg["steps"])):
        s = Solver(cfg["shape"], precision=prec, **cfg["params"])
        s.set_geometry(cfg["flags"], cfg["wall_vel"])
        d = []
        for _ in range(steps // 2000):
            s.step(2000)
            d.append(s.body_forces()[2][0])
        hist[prec] = np.array(d)
        s.close()
    ref, d32, d16 = hist["f64"], hist["f32"], hist["bf16"]
    k = len(ref)
    scale = np.abs(d32).max()  # the steady drag: differences relative to it
    e32 = np.abs(d32[:k] - ref).max() / scale
    e16 = np.abs(d16[:k] - ref).max() / scale
    e16_32 = np.abs(d16 - d32).max() / scale
    # Stokes drag of the sphere at the empty-duct centreline velocity (no wall correction)
    stokes = 6.0 * np.pi * cfg["params"]["eta"] * 12.0 * cfg["u_ref"]
    with capsys.disabled():
        print(f"\n[sphere duct 128^3, {cfg['steps']} steps] drag f32 {d32[-1]:.5e} "
              f"({d32[-1] / stokes:.2f} x Stokes at u_ref); first {2000 * k} steps against f64: f32 {e32:.2e}, "
              f"bf16 {e16:.2e}; whole run bf16 against f32 {e16_32:.2e}")
    assert np.all(np.isfinite(d32)) and d32[-1] > 0.0
    assert abs(d32[-1] - d32[-2]) <= 0.05 * d32[-1]  # close to steady
    assert e32 <= 1e-4
    assert e16 <= 1e-2
    assert e16_32 <= 1e-2
