"""Shared helpers of the GPU parity tests: build the same solve on the CUDA library and on
the FP64 oracle from one workload description, and compare fields."""
import numpy as np

TOL_F64 = 1e-12  # relative L2, FP64 mode after up to 1000 steps
TOL_F32 = 1e-5   # relative L2, FP32 mode after up to 1000 steps


def require_gpu():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2009_12279_gb300 import build, lbve

    build.build()
    lbve.load()
    return torch


def oracle_kwargs(params):
    kw = dict(params)
    if "body_force" in kw:
        kw["g"] = kw.pop("body_force")
    for k in ("precision", "pdf_scale_log2", "schedule", "block_x"):
        kw.pop(k, None)
    return kw


def pair(shape, params, flags=None, wall_vel=(), rho=None, u=None, tau=None, precision="f64", **gpu_kw):
    from oracle import oracle
    from paper_2009_12279_gb300 import Solver

    g = Solver(shape, precision=precision, **params, **gpu_kw)
    o = oracle.Oracle(shape, wall_vel=wall_vel, **oracle_kwargs(params))
    if flags is not None:
        g.set_geometry(flags, wall_vel)
        o.set_flags(flags)
    if rho is not None or u is not None or tau is not None:
        g.init_fields(rho=rho, u=u, tau=tau)
        o.init_fields(rho=rho, u=u, tau=tau)
    return g, o


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    na = np.linalg.norm(a - b)
    if nb == 0.0:
        return na
    return na / nb


def compare(g, o, fluid=None):
    """Relative L2 errors of PDFs, u and tau and the max abs density error (fluid cells)."""
    rg, ug, tg, fg = g.read_fields()
    ro, uo, to, fo = o.read_fields()
    assert np.array_equal(fg, fo), "flag fields differ"
    fluid = fg == 0 if fluid is None else fluid
    pg, po = g.read_pdfs(), o.read_pdfs()
    return {
        "f": rel_l2(pg[:, fluid], po[:, fluid]),
        "rho": float(np.abs(rg[fluid] - ro[fluid]).max()) if fluid.any() else 0.0,
        "u": rel_l2(ug[:, fluid], uo[:, fluid]),
        "tau": rel_l2(tg[:, fluid], to[:, fluid]),
    }


def oracle_subbox_centre(params, flags_sub, u_sub, steps):
    """The oracle's (19 PDFs, rho, u, tau) after `steps` steps at the centre of a periodic
    sub-box (side 2M + 1, flags (z, y, x), u (3, z, y, x)) cut around one cell of a larger
    periodic solve.  A cell depends only on cells within 2 per step, so for M > 2 steps the
    centre equals that cell of the full solve."""
    from oracle import oracle

    side = flags_sub.shape[0]
    M = side // 2
    o = oracle.Oracle((side, side, side), **oracle_kwargs(params))
    o.set_flags(flags_sub)
    o.init_fields(u=u_sub)
    o.step(steps)
    rho, u, tau, fl = o.read_fields()
    f = o.read_pdfs()
    o.close()
    c = M + side * (M + side * M)
    out = np.zeros(29)
    out[:19] = f.reshape(19, -1)[:, c]
    if fl.reshape(-1)[c] == 0:
        out[19] = rho.reshape(-1)[c]
        out[20:23] = u.reshape(3, -1)[:, c]
        out[23:29] = tau.reshape(6, -1)[:, c]
    return out
