"""The oracle against an independent brute-force evaluation of whole time steps on tiny
grids (3^3 and 4^3 cells), element by element.

The brute force (``tests/brute_force.py``) restates the step cell by cell from the
paper's equations, with no code in common with the oracle.  Tiny grids wrap around so
that most cells sit next to a boundary of some kind: resting no-slip cells, two moving
wall classes, closed sides and a moving particle that converts cells in each step.  The
fields are random and off equilibrium, every finite-volume variant is exercised, and the
Giesekus term is switched on in some cases.  This pins the per-cell arithmetic of
boundary-adjacent cells, which the integral and analytic pins cannot see one cell at a
time: the gradient with two solid faces, the extrapolated stress next to a moving wall,
the bounced populations of moving boundaries, and the created-cell density and stress.
"""
import numpy as np
import pytest

import brute_force as bf

FV_FLUX, FV_SOURCE, FV_CTU, FV_DIVU = 1, 2, 4, 8
TOL = 1e-14


def _random_case(shape, periodic, seed, wall_classes=2, noslip_frac=0.2, wall_frac=0.12):
    """Flags (x, y, z), random rho, u, off-equilibrium PDFs and stress on every cell."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    flags = np.zeros(shape, np.uint8)
    r = rng.random(shape)
    flags[r < noslip_frac] = bf.NOSLIP
    for k in range(wall_classes):
        flags[(r >= noslip_frac + k * wall_frac) & (r < noslip_frac + (k + 1) * wall_frac)] = bf.WALL0 + k
    for a in range(3):  # a closed side has solid first and last layers
        if not periodic[a]:
            idx = [slice(None)] * 3
            idx[a] = 0
            flags[tuple(idx)] = bf.NOSLIP
            idx[a] = shape[a] - 1
            flags[tuple(idx)] = bf.WALL0 if wall_classes else bf.NOSLIP
    rho = 1.0 + 0.02 * rng.standard_normal(shape)
    u = rng.uniform(-0.05, 0.05, (3,) + shape)
    f = np.zeros((19,) + shape)
    for x in range(nx):
        for y in range(ny):
            for z in range(nz):
                f[:, x, y, z] = bf.Grid.equilibrium(rho[x, y, z], u[:, x, y, z]) * \
                    (1.0 + 0.05 * rng.standard_normal(19))
    t = 1e-3 * rng.standard_normal((3, 3) + shape)
    tau = 0.5 * (t + t.transpose(1, 0, 2, 3, 4))
    return flags, f, tau


def _oracle_order():
    from oracle import oracle

    c_o, _, _ = oracle.lattice()
    # index into the brute force's lattice of each of the oracle's directions
    return np.array([int(np.nonzero((bf.C == c).all(axis=1))[0][0]) for c in c_o])


def _to_zyx(a):
    """(..., x, y, z) -> (..., z, y, x)"""
    return np.ascontiguousarray(np.moveaxis(a, (-3, -1), (-1, -3)))


def _tau6(t33):
    """(3, 3, x, y, z) -> (6, z, y, x) in the layout xx, yy, zz, xy, xz, yz."""
    comps = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    return _to_zyx(np.stack([t33[i, j] for i, j in comps]))


CASES = [
    # shape, periodic, fv_terms, alpha, particle (X, R, rho_p, v, w), seed
    ((3, 3, 3), (1, 1, 1), FV_FLUX | FV_SOURCE, 0.0, None, 1),
    ((3, 3, 3), (1, 1, 1), FV_FLUX | FV_SOURCE | FV_CTU | FV_DIVU, 0.3, None, 2),
    ((4, 4, 4), (1, 0, 1), FV_FLUX, 0.0, None, 3),
    ((4, 4, 4), (1, 0, 1), FV_SOURCE, 0.2, None, 4),
    ((4, 4, 4), (0, 1, 1), FV_FLUX | FV_SOURCE | FV_CTU, 0.0, None, 5),
    ((4, 4, 4), (1, 1, 0), FV_FLUX | FV_SOURCE | FV_DIVU, 0.5, None, 6),
    ((4, 5, 4), (1, 0, 1), FV_FLUX | FV_SOURCE, 0.0,
     ((1.45, 2.0, 1.5), 1.05, 20.0, (0.35, 0.02, -0.01), (0.01, -0.02, 0.03)), 7),
    ((4, 5, 4), (1, 0, 1), FV_FLUX | FV_SOURCE | FV_CTU | FV_DIVU, 0.25,
     ((2.1, 2.2, 1.4), 1.2, 1.1, (-0.3, 0.05, 0.2), (-0.02, 0.01, 0.01)), 8),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_oracle_steps_equal_the_brute_force(oracle_mod, case):
    shape, periodic, fv_terms, alpha, part, seed = CASES[case]
    rng = np.random.default_rng(100 + seed)
    eta = rng.uniform(0.1, 0.3)
    beta = rng.uniform(0.2, 0.8)
    lam = rng.uniform(20.0, 80.0)
    g = rng.uniform(-1e-3, 1e-3, 3)
    wall = [tuple(rng.uniform(-2e-2, 2e-2, 3)) for _ in range(2)]
    flags, f, tau = _random_case(shape, periodic, seed)
    if part is not None:  # a fluid interior, so that the particle converts cells on its way,
        inner = flags[:, 1:-1, :]  # with one resting and one moving obstacle cell in it
        inner[...] = bf.FLUID
        inner[3, 0, 3] = bf.NOSLIP
        inner[0, 2, 3] = bf.WALL0 + 1
    kw = dict(periodic=periodic, eta=eta, beta=beta, lambda_p=lam, rho0=1.0, g=tuple(g), magic=3.0 / 16.0)

    grid = bf.Grid(shape, periodic, eta, beta, lam, 1.0, g, 3.0 / 16.0, wall, bool(fv_terms & FV_FLUX),
                   bool(fv_terms & FV_SOURCE), bool(fv_terms & FV_CTU), bool(fv_terms & FV_DIVU), alpha)
    o = oracle_mod.Oracle(shape, wall_vel=wall, fv_terms=fv_terms, giesekus_alpha=alpha, **kw)
    o.set_flags(_to_zyx(flags))
    perm = _oracle_order()
    o.write_pdfs(_to_zyx(f[perm]))
    o.write_tau(_tau6(tau))

    fd = {r: f[(slice(None),) + r].copy() for r in grid.cells()}
    td = {r: tau[(slice(None), slice(None)) + r].copy() for r in grid.cells()}
    fl = flags.copy()
    if part is not None:
        X, R, rho_p, v, w = part
        grid.place(bf.Particle(X, R, rho_p, v, w), fl, td)
        o.add_particle(X, R, rho_p, v=v, w=w)

    for step in range(3):
        fd, td, fl = grid.step(fd, td, fl)
        o.step(1)
        _, _, tau_o, flags_o = o.read_fields()
        f_o = o.read_pdfs()
        assert np.array_equal(flags_o, _to_zyx(fl)), f"step {step}: flags differ"
        fluid = flags_o == 0
        f_xyz = np.zeros((19,) + shape)
        t_xyz = np.zeros((3, 3) + shape)
        for r in grid.cells():
            f_xyz[(slice(None),) + r] = fd[r][perm]
            t_xyz[(slice(None), slice(None)) + r] = td[r]
        f_b, t_b = _to_zyx(f_xyz), _tau6(t_xyz)
        df = np.abs(f_b[:, fluid] - f_o[:, fluid]).max()
        dt = np.abs(t_b[:, fluid] - tau_o[:, fluid]).max() / max(np.abs(tau_o[:, fluid]).max(), 1e-300)
        assert df <= TOL, f"step {step}: PDFs differ by {df:.3e}"
        assert dt <= TOL * 10, f"step {step}: stress differs by {dt:.3e} (relative)"
        bo = o.body_forces()
        for k, Fb in grid.body_force.items():
            assert np.abs(bo[k] - Fb).max() <= TOL * max(1.0, np.abs(Fb).max()), (step, k, bo[k], Fb)
        if part is not None:
            P = grid.particles[0]
            po = o.read_particle(0)
            for name, a, b in (("X", P.X, po["X"]), ("v", P.v, po["v"]), ("w", P.w, po["w"]),
                               ("F", P.F, po["F"]), ("T", P.T, po["T"])):
                assert np.abs(a - b).max() <= TOL * max(1.0, np.abs(b).max()), (step, name, a, b)
            d = o.diag()
            assert (d["destroyed"], d["created"]) == (grid.destroyed, grid.created)
            dropped = [grid.dropped[i, j] for i, j in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))]
            assert np.abs(d["dropped_tau"] - dropped).max() <= 1e-18
    if part is not None:
        assert grid.destroyed > 0 and grid.created > 0, "the particle must convert cells both ways"
    o.close()


def test_brute_force_lattice_is_d3q19():
    """The generated velocity set: 19 velocities, weights summing to 1, isotropic second
    moment sum w c c = I/3, and opposite directions paired."""
    assert bf.C.shape == (19, 3)
    assert abs(bf.W.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia,ib->ab", bf.W, bf.C, bf.C), np.eye(3) / 3.0, atol=1e-15)
    assert (bf.C[bf.OPP] == -bf.C).all()
