"""The synthetic input recipe: the generators reproduce the configurations they stand for
(shapes, walls, obstacle fractions, parameter derivations), seeded and reproducible.
CPU only."""
import math

import numpy as np
import pytest

from paper_2009_12279_gb300 import workloads


def test_square_duct_centreline_factor():
    """Textbook Fourier series for Poiseuille flow in a square duct of side H: the
    centreline velocity is 0.07367 g H^2 / eta; a very flat duct tends to the plane
    channel's 1/8 (in the narrow side)."""
    assert workloads.duct_centreline_factor(1.0) == pytest.approx(0.073671, abs=2e-6)
    assert workloads.duct_centreline_factor(50.0) == pytest.approx(0.125, rel=1e-6)


def test_sphere_duct_configuration():
    cfg = workloads.config_sphere_duct(128, radius=12.0, beta=0.5, wi=0.5, g=5e-6, eta=1.0)
    fl = cfg["flags"]
    n = 128
    assert fl.shape == (n, n, n) and cfg["params"]["periodic"] == (1, 0, 0)
    # walls on the y and z faces, none inside the x-periodic direction
    assert np.all(fl[:, 0, :] == workloads.NOSLIP) and np.all(fl[:, -1, :] == workloads.NOSLIP)
    assert np.all(fl[0] == workloads.NOSLIP) and np.all(fl[-1] == workloads.NOSLIP)
    # the sphere: cells within R of the box centre (63.5, 63.5, 63.5)
    c = (n - 1) / 2.0
    z, y, x = np.nonzero(fl == workloads.WALL0)
    d2 = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2
    assert d2.max() <= 144.0
    assert len(x) == pytest.approx(4.0 / 3.0 * math.pi * 12.0**3, rel=0.05)
    # lambda from Wi = lambda u_ref / R with the duct centreline velocity of side H = n - 2
    u_ref = 0.073671 * 5e-6 * (n - 2.0) ** 2 / 1.0
    assert cfg["u_ref"] == pytest.approx(u_ref, rel=1e-4)
    assert cfg["params"]["lambda_p"] * cfg["u_ref"] / 12.0 == pytest.approx(0.5, rel=1e-12)
    assert cfg["steps"] == 50000


def test_throughput_configuration_is_seeded():
    cfg = workloads.config_throughput(48)
    a, b = cfg["flags_fn"](), cfg["flags_fn"]()
    assert np.array_equal(a, b)
    frac = float((a != 0).mean())
    assert 0.007 < frac < 0.013  # Bernoulli(0.01) obstacles
    assert cfg["params"]["periodic"] == (1, 1, 1)
    assert cfg["params"]["beta"] == 0.5 and cfg["params"]["lambda_p"] == 1000.0
    other = workloads.config_throughput(48, seed=1)["flags_fn"]()
    assert not np.array_equal(a, other)


def test_channel_configuration():
    cfg = workloads.config_channel()
    fl = cfg["flags"]
    assert cfg["shape"] == (4, 32, 4) and fl.shape == (4, 32, 4)
    assert np.all(fl[:, 0, :] != 0) and np.all(fl[:, 31, :] != 0) and np.all(fl[:, 1:31, :] == 0)
    p = cfg["params"]
    assert p["eta"] == pytest.approx(1.0 / 6.0) and p["beta"] == 0.5 and p["lambda_p"] == 3000.0
    assert tuple(p["body_force"]) == (1e-6, 0.0, 0.0)
