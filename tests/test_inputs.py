"""Seeded input generators: SplitMix64 against its published reference outputs, and the
parameter recipes."""
import numpy as np
import pytest

from paper_1310_7450_gb300 import inputs


def test_splitmix64_published_outputs():
    # reference outputs of SplitMix64 seeded with 1234567 and with 0 (Vigna's splitmix64.c)
    got = [int(v) for v in inputs.splitmix64(1234567, np.arange(1, 6))]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]
    assert int(inputs.splitmix64(0, [1])[0]) == 0xE220A8397B1DCDAF


def test_uniform_range_and_density():
    u = inputs.uniform_pm1(3, np.arange(1, 100001))
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01
    rho = inputs.initial_density(8, 16, 1.0, 1e-6, 1)
    assert rho.shape == (16, 8) and np.abs(rho - 1).max() <= 1e-6
    assert np.array_equal(inputs.initial_density(8, 16, 1.0, 0.0, 1), np.ones((16, 8)))
    # a sub-grid drawn with an offset reproduces the rows of the full grid
    full = inputs.initial_density(8, 16, 1.0, 1e-3, 9)
    part = inputs.initial_density(8, 4, 1.0, 1e-3, 9, node_offset=8 * 5)
    assert np.array_equal(part, full[5:9])


def test_matched_params_viscosity():
    p = inputs.matched_params(0.9, 100.0, 0.1, 1e-3, 1e-6)
    assert p["G_inf"] * p["tau0"] * (1 + p["theta"]) == pytest.approx((0.9 - 0.5) / 3)
    y = inputs.yield_stress_channel(64, tau=1e4)
    assert y["tau0"] == pytest.approx(100.0) and y["G_inf"] == pytest.approx(1.3201320132e-5)
    assert y["g_x"] * 32 / y["G_inf"] == pytest.approx(0.5)


def test_sweep_draws_ranges():
    ny, b, eps = inputs.sweep_draws(512, 3)
    assert ny.min() >= 32 and ny.max() <= 1024 and 1e-8 <= b.min() and b.max() <= 1e-5
    assert np.abs(eps).max() <= 0.1
