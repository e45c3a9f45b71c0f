"""The closed forms used as pins are themselves checked: the printed root of the quadratic,
its limits (Sec. III B), the plug asymptotes, and the printed plug half-width."""
import json
import math
import os

import numpy as np
import pytest

from oracle import analytic

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("theta", [0.5, 10.0, 100.0, 1000.0])
def test_printed_root_solves_quadratic(theta):
    for wpH in [0.05, 0.5, 3.0]:
        for d in np.linspace(0.0, 1.0, 11):
            x = analytic.dvdd(d, wpH, theta, 0.1)
            scale = wpH * d + 1e-300
            assert abs(analytic.quadratic_residual(d, x, wpH, theta, 0.1)) <= 1e-12 * max(scale, 1e-12) * (1 + theta)
            assert x <= 0.0  # velocity decreases towards the wall


def test_force_balance_of_root():
    """Eq. (nspoiseuille) at steady state: (1 + theta/(1 + theta|v'|/gamma_c)) v' = -wp H d."""
    for theta in [1.0, 100.0]:
        for d in [0.1, 0.5, 0.9]:
            x = analytic.dvdd(d, 0.5, theta, 0.1)
            assert (1 + theta / (1 + theta * abs(x) / 0.1)) * x == pytest.approx(-0.5 * d, rel=1e-12)


def test_small_theta_and_small_pressure_limits():
    """Sec. III B: small theta -> -wpH d (1 - theta); small wp -> -wpH d/(1+theta)."""
    d = 0.7
    th = 1e-4
    assert analytic.dvdd(d, 0.5, th, 0.1) == pytest.approx(-0.5 * d * (1 - th), rel=1e-6)
    wpH = 1e-7
    assert analytic.dvdd(d, wpH, 10.0, 0.1) == pytest.approx(-wpH * d / 11.0, rel=1e-5)
    assert analytic.dvdd(d, 0.5, 0.0, 0.1) == -0.35


def test_large_pressure_limit():
    """Sec. III B: wp >> gamma_c/(H d): dv/dd -> -wp H d + gamma_c."""
    d, wpH = 0.9, 1e4
    assert analytic.dvdd(d, wpH, 10.0, 0.1) == pytest.approx(-wpH * d + 0.1, rel=1e-4)


def test_plug_asymptotes_and_printed_half_width():
    """Eq. (plug) for theta -> infinity and the plug half-width 0.2 printed in Sec. IV A."""
    g = GOLDEN["plug_half_width"]
    dc = analytic.plug_half_width(g["wpH"], g["gamma_c"])
    assert dc == pytest.approx(g["value"], rel=1e-15)
    theta = 1e7
    for d in [0.5, 0.8, 1.0]:  # outer branch
        assert analytic.dvdd(d, 0.5, theta, 0.1) == pytest.approx(analytic.plug_asymptote(d, 0.5, theta, 0.1), rel=1e-5)
    for d in [0.02, 0.1]:  # inner branch, O(1/theta)
        x = analytic.dvdd(d, 0.5, theta, 0.1)
        assert x == pytest.approx(analytic.plug_asymptote(d, 0.5, theta, 0.1), rel=1e-3)
        assert abs(x) < 1e-6


def test_plug_edge_is_where_shear_stress_equals_yield_stress():
    """Sec. III B: |sigma_xy(d_c)| = G gamma_c, and the normal-stress asymptotes of Eq. (mwnd)."""
    dc = analytic.plug_half_width(0.5, 0.1)
    assert 0.5 * dc == pytest.approx(0.1)
    assert analytic.normal_stress_asymptote(0.9, 0.5, 1.0, 0.1) == pytest.approx(2 * 0.1 ** 2)
    assert analytic.normal_stress_asymptote(0.1, 0.5, 1.0, 0.1) == pytest.approx(2 * 0.05 ** 2)


def test_profile_integration_newtonian():
    """theta = 0: the integrated profile is the parabola (H/tau0) wp H (1 - d^2)/2."""
    ny, g, G, tau0 = 40, 1e-6, 1e-3, 7.0
    u = analytic.channel_profile(ny, g, G, tau0, 0.0, 0.1)
    np.testing.assert_allclose(u, analytic.newtonian_parabola(ny, g, G * tau0), rtol=1e-12)


def test_startup_series_limits():
    ny, g, nu = 32, 1e-6, 0.1
    assert np.abs(analytic.newtonian_startup(ny, g, nu, 0.0)).max() < 1e-6 * analytic.newtonian_parabola(ny, g, nu).max()
    np.testing.assert_allclose(analytic.newtonian_startup(ny, g, nu, 1e7), analytic.newtonian_parabola(ny, g, nu), rtol=1e-12)
    # early times: u = g t in the core (diffusion has not reached it)
    assert analytic.newtonian_startup(ny, g, nu, 10.0)[ny // 2] == pytest.approx(g * 10.0, rel=1e-6)


def test_yield_drop():
    assert analytic.yield_pressure_drop(1e-3, 0.1, 32.0) == pytest.approx(2e-3 * 0.1 / 64)
    assert math.isclose(GOLDEN["gamma_c"]["value"], 0.1)
