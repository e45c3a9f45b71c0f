"""Per-node pins of the oracle (CPU): equilibrium, forcing term, constitutive equation.

Each check is fixed by the paper or by mathematics, not by re-typing the oracle's formula:
moments of n^eq (Eq. pieq / rhoj), moment conditions of F_i (below Eq. lbfab), the simple-shear,
planar-extension and yield-stress closed forms of Sec. III A, and an independent elimination.
"""
import math

import numpy as np
import pytest

from oracle import analytic

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)
CS2 = 1.0 / 3.0


def moments(v):
    m0 = v.sum()
    m1 = np.array([(CX * v).sum(), (CY * v).sum()])
    m2 = np.array([[(CX * CX * v).sum(), (CX * CY * v).sum()], [(CY * CX * v).sum(), (CY * CY * v).sum()]])
    return m0, m1, m2


def test_equilibrium_moments(oracle_mod):
    """Eq. (neq) must give sum n^eq = rho, sum c n^eq = rho u (Eq. rhoj) and
    sum c c n^eq = p0 + rho u u with p0 = rho c_s^2 (Eq. pieq)."""
    rng = np.random.default_rng(11)
    for _ in range(50):
        rho = 1.0 + 0.1 * rng.uniform(-1, 1)
        u = 0.1 * rng.uniform(-1, 1, 2)
        m0, m1, m2 = moments(oracle_mod.equilibrium(rho, u[0], u[1]))
        assert abs(m0 - rho) < 1e-15
        np.testing.assert_allclose(m1, rho * u, atol=1e-16)
        np.testing.assert_allclose(m2, rho * CS2 * np.eye(2) + rho * np.outer(u, u), atol=2e-16)


def test_equilibrium_rest_weights(oracle_mod):
    """At rest n^eq = a^{c_i} rho with the D2Q9 weights 4/9, 1/9, 1/36 (Sec. II A)."""
    w = oracle_mod.equilibrium(1.0, 0.0, 0.0)
    np.testing.assert_allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, rtol=0, atol=1e-17)


def test_forcing_moments(oracle_mod):
    """Moment conditions on F_i stated with Eq. (lbfab):
    sum F = (1 - 1/2tau) S,  sum c F = (1 - 1/2tau) f,
    sum c c F = (1-1/2tau)(u f + f u) + (1-1/2tau)(c_s^2 1 - u u) S - Sbar/tau."""
    rng = np.random.default_rng(12)
    for _ in range(50):
        tau = 0.55 + 1.5 * rng.uniform()
        sb = 1e-3 * rng.uniform(-1, 1, 2)
        sbar = np.array([sb[0], sb[1], -sb[0]])  # traceless
        S = 1e-4 * rng.uniform(-1, 1)
        u = 0.05 * rng.uniform(-1, 1, 2)
        f = 1e-4 * rng.uniform(-1, 1, 2)
        F = oracle_mod.forcing(tau, sbar, S, u, f)
        m0, m1, m2 = moments(F)
        k = 1.0 - 1.0 / (2.0 * tau)
        Sb = np.array([[sbar[0], sbar[1]], [sbar[1], sbar[2]]])
        want2 = k * (np.outer(u, f) + np.outer(f, u)) + k * (CS2 * np.eye(2) - np.outer(u, u)) * S - Sb / tau
        assert abs(m0 - k * S) < 1e-18
        np.testing.assert_allclose(m1, k * f, atol=1e-19)
        np.testing.assert_allclose(m2, want2, atol=1e-18)


def test_forcing_first_line_only_without_force_and_pressure(oracle_mod):
    """With f = 0 and S = 0 only the traceless-stress line of Eq. (bodyforce) remains (text below
    it): F_i has zero mass and momentum and second moment -Sbar/tau_LB."""
    sbar = np.array([2e-4, -3e-4, -2e-4])
    F = oracle_mod.forcing(0.9, sbar, 0.0, [0.01, 0.02], [0.0, 0.0])
    m0, m1, m2 = moments(F)
    assert abs(m0) < 1e-19 and np.abs(m1).max() < 1e-19
    np.testing.assert_allclose(m2, -np.array([[2e-4, -3e-4], [-3e-4, -2e-4]]) / 0.9, atol=1e-19)


def random_kappa(rng, scale):
    return scale * rng.uniform(-1, 1, 4)


def test_series_equals_independent_elimination(oracle_mod):
    """Eq. (sigtsum) summed term by term equals the direct solution of the steady equation it
    expands (sigma/tau_M - kappa sigma - sigma kappa^T = G D), where the series converges."""
    rng = np.random.default_rng(13)
    checked = 0
    for _ in range(400):
        kap = random_kappa(rng, 1e-2)
        tau_M = rng.uniform(0.1, 40.0)
        s_ser, n = oracle_mod.stress_series(kap, tau_M, 1e-3)
        if n < 0:
            continue
        s_ge = oracle_mod.stress_gauss(kap, tau_M, 1e-3)
        scale = np.abs(s_ge).max()
        assert np.abs(s_ser - s_ge).max() <= 1e-13 * scale
        checked += 1
    assert checked > 100


def test_simple_shear_closed_forms(oracle_mod):
    """Simple shear kappa_xy = gdot (Sec. III A): sigma_xy = G gdot tau_M, N1 = 2 G gdot^2 tau_M^2,
    sigma_yy = 0, G N1 / sigma_xy^2 = 2; the series stops after n = 2 (kappa^2 = 0)."""
    G = 2e-3
    for gdot in [1e-5, 3e-3, -7e-2]:
        for tau_M in [0.5, 10.0, 1e3]:
            s, n = oracle_mod.stress_series([0.0, gdot, 0.0, 0.0], tau_M, G)
            if n < 0:  # nilpotent kappa: radius 0, always summed
                pytest.fail("series refused a nilpotent kappa")
            assert n <= 3
            assert s[1] == pytest.approx(G * gdot * tau_M, rel=1e-15)
            assert s[0] - s[2] == pytest.approx(2 * G * gdot ** 2 * tau_M ** 2, rel=1e-15)
            assert s[2] == 0.0
            assert G * (s[0] - s[2]) / s[1] ** 2 == pytest.approx(2.0, rel=1e-14)


def test_planar_extension_closed_form(oracle_mod):
    """kappa_xx = -kappa_yy = edot: sigma_xx = 2 G edot tau/(1 - 2 edot tau) for edot tau < 1/2
    (Sec. III A).  Covers both the summed series and the elimination fallback."""
    G = 1e-3
    for et in [0.01, 0.2, 0.39, 0.45, 0.49]:
        tau_M = 10.0
        edot = et / tau_M
        kap = [edot, 0.0, 0.0, -edot]
        s, n = oracle_mod.stress_series(kap, tau_M, G)
        if n < 0:
            s = oracle_mod.stress_gauss(kap, tau_M, G)
        assert s[0] == pytest.approx(analytic.planar_extension_xx(edot, G, tau_M), rel=1e-13)
        assert s[1] == 0.0


def test_nlm_extension_is_bounded(oracle_mod):
    """With Eq. (nlmaxwell), II_D = (2 edot)^2 in planar extension, so 2 edot tau_M < gamma_c and
    the extensional stress stays finite for any edot (Sec. III A) -- unlike the UCM."""
    G, tau, gc = 1e-3, 1e4, 0.1
    for edot in [1e-6, 1e-3, 1.0]:
        tau_M = oracle_mod.relaxation_time(tau, gc, (2 * edot) ** 2)
        assert 2 * edot * tau_M < gc
        s, n = oracle_mod.stress_series([edot, 0.0, 0.0, -edot], tau_M, G)
        assert n > 0
        assert s[0] == pytest.approx(analytic.planar_extension_xx(edot, G, tau_M), rel=1e-13)
        assert s[0] < 2 * G * gc / (1 - gc) * 1.0000001


def test_yield_stress_limit(oracle_mod):
    """tau -> infinity: sigma -> sigma_y of Eq. (yieldstress), independent of the flow rate K."""
    G, gc = 1e-3, 0.1
    want = analytic.simple_shear_yield_stress(G, gc)
    for K in [1e-4, 1.0, 1e3]:
        tau_M = oracle_mod.relaxation_time(1e15, gc, K * K)
        s, n = oracle_mod.stress_series([0.0, K, 0.0, 0.0], tau_M, G)
        np.testing.assert_allclose(s, want, rtol=1e-9, atol=1e-18)


def test_relaxation_time_simple_shear(oracle_mod):
    """Eq. (nlmaxwell) in simple shear (II_D = gdot^2), including theta = 0 (tau_M = 0)."""
    for gdot, tau, gc in [(1e-3, 1e4, 0.1), (0.0, 5.0, 0.1), (2e-2, 3.0, math.inf)]:
        _, _, want = analytic.simple_shear(gdot, 1.0, tau, gc)
        assert oracle_mod.relaxation_time(tau, gc, gdot ** 2) == pytest.approx(want, rel=1e-15)
    assert oracle_mod.relaxation_time(0.0, 0.1, 1.0) == 0.0


def test_time_stepped_stress_fixed_point(oracle_mod):
    """Stress mode 1: repeated backward-Euler steps of Eq. (gkder) with -sigma/tau_M memory at a
    fixed kappa converge to the steady solution of Eq. (sigtsum)."""
    rng = np.random.default_rng(14)
    for _ in range(10):
        kap = random_kappa(rng, 2e-3)
        tau_M = rng.uniform(1.0, 30.0)
        s_ss, n = oracle_mod.stress_series(kap, tau_M, 1e-3)
        assert n > 0
        s = np.zeros(3)
        for _ in range(int(60 * tau_M) + 200):
            s = oracle_mod.stress_step(kap, tau_M, 1e-3, s)
        np.testing.assert_allclose(s, s_ss, rtol=1e-10, atol=1e-12 * np.abs(s_ss).max())


def test_equilibrium_offset_form(oracle_mod):
    """The offset form used by the stepping equals Eq. (neq) minus the weights."""
    rng = np.random.default_rng(15)
    for _ in range(50):
        rho = 1.0 + 0.05 * rng.uniform(-1, 1)
        u = 0.1 * rng.uniform(-1, 1, 2)
        full = oracle_mod.equilibrium(rho, u[0], u[1]) - oracle_mod.WEIGHTS
        off = oracle_mod.equilibrium_offset(rho - 1.0, u[0], u[1])
        np.testing.assert_allclose(off, full, rtol=0, atol=2e-16)


def test_time_stepped_stress_transient_simple_shear(oracle_mod):
    """Stress mode 1 from rest under steady simple shear (kappa_xy = gdot): the backward-Euler
    recursion of Eq. (gkder), (1 + 1/tau_M) s' - (kappa s' + s' kappa^T) = s + G D, decouples into
    s_yy = 0, s_xy(n) = a (s_xy(n-1) + G gdot) and s_xx(n) = a (s_xx(n-1) + 2 gdot s_xy(n)),
    a = tau_M/(tau_M + 1), solved by hand:
      s_xy(n) = Y (1 - a^n),  s_xx(n) = 2 a gdot Y [(1 - a^n)/(1 - a) - n a^n],  Y = G gdot tau_M,
    whose limits are the simple-shear sigma_xy and N1 = 2 G gdot^2 tau_M^2."""
    G = 1e-3
    for gdot, tau_M in [(1e-3, 7.0), (4e-3, 40.0), (-2e-3, 1.5)]:
        a = tau_M / (tau_M + 1.0)
        Y = G * gdot * tau_M
        s = np.zeros(3)
        for n in range(1, 400):
            s = oracle_mod.stress_step([0.0, gdot, 0.0, 0.0], tau_M, G, s)
            want_xy = Y * (1.0 - a ** n)
            want_xx = 2.0 * a * gdot * Y * ((1.0 - a ** n) / (1.0 - a) - n * a ** n)
            assert s[2] == 0.0
            assert s[1] == pytest.approx(want_xy, rel=1e-12, abs=1e-22)
            assert s[0] == pytest.approx(want_xx, rel=1e-11, abs=1e-22)


def test_time_stepped_stress_transient_planar_extension(oracle_mod):
    """Stress mode 1 from rest under planar extension (kappa = diag(e, -e)): the normal components
    relax geometrically, s_xx(n) = X (1 - bx^n) with bx = 1/(1 + 1/tau_M - 2e) and X = 2 G e tau_M /
    (1 - 2 e tau_M) (the steady planar-extension stress), s_yy likewise with -e, s_xy = 0."""
    G = 1e-3
    for e, tau_M in [(1e-3, 20.0), (-3e-3, 9.0)]:
        bx = 1.0 / (1.0 + 1.0 / tau_M - 2.0 * e)
        by = 1.0 / (1.0 + 1.0 / tau_M + 2.0 * e)
        X = 2.0 * G * e * tau_M / (1.0 - 2.0 * e * tau_M)
        Yy = -2.0 * G * e * tau_M / (1.0 + 2.0 * e * tau_M)
        s = np.zeros(3)
        for n in range(1, 300):
            s = oracle_mod.stress_step([e, 0.0, 0.0, -e], tau_M, G, s)
            assert s[0] == pytest.approx(X * (1.0 - bx ** n), rel=1e-12)
            assert s[2] == pytest.approx(Yy * (1.0 - by ** n), rel=1e-12)
            assert s[1] == 0.0
