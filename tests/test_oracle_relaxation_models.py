"""Pins of the oracle's relaxation-time extensions, which the paper leaves for further study: a
Maxwell time that depends on the local density, tau(rho) (conclusions), and a flow dependence of
tau_M that is not instantaneous but carries the history of the shear rate (Sec. III A, the
fluidity models).  The paper fixes neither form; the oracle takes
    tau(rho) = tau exp(beta_rho (rho - rho_ref) / rho_ref),
    d phi/dt = (phi_ss - phi) / tau_f,  phi = 1/tau_M,  phi_ss = 1/tau + II_D^{1/2}/gamma_c
(Eq. nlmaxwell is phi = phi_ss), the latter stepped by backward Euler.

What fixes them: planar Couette flow imposes the shear rate u_wall/H kinematically, so the steady
stress must be the simple-shear closed form of Sec. III A at whatever tau the model gives; the
memory must not change any steady state; the backward-Euler recursion of the memory has a closed
form under a constant shear rate; and a long memory produces the stress overshoot of start-up
shear that distinguishes the fluidity models from the instantaneous one.
"""
import math

import numpy as np
import pytest

from oracle import analytic
from paper_1310_7450_gb300 import inputs

NY, UW, G, THETA = 16, 0.01, 1e-3, 10.0


def couette_params(**kw):
    p = dict(inputs.matched_params(0.9, THETA, 0.1, G, 0.0), top_wall="moving", u_wall=UW)
    p.update(kw)
    return p


def test_fluidity_step_recursion_closed_form(oracle_mod):
    """Under a constant phi_ss the recursion phi_{n+1} = (tau_f phi_n + phi_ss)/(tau_f + 1) has the
    solution phi_n = phi_ss + (phi_0 - phi_ss) q^n, q = tau_f/(tau_f + 1); tau_f = 0 is Eq. (nlmaxwell)
    itself, and a state without a stored fluidity (0) starts from phi_ss."""
    phi0, phi_ss, tau_f = 1.0 / 121.0, 0.05, 37.5
    q = tau_f / (tau_f + 1.0)
    phi = phi0
    for n in range(1, 200):
        phi = oracle_mod.fluidity_step(phi, phi_ss, tau_f)
        assert phi == pytest.approx(phi_ss + (phi0 - phi_ss) * q ** n, rel=1e-13)
    assert oracle_mod.fluidity_step(phi0, phi_ss, 0.0) == phi_ss
    assert oracle_mod.fluidity_step(0.0, phi_ss, tau_f) == phi_ss


def test_defaults_leave_the_paper_model_unchanged(oracle_mod):
    """beta_rho = 0 and tau_f = 0 given explicitly reproduce the default run bitwise."""
    rng = np.random.default_rng(8)
    p = inputs.matched_params(0.9, 10.0, 0.1, 1e-3, 1e-5)
    a = oracle_mod.init_state(1.0 + 1e-3 * rng.uniform(-1, 1, (9, 5)))
    b = a.copy()
    oracle_mod.run(p, a, 300)
    oracle_mod.run(dict(p, beta_rho=0.0, rho_ref=1.3, tau_f=0.0), b, 300)
    assert np.array_equal(a.dev, b.dev) and np.array_equal(a.drho, b.drho)


@pytest.mark.parametrize("beta", [5.0, -8.0])
def test_density_dependent_tau_in_homogeneous_shear(oracle_mod, beta):
    """Couette flow at the uniform density 1.02 with rho_ref = 1: the steady stress equals the
    simple-shear closed form with tau exp(0.02 beta) everywhere (1e-12), and not the one with tau
    (the difference is several percent)."""
    p = couette_params(beta_rho=beta, rho_ref=1.0)
    st = oracle_mod.init_state(np.full((NY, 2), 1.02))
    oracle_mod.run(p, st, 50000)
    _, s, rho = oracle_mod.fields(p, st)
    assert np.ptp(rho) <= 1e-13 and abs(rho.mean() - 1.02) <= 1e-12
    H = NY - 0.5
    tau = THETA * p["tau0"]
    sxy, n1, _ = analytic.simple_shear(UW / H, G, tau * math.exp(0.02 * beta), 0.1)
    assert np.abs(s[..., 3] / sxy - 1).max() <= 1e-12
    assert np.abs((s[..., 0] - s[..., 1]) / n1 - 1).max() <= 1e-12
    plain, _, _ = analytic.simple_shear(UW / H, G, tau, 0.1)
    assert abs(s[NY // 2, 0, 3] / plain - 1) > 0.02


def startup_history(oracle_mod, tau_f, chunks=100, every=500):
    p = couette_params(tau_f=tau_f, stress_mode=1)
    st = oracle_mod.init_state(np.ones((NY, 2)))
    hist = []
    for _ in range(chunks):
        oracle_mod.run(p, st, every)
        hist.append(oracle_mod.fields(p, st)[1][NY // 2, 0, 3])
    return p, st, np.array(hist)


def test_fluidity_memory_keeps_the_steady_state_and_adds_start_up_overshoot(oracle_mod):
    """Start-up of Couette flow with the time-stepped stress (the integral model's differential
    form): with tau_f = 500 the steady stress is the closed form of the instantaneous model
    (1e-12); with the long memory tau_f = 3000 the fluidity lags behind the shear rate, tau_M stays
    long while the stress builds up, and the mid-gap shear stress overshoots its steady value by
    more than 10 % (measured 13.6 %), against less than 1 % without memory (0.8 %)."""
    H = NY - 0.5
    p, st, _ = startup_history(oracle_mod, 500.0)
    s = oracle_mod.fields(p, st)[1]
    sxy, _, _ = analytic.simple_shear(UW / H, G, THETA * p["tau0"], 0.1)
    assert np.abs(s[..., 3] / sxy - 1).max() <= 1e-12
    assert np.all(st.phi > 0)
    _, _, long_mem = startup_history(oracle_mod, 3000.0)
    _, _, no_mem = startup_history(oracle_mod, 0.0)
    assert long_mem.max() / sxy > 1.10
    assert no_mem.max() / sxy < 1.01
    assert abs(long_mem[-1] / sxy - 1) < 1e-3       # it relaxes back to the steady value


def test_relaxation_extensions_reject_bad_parameters(oracle_mod):
    p = couette_params()
    st = oracle_mod.init_state(np.ones((NY, 2)))
    for bad in (dict(p, tau_f=-1.0), dict(p, rho_ref=0.0), dict(p, scheme="generalized_newtonian", top_wall="bounce_back", tau_f=10.0)):
        with pytest.raises(ValueError):
            oracle_mod.run(bad, st, 1)
