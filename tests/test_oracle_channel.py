"""Whole-step pins of the oracle (CPU) against what the paper and mathematics fix.

Newtonian limit: the discrete steady profile and the start-up series; non-Newtonian: the
analytic steady channel solution Eq. (maxwellpoiseuille) with second-order grid convergence,
the linear shear-stress law and N1; invariants: mass, mirror symmetry, x-invariance; the
Newtonian cross-check of the forcing term (text below Eq. bodyforce); and agreement with the
independently written NumPy twin on tiny grids.
"""
import numpy as np
import pytest

from oracle import analytic, bruteforce
from paper_1310_7450_gb300 import inputs

NU = inputs.nu_lb(0.9)


def newtonian(g=1e-6):
    return inputs.matched_params(0.9, 0.0, 0.1, 1e-3, g)


def nlm_channel(ny, theta, umax=0.05, wpH=0.5):
    """theta, gamma_c = 0.1, wp H given; tau0 chosen so that the analytic peak speed is umax."""
    v0 = analytic.v_of_d(0.0, wpH, theta, 0.1)
    tau0 = (ny / 2.0) * v0 / umax
    return inputs.yield_stress_channel(ny, theta=theta, tau=theta * tau0, wpH=wpH)


def analytic_profile(ny, p):
    return analytic.channel_profile(ny, p["g_x"], p["G_inf"], p["tau0"], p["theta"], p["gamma_c"])


def test_newtonian_steady_is_discrete_parabola(oracle_mod):
    """theta = 0: Sigma^nN = 0 and the scheme is BGK with the forcing of Eq. (bodyforce).  The
    steady interior second difference equals -g/nu exactly (up to rounding); the profile is
    mirror symmetric and within 1e-4 of g/(2nu)(H^2 - y^2) (the bounce-back wall slip)."""
    ny = 64
    p = newtonian()
    st = oracle_mod.init_state(np.ones((ny, 1)))
    # slowest mode decays as exp(-pi^2 nu t / (4 H^2)) ~ exp(-3.2e-4 t): 1.5e5 steps -> 1e-21
    oracle_mod.run(p, st, 150000)
    u, _, _ = oracle_mod.fields(p, st)
    ux = u[:, 0, 0]
    d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
    np.testing.assert_allclose(d2, -p["g_x"] / NU, rtol=1e-8)
    assert np.abs(ux - ux[::-1]).max() <= 1e-13 * ux.max()
    par = analytic.newtonian_parabola(ny, p["g_x"], NU)
    assert np.abs(ux - par).max() <= 1e-4 * par.max()
    # u_y is a rounding-level checkerboard (about 1e-11 u_max), not a flow
    assert np.abs(u[:, 0, 1]).max() <= 1e-10 * ux.max()


def test_newtonian_startup_series(oracle_mod):
    """Start-up from rest follows the Fourier series of the diffusion problem (Newtonian case of
    Sec. IV B).  The state after k steps carries k + 1/2 force impulses (j = sum c n + f/2)."""
    ny = 64
    p = newtonian()
    st = oracle_mod.init_state(np.ones((ny, 4)))
    umax = analytic.newtonian_parabola(ny, p["g_x"], NU).max()
    for T in [500, 3000, 12000]:
        oracle_mod.run(p, st, T - st.step)
        u, _, _ = oracle_mod.fields(p, st)
        ser = analytic.newtonian_startup(ny, p["g_x"], NU, T + 0.5)
        assert np.abs(u[:, :, 0] - ser[:, None]).max() <= 1e-4 * umax


@pytest.mark.parametrize("ny,bound", [(32, 0.015), (64, 0.004)])
def test_nlm_steady_profile_matches_analytic(oracle_mod, ny, bound):
    """Steady nlM channel (theta = 10, gamma_c = 0.1, wp H = 1/2) against Eq. (maxwellpoiseuille)
    integrated to v(1) = 0.  The bound shrinks 4x per grid doubling (second order)."""
    p = nlm_channel(ny, 10.0)
    ua = analytic_profile(ny, p)
    st = oracle_mod.flow_state(np.ones((ny, 1)), ua[:, None], np.zeros((ny, 1)), p["g_x"])
    st, r = oracle_mod.run_to_steady(p, st, 1e-10, check_every=1000, max_steps=600000)
    assert r <= 1e-10
    u, s, _ = oracle_mod.fields(p, st)
    err = np.abs(u[:, 0, 0] - ua).max() / ua.max()
    assert err < bound
    # total shear stress Sigma_xy = sigma_xy + eta_inf kappa_xy obeys the linear law -g (y - y_c)
    kxy = oracle_mod.intermediates(p, st)[:, 0, 1]
    Sxy = s[:, 0, 3] + p["G_inf"] * p["tau0"] * kxy
    lin = -p["g_x"] * (np.arange(ny) - (ny - 1) / 2.0)
    assert np.abs(Sxy - lin).max() <= 3.3 * bound * np.abs(lin).max()
    # N1 = 2 G gdot^2 tau_M^2 with the analytic shear rate (Sec. III B, below Eq. plug)
    gd = analytic.channel_shear_rate(ny, p["g_x"], p["G_inf"], p["tau0"], p["theta"], p["gamma_c"])
    N1a = np.array([analytic.simple_shear(x, p["G_inf"], p["theta"] * p["tau0"], 0.1)[1] for x in gd])
    N1 = s[:, 0, 0] - s[:, 0, 1]
    assert np.abs(N1 - N1a).max() <= 10 * bound * N1a.max()
    # u_y = 0 and only kappa_xy nonzero in the x-invariant channel (Sec. IV A, kappa figure)
    assert np.abs(u[:, 0, 1]).max() <= 1e-10 * ua.max()


def test_nlm_below_yield_is_newtonian_at_low_shear_viscosity(oracle_mod):
    """wp H < gamma_c: no yielding anywhere; d v/d d = -wp H d/(1+theta) + O(wp^2) (Sec. III B),
    i.e. the parabola of the low-shear viscosity G (tau + tau0) = nu_LB."""
    ny = 32
    p = nlm_channel(ny, 10.0, umax=0.01, wpH=0.001)
    par = analytic.newtonian_parabola(ny, p["g_x"], NU)
    st = oracle_mod.flow_state(np.ones((ny, 1)), par[:, None], np.zeros((ny, 1)), p["g_x"])
    st, r = oracle_mod.run_to_steady(p, st, 1e-10, check_every=1000, max_steps=400000)
    u, _, _ = oracle_mod.fields(p, st)
    ua = analytic_profile(ny, p)
    assert np.abs(u[:, 0, 0] - ua).max() <= 2e-3 * ua.max()
    # ... and both approach the low-shear parabola (relative O(theta tau gdot / gamma_c) ~ 1e-2)
    assert np.abs(ua - par).max() <= 0.015 * par.max()
    assert np.abs(u[:, 0, 0] - par).max() <= 0.015 * par.max()


def test_newtonian_equivalence_of_stress_forcing(oracle_mod):
    """Cross-check below Eq. (bodyforce): a Newtonian Sigma^nN = Delta eta D added through F_i acts
    like BGK with eta + Delta eta.  Here theta = 0 and eta_inf = G tau0 = 0.1 nu_LB, so
    Sigma^nN = -0.9 nu_LB D and the steady profile is the parabola of 0.1 nu_LB."""
    ny = 20
    frac = 0.1
    g = 1e-7
    p = dict(tau_lb=0.9, g_x=g, G_inf=1e-3, tau0=frac * NU / 1e-3, theta=0.0, gamma_c=0.1,
             rho0=1.0, stress_mode=0)
    par = analytic.newtonian_parabola(ny, g, frac * NU)
    st = oracle_mod.flow_state(np.ones((ny, 1)), par[:, None], np.zeros((ny, 1)), g)
    st, r = oracle_mod.run_to_steady(p, st, 1e-10, check_every=1000, max_steps=600000)
    u, _, _ = oracle_mod.fields(p, st)
    assert np.abs(u[:, 0, 0] - par).max() <= 4e-3 * par.max()
    # the sign matters: the same stress with the opposite sign would give 1.9 nu_LB
    assert u[:, 0, 0].max() > 5 * analytic.newtonian_parabola(ny, g, NU).max()


def random_state(oracle_mod, nx, ny, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    st = oracle_mod.init_state(1.0 + amp * rng.uniform(-1, 1, (ny, nx)))
    w = oracle_mod.equilibrium(1.0, 0.0, 0.0)
    st.dev += amp * rng.uniform(-1, 1, st.dev.shape) * w[:, None, None]
    st.drho[:] = 1e-2 * amp * rng.uniform(-1, 1, (ny, nx))
    return st


def test_mass_invariant(oracle_mod):
    """sum_r (sum_i n*_i - delta rho) is conserved: the collision adds exactly S per node
    (zeroth-moment condition below Eq. lbfab), streaming and bounce-back conserve."""
    nx, ny = 5, 7
    p = inputs.matched_params(0.9, 10.0, 0.1, 1e-3, 1e-5)
    st = random_state(oracle_mod, nx, ny, 21)
    m0 = oracle_mod.mass(st)
    for _ in range(5):
        oracle_mod.run(p, st, 60)
        assert abs(oracle_mod.mass(st) - m0) <= 1e-13 * nx * ny
    assert np.abs(st.drho).max() > 0  # flow-induced density is active


def test_mirror_symmetry_and_x_invariance(oracle_mod):
    """A mirror-symmetric, x-invariant state stays so: u_x(y) = u_x(Ny-1-y), sigma_xy odd, N1 even
    (Sec. III B symmetry), every column bitwise identical, u_y = 0 to rounding."""
    nx, ny = 4, 24
    p = nlm_channel(ny, 10.0)
    st = oracle_mod.init_state(np.ones((ny, nx)))
    oracle_mod.run(p, st, 3000)
    u, s, rho = oracle_mod.fields(p, st)
    for x in range(1, nx):
        assert np.array_equal(u[:, x], u[:, 0]) and np.array_equal(s[:, x], s[:, 0])
    ux = u[:, 0, 0]
    assert np.abs(ux - ux[::-1]).max() <= 1e-13 * np.abs(ux).max()
    sxy = s[:, 0, 3]
    assert np.abs(sxy + sxy[::-1]).max() <= 1e-11 * np.abs(sxy).max()
    n1 = s[:, 0, 0] - s[:, 0, 1]
    assert np.abs(n1 - n1[::-1]).max() <= 1e-11 * np.abs(n1).max()
    assert np.abs(u[:, :, 1]).max() <= 1e-10 * np.abs(ux).max()


def test_threads_do_not_change_the_result(oracle_mod):
    """The oracle's OpenMP split over rows (used for the timed CPU baseline) updates every node from
    the same inputs in the same order of operations: 1, 3 and 8 threads give bitwise equal states."""
    nx, ny = 9, 23
    p = inputs.matched_params(0.9, 10.0, 0.1, 1e-3, 1e-5)
    out = []
    for nt in (1, 3, 8):
        st = random_state(oracle_mod, nx, ny, 33)
        oracle_mod.run(p, st, 40, nthreads=nt)
        out.append((st.dev.copy(), st.drho.copy()))
    for dev, drho in out[1:]:
        assert np.array_equal(dev, out[0][0]) and np.array_equal(drho, out[0][1])


@pytest.mark.parametrize("ny", [3, 4, 5, 8])
def test_bruteforce_twin_tiny_grids(oracle_mod, ny):
    """The independently written NumPy twin (push streaming, 4x4 Kronecker stress solve) agrees
    with the C oracle on random non-uniform states for 50 steps."""
    nx = 4
    p = inputs.matched_params(0.9, 10.0, 0.1, 1e-3, 1e-5)
    st = random_state(oracle_mod, nx, ny, 100 + ny, amp=1e-2)
    n0, d0 = st.nstar.copy(), st.drho.copy()
    oracle_mod.run(p, st, 50)
    nb, db = bruteforce.run(p, n0, d0, 50)
    assert np.abs(nb - st.nstar).max() <= 1e-13 * np.abs(st.nstar).max()
    # delta rho = -(3/2) tr(sigma - G tau D) cancels ~3 digits, hence the looser bound
    assert np.abs(db - st.drho).max() <= 1e-11 * np.abs(st.drho).max()
    fl = bruteforce.fields(p, nb, db)
    u, s, rho = oracle_mod.fields(p, st)
    assert np.abs(fl["u"] - u).max() <= 1e-11 * np.abs(u).max()
    assert np.abs(fl["sigma"][..., 0, 1] - s[..., 3]).max() <= 1e-10 * np.abs(s[..., 3]).max()
    assert np.abs(fl["rho"] - rho).max() <= 1e-14


def test_time_stepped_mode_reaches_same_steady_state(oracle_mod):
    """Stress mode 1 (backward Euler of Eq. gkder) has the steady state of Eq. (sigtsum): started
    from the converged mode-0 channel it stays there."""
    ny = 16
    p = nlm_channel(ny, 10.0)
    ua = analytic_profile(ny, p)
    st = oracle_mod.flow_state(np.ones((ny, 1)), ua[:, None], np.zeros((ny, 1)), p["g_x"])
    st, _ = oracle_mod.run_to_steady(p, st, 1e-11, check_every=1000, max_steps=300000)
    u0, s0, _ = oracle_mod.fields(p, st)
    pb = dict(p, stress_mode=1)
    stb = st.copy()
    stb.sig[0], stb.sig[1], stb.sig[2] = s0[:, :, 0], s0[:, :, 3], s0[:, :, 1]
    oracle_mod.run(pb, stb, 20000)
    ub, sb, _ = oracle_mod.fields(pb, stb)
    # (the mode-0 state is converged to r ~ 1e-11, i.e. to ~1e-8 of its own fixed point)
    assert np.abs(ub - u0).max() <= 1e-7 * np.abs(u0).max()
    assert np.abs(sb - s0).max() <= 1e-7 * np.abs(s0).max()


def test_rejects_bad_grid(oracle_mod):
    p = newtonian()
    st = oracle_mod.init_state(np.ones((2, 4)))
    with pytest.raises(ValueError):
        oracle_mod.run(p, st, 1)
