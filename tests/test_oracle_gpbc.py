"""Pins of the oracle's pressure-driven channel: the generalized periodic boundaries of Sec. II B
(Kim and Pitsch), with no body force, no flow-induced density and the first line of
Eq. (bodyforce) only.

* brute force: the NumPy twin builds the crossing populations in push form from the node they
  leave; the C oracle in pull form from the node they come from;
* the Newtonian steady state: the column-mean densities lie on the straight line between the
  imposed inlet and outlet densities, the mass flux is the same through every column, and the
  velocity is the body-force Poiseuille profile up to the weakly compressible terms;
* the statement of Sec. II B that pressure-driven (GPBC) and body-force-driven channels reach the
  same steady state: they do, up to the dynamic-pressure term of the lattice's momentum flux.  With
  rho u_x fixed along x, d_x(rho u_x^2) = -u_x^2 d_x rho, so a pressure gradient drives with
  (1 - 3 u_x^2) g where a body force drives with g: the gap is O(u_max^2) and falls 4x when
  u_max halves;
* the flow-induced pressure (Sec. IV, lower panel of the stress figure): higher inside the plug
  than at the walls, mirror symmetric.
"""
import numpy as np
import pytest

from oracle import analytic, bruteforce
from paper_1310_7450_gb300 import inputs


def gpbc(p):
    return dict(p, x_mode="gpbc")


def linear_start(oracle_mod, p, nx, ny):
    rin, rout = oracle_mod.gpbc_densities(p, nx)
    return oracle_mod.init_state(inputs.linear_density(nx, ny, rin, rout))


def nlm_channel(ny, theta, umax, wpH=0.5):
    v0 = analytic.v_of_d(0.0, wpH, theta, 0.1)
    tau0 = (ny / 2.0) * v0 / umax
    return inputs.yield_stress_channel(ny, theta=theta, tau=theta * tau0, wpH=wpH)


def two_step_average(oracle_mod, p, st):
    """Fields averaged over two consecutive steps: the boundary excites a staggered mode that
    alternates sign every step and every column (period 2 in t and x) and decays slowly; the
    average removes it."""
    u0, s0, r0 = oracle_mod.fields(p, st)
    oracle_mod.run(p, st, 1)
    u1, s1, r1 = oracle_mod.fields(p, st)
    return 0.5 * (u0 + u1), 0.5 * (s0 + s1), 0.5 * (r0 + r1)


@pytest.mark.parametrize("nx,ny", [(1, 3), (3, 5), (4, 8)])
def test_gpbc_bruteforce_twin(oracle_mod, nx, ny):
    """Random non-uniform states, 50 steps, a pressure drop large enough to matter (g = 1e-4):
    the C oracle (pull) and the NumPy twin (push) agree."""
    rng = np.random.default_rng(7 + nx * ny)
    p = gpbc(inputs.matched_params(0.9, 10.0, 0.1, 1e-3, 1e-4))
    rho = 1.0 + 1e-2 * rng.uniform(-1, 1, (ny, nx))
    st = oracle_mod.flow_state(rho, 1e-2 * rng.uniform(-1, 1, (ny, nx)), 1e-2 * rng.uniform(-1, 1, (ny, nx)), 0.0)
    n0, d0 = st.nstar.copy(), st.drho.copy()
    oracle_mod.run(p, st, 50)
    nb, db = bruteforce.run(p, n0, d0, 50)
    assert np.abs(st.nstar - n0).max() > 1e-4          # the state moved
    assert np.abs(nb - st.nstar).max() <= 1e-13 * np.abs(st.nstar).max()
    assert np.all(st.drho == 0.0) and np.all(db == 0.0)
    fl = bruteforce.fields(p, nb, db)
    u, s, r = oracle_mod.fields(p, st)
    assert np.abs(fl["u"] - u).max() <= 1e-11 * np.abs(u).max()
    assert np.abs(fl["sigma"][..., 0, 1] - s[..., 3]).max() <= 1e-10 * np.abs(s[..., 3]).max()
    assert np.abs(fl["rho"] - r).max() <= 1e-14


def test_gpbc_newtonian_steady_state(oracle_mod):
    nx, ny, g = 4, 16, 1e-6
    p = gpbc(inputs.matched_params(0.9, 0.0, 0.1, 1e-3, g))
    st = linear_start(oracle_mod, p, nx, ny)
    oracle_mod.run(p, st, 40000)   # slowest mode exp(-pi^2 nu t / (4 H^2)) = exp(-5.1e-3 t)
    u, _, rho = two_step_average(oracle_mod, p, st)
    rin, rout = oracle_mod.gpbc_densities(p, nx)
    line = rin + (rout - rin) * (np.arange(nx) + 1.0) / (nx + 1.0)
    assert np.abs(rho.mean(axis=0) - line).max() <= 1e-12
    flux = (rho * u[..., 0]).sum(axis=0)
    assert np.abs(flux - flux.mean()).max() <= 1e-9 * flux.mean()
    # body-force run of the same g
    pb = dict(p, x_mode="periodic")
    sb = oracle_mod.init_state(np.ones((ny, nx)))
    oracle_mod.run(pb, sb, 40000)
    ub, _, _ = oracle_mod.fields(pb, sb)
    umax = ub[..., 0].max()
    bound = 3 * umax ** 2 + 3 * (rin - rout)   # dynamic pressure + density variation along x
    assert np.abs(u - ub).max() <= bound * umax
    nu = inputs.nu_lb(0.9)
    d2 = u[2:, :, 0] - 2 * u[1:-1, :, 0] + u[:-2, :, 0]
    assert np.abs(d2 / (-g / nu) - 1.0).max() <= bound


def test_gpbc_nlm_matches_body_force_up_to_mach_squared(oracle_mod):
    """Yield-stress channel (theta = 10, gamma_c = 0.1, wp H = 1/2), steady states from the
    closed-form start: the GPBC and body-force states differ by at most 6 u_max^2, and halving
    u_max divides the gap by about 4."""
    nx, ny = 2, 8
    gaps = []
    for umax in (0.01, 0.005):
        pb = nlm_channel(ny, 10.0, umax)
        ua = analytic.channel_profile(ny, pb["g_x"], pb["G_inf"], pb["tau0"], pb["theta"], pb["gamma_c"])
        sb = oracle_mod.flow_state(np.ones((ny, nx)), np.repeat(ua[:, None], nx, 1), np.zeros((ny, nx)), pb["g_x"])
        oracle_mod.run(pb, sb, 200000)
        ub, sgb, _ = oracle_mod.fields(pb, sb)
        pg = gpbc(pb)
        rin, rout = oracle_mod.gpbc_densities(pg, nx)
        sg = oracle_mod.flow_state(inputs.linear_density(nx, ny, rin, rout), np.repeat(ua[:, None], nx, 1),
                                   np.zeros((ny, nx)), 0.0)
        oracle_mod.run(pg, sg, 200000)
        ug, sgg, _ = two_step_average(oracle_mod, pg, sg)
        gap_u = np.abs(ug - ub).max() / np.abs(ub).max()
        gap_s = np.abs(sgg[..., 3] - sgb[..., 3]).max() / np.abs(sgb[..., 3]).max()
        n1g, n1b = sgg[..., 0] - sgg[..., 1], sgb[..., 0] - sgb[..., 1]
        gap_n = np.abs(n1g - n1b).max() / np.abs(n1b).max()
        assert max(gap_u, gap_s, gap_n) <= 6 * umax ** 2
        gaps.append(gap_u)
    assert 2.5 <= gaps[0] / gaps[1] <= 5.5


def test_gpbc_flow_induced_pressure_peaks_in_the_plug(oracle_mod):
    """Without the density correction the lattice density carries the normal-stress pressure:
    in a unidirectional flow the transverse momentum balance is c_s^2 d_y rho = d_y Sbar_yy with
    Sbar_yy = -N1/2 (sigma_yy = 0, D_xx = D_yy = 0), so rho + (3/2) N1 is constant across the
    channel and the pressure is highest in the plug, where N1 is smallest (Sec. IV)."""
    nx, ny = 2, 16
    p = gpbc(nlm_channel(ny, 100.0, 0.01))
    ua = analytic.channel_profile(ny, p["g_x"], p["G_inf"], p["tau0"], p["theta"], p["gamma_c"])
    rin, rout = oracle_mod.gpbc_densities(p, nx)
    st = oracle_mod.flow_state(inputs.linear_density(nx, ny, rin, rout), np.repeat(ua[:, None], nx, 1),
                               np.zeros((ny, nx)), 0.0)
    oracle_mod.run(p, st, 100000)
    _, s, rho = two_step_average(oracle_mod, p, st)
    prof = rho[:, 0] - rho[:, 0].mean()
    n1 = s[:, 0, 0] - s[:, 0, 1]
    assert np.abs(prof - prof[::-1]).max() <= 1e-6 * np.abs(prof).max()
    assert prof[ny // 2] > 0 > prof[0]
    assert np.argmax(prof) in (ny // 2 - 1, ny // 2)
    balance = prof + 1.5 * n1
    assert np.ptp(balance) <= 0.05 * np.ptp(1.5 * n1)
