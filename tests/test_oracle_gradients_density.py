"""Direct pins of two oracle parts that the whole-step tests only reach indirectly (CPU).

1. The three-point velocity gradients of Sec. II C (second-order finite differences): central in
   the interior and along periodic x, one-sided at the first and last fluid rows.  A three-point
   stencil is exact on a quadratic, so a velocity field that is quadratic in y (plus a periodic
   profile in x, where the central difference has a known exact value) must give every kappa
   component exactly on every row, the wall rows included.  The field is planted in the
   post-streaming populations by inverting the pull-streaming with bounce-back (a bijection), so
   the gradient velocity j/R0 the oracle differentiates is exactly the chosen one.

2. The flow-induced density of Eq. (rhoplus): in a steady body-force channel the scheme must let
   the pressure build up against the normal stresses.  The y-momentum balance fixes the lattice
   density rho_eq (which carries the pressure) to const - (3/2) N1 (the traceless stress enters
   through the second moment of Eq. bodyforce), and delta rho = -tr Sigma^nN / (c_s^2 d) makes the
   hydrodynamic density rho_eq - delta rho uniform across the channel.  A delta rho with a wrong
   factor or sign leaves a spread of order N1 in the hydrodynamic density.
"""
import numpy as np
import pytest

from oracle import analytic
from paper_1310_7450_gb300 import inputs

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])


def unstream(n_post: np.ndarray) -> np.ndarray:
    """Post-collision populations n*[9, ny, nx] whose pull-streaming with half-way bounce-back
    (walls beyond rows 0 and ny-1, periodic x) gives n_post: n_i(r) = n*_i(r - c_i) where the
    source is a fluid row, else n_i(r) = n*_opp(i)(r).  Every n*_j(s) is used exactly once."""
    _, ny, nx = n_post.shape
    nstar = np.full_like(n_post, np.nan)
    for i in range(9):
        for y in range(ny):
            for x in range(nx):
                ys = y - CY[i]
                if 0 <= ys < ny:
                    nstar[i, ys, (x - CX[i]) % nx] = n_post[i, y, x]
                else:
                    nstar[OPP[i], y, x] = n_post[i, y, x]
    assert not np.isnan(nstar).any()
    return nstar


def test_unstream_is_the_inverse_of_the_oracle_streaming(oracle_mod):
    """The helper itself: a random post-streaming field, unstreamed, then streamed by the oracle
    (its first step's moments), gives back the field's own zeroth moment everywhere."""
    rng = np.random.default_rng(4)
    nx, ny = 5, 6
    n_post = (oracle_mod.WEIGHTS[:, None, None] * (1.0 + 1e-3 * rng.uniform(-1, 1, (9, ny, nx))))
    st = oracle_mod.state_from_populations(unstream(n_post), np.zeros((ny, nx)))
    # theta = 0 with tau_LB matched to eta_inf: sigma = 0 and Sigma^nN = 0, so S = 0
    p = inputs.matched_params(0.9, 0.0, 0.1, 1e-3, 0.0)
    rho_eq = oracle_mod.intermediates(p, st)[..., 7]   # R0 + S/2
    np.testing.assert_allclose(rho_eq, n_post.sum(axis=0), rtol=0, atol=1e-14)


def velocity_field(nx, ny):
    """u_x = a0 + a1 y + a2 y^2 + b sin(k x), u_y = c0 + c1 y + c2 y^2 + e cos(k x), k = 2 pi/nx,
    and the exact three-point differences of it: kappa_ab = d_b u_a."""
    a0, a1, a2, b = 1.0e-3, 2.0e-4, -3.0e-5, 5.0e-4
    c0, c1, c2, e = -2.0e-4, 1.0e-4, 4.0e-5, 3.0e-4
    k = 2 * np.pi / nx
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    x = np.arange(nx, dtype=np.float64)[None, :] * np.ones((ny, 1))
    ux = a0 + a1 * y + a2 * y * y + b * np.sin(k * x)
    uy = c0 + c1 * y + c2 * y * y + e * np.cos(k * x)
    kap = np.zeros((ny, nx, 4))
    kap[..., 0] = b * np.cos(k * x) * np.sin(k)       # (u(x+1) - u(x-1))/2 of b sin(kx)
    kap[..., 1] = a1 + 2 * a2 * y                      # exact for a quadratic, every row
    kap[..., 2] = -e * np.sin(k * x) * np.sin(k)
    kap[..., 3] = c1 + 2 * c2 * y
    return ux, uy, kap


@pytest.mark.parametrize("nx,ny", [(8, 7), (3, 3), (6, 12)])
def test_three_point_gradients_exact_on_quadratic_profile(oracle_mod, nx, ny):
    """kappa_xx, kappa_xy, kappa_yx, kappa_yy of the oracle equal the exact three-point values on
    every row, including the one-sided wall rows 0 and ny-1 (Sec. II C, second-order stencils)."""
    ux, uy, kap = velocity_field(nx, ny)
    # planted as offsets n - w (w_opp(i) = w_i, so the offsets permute like the populations)
    dev_post = np.zeros((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            dev_post[:, y, x] = oracle_mod.equilibrium_offset(0.0, ux[y, x], uy[y, x])
    st = oracle_mod.State(unstream(dev_post), np.zeros((ny, nx)), np.zeros((3, ny, nx)))
    # no body force (j = sum c n), no stress: the gradient velocity is j / R0 = u
    p = dict(tau_lb=0.9, g_x=0.0, G_inf=0.0, tau0=0.0, theta=0.0, gamma_c=np.inf, rho0=1.0,
             stress_mode=0)
    got = oracle_mod.intermediates(p, st)[..., :4]
    for c in range(4):
        scale = np.abs(kap[..., c]).max()
        assert np.abs(got[..., c] - kap[..., c]).max() <= 1e-13 * scale, f"kappa component {c}"
    # the wall rows are where a one-sided stencil with a wrong sign or factor would show
    assert np.abs(got[[0, -1], :, 1] - kap[[0, -1], :, 1]).max() <= 1e-13 * np.abs(kap[..., 1]).max()


def nlm_channel(ny, theta, umax=0.05, wpH=0.5):
    v0 = analytic.v_of_d(0.0, wpH, theta, 0.1)
    tau0 = (ny / 2.0) * v0 / umax
    return inputs.yield_stress_channel(ny, theta=theta, tau=theta * tau0, wpH=wpH)


@pytest.mark.parametrize("theta", [10.0, 100.0])
def test_flow_induced_density_counters_normal_stress(oracle_mod, theta):
    """Eq. (rhoplus) in a steady body-force nlM channel (Ny = 32, from the closed-form profile):
    the hydrodynamic density rho_eq - delta rho is uniform across the channel, while the lattice
    density rho_eq carries the normal-stress pressure, rho_eq + (3/2) N1 = const.  Both to 1e-3 of
    the spread of (3/2) N1."""
    ny = 32
    p = nlm_channel(ny, theta)
    ua = analytic.channel_profile(ny, p["g_x"], p["G_inf"], p["tau0"], p["theta"], p["gamma_c"])
    st = oracle_mod.flow_state(np.ones((ny, 1)), ua[:, None], np.zeros((ny, 1)), p["g_x"])
    st, r = oracle_mod.run_to_steady(p, st, 1e-11, check_every=1000, max_steps=2_000_000)
    assert r <= 1e-11
    _, s, rho_h = oracle_mod.fields(p, st)
    rho_eq = oracle_mod.intermediates(p, st)[:, 0, 7]
    N1 = s[:, 0, 0] - s[:, 0, 1]
    spread = np.ptp(1.5 * N1)
    assert spread > 1e-8                              # normal stresses are present
    assert np.abs(s[:, 0, 1]).max() <= 1e-6 * spread   # sigma_yy = 0 in simple shear (to rounding)
    assert np.ptp(rho_h[:, 0]) <= 1e-3 * spread
    assert np.ptp(rho_eq + 1.5 * N1) <= 1e-3 * spread
    assert np.ptp(rho_eq) >= 0.99 * spread            # the pressure varies across the channel
