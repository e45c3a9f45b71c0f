"""Pins of the oracle's planar Couette flow (Sec. IV C): the bottom wall is the half-way
bounce-back wall at y = -1/2, the last row y = ny-1 lies on a wall moving with (u_wall, 0) whose
incoming populations follow Zou and He, so the gap is H = ny - 1/2.

* brute force: the NumPy twin solves the Zou-He conditions as a 4x4 linear system per node;
* Newtonian limit: the steady profile is exactly linear, and the start-up from rest follows the
  Fourier series of the diffusion problem with one moving wall with an error that falls as H^-2;
* nlM: the steady flow is homogeneous simple shear at gdot = u_wall / H (the total shear stress
  sigma(gdot) + eta_inf gdot is uniform and increasing in gdot), so sigma_xy and N1 equal the
  closed forms of Sec. III A everywhere.
"""
import math

import numpy as np
import pytest

from oracle import analytic, bruteforce
from paper_1310_7450_gb300 import inputs

NU = inputs.nu_lb(0.9)


def couette(p, u_wall):
    return dict(p, top_wall="moving", u_wall=u_wall)


def startup_series(ny, u_wall, nu, t, nterms=4000):
    """u(y', t) = u_w y'/H + sum_n 2 u_w (-1)^n/(n pi) sin(n pi y'/H) exp(-nu (n pi/H)^2 t), y' = y + 1/2:
    the diffusion equation with u(0) = 0, u(H) = u_w and u(y', 0) = 0."""
    H = ny - 0.5
    yy = np.arange(ny) + 0.5
    u = u_wall * yy / H
    for n in range(1, nterms):
        u = u + 2 * u_wall * (-1) ** n / (n * math.pi) * np.sin(n * math.pi * yy / H) * math.exp(-nu * (n * math.pi / H) ** 2 * t)
    return u


@pytest.mark.parametrize("nx,ny", [(1, 3), (4, 5), (3, 8)])
def test_couette_bruteforce_twin(oracle_mod, nx, ny):
    rng = np.random.default_rng(nx * 10 + ny)
    p = couette(inputs.matched_params(0.9, 10.0, 0.1, 1e-3, 0.0), 0.02)
    st = oracle_mod.flow_state(1 + 1e-2 * rng.uniform(-1, 1, (ny, nx)), 1e-2 * rng.uniform(-1, 1, (ny, nx)),
                               1e-2 * rng.uniform(-1, 1, (ny, nx)), 0.0)
    st.drho[:] = 1e-4 * rng.uniform(-1, 1, (ny, nx))
    n0, d0 = st.nstar.copy(), st.drho.copy()
    oracle_mod.run(p, st, 50)
    nb, db = bruteforce.run(p, n0, d0, 50)
    assert np.abs(nb - st.nstar).max() <= 1e-13 * np.abs(st.nstar).max()
    assert np.abs(db - st.drho).max() <= 1e-11 * np.abs(st.drho).max()
    u, _, _ = oracle_mod.fields(p, st)
    assert np.abs(bruteforce.fields(p, nb, db)["u"] - u).max() <= 1e-11 * np.abs(u).max()


def test_couette_newtonian_steady_is_linear(oracle_mod):
    ny, uw = 16, 0.01
    p = couette(inputs.matched_params(0.9, 0.0, 0.1, 1e-3, 0.0), uw)
    st = oracle_mod.init_state(np.ones((ny, 2)))
    oracle_mod.run(p, st, 20000)   # slowest mode exp(-nu pi^2 t / H^2) = exp(-5.5e-3 t)
    u, _, _ = oracle_mod.fields(p, st)
    lin = uw * (np.arange(ny) + 0.5) / (ny - 0.5)
    assert np.abs(u[..., 0] - lin[:, None]).max() <= 1e-12 * uw
    assert np.abs(u[..., 1]).max() <= 1e-15


def test_couette_newtonian_startup_series_second_order(oracle_mod):
    """At the same nu t / H^2 = 0.05 the deviation from the series falls ~4x per doubling of ny."""
    uw = 0.01
    p = couette(inputs.matched_params(0.9, 0.0, 0.1, 1e-3, 0.0), uw)
    errs = []
    for ny in (8, 16, 32):
        T = int(0.05 * (ny - 0.5) ** 2 / NU)
        st = oracle_mod.init_state(np.ones((ny, 1)))
        oracle_mod.run(p, st, T)
        u, _, _ = oracle_mod.fields(p, st)
        errs.append(np.abs(u[:, 0, 0] - startup_series(ny, uw, NU, T)).max() / uw)
    assert errs[1] <= 2e-3
    assert 3.0 <= errs[0] / errs[1] <= 5.5 and 3.0 <= errs[1] / errs[2] <= 5.5


@pytest.mark.parametrize("theta", [10.0, 100.0])
def test_couette_nlm_homogeneous_shear(oracle_mod, theta):
    ny, uw, G = 16, 0.01, 1e-3
    p = couette(inputs.matched_params(0.9, theta, 0.1, G, 0.0), uw)
    st = oracle_mod.init_state(np.ones((ny, 2)))
    oracle_mod.run(p, st, 50000)
    u, s, _ = oracle_mod.fields(p, st)
    H = ny - 0.5
    sxy, n1, _ = analytic.simple_shear(uw / H, G, theta * p["tau0"], 0.1)
    assert np.abs(s[..., 3] / sxy - 1).max() <= 1e-11
    assert np.abs((s[..., 0] - s[..., 1]) / n1 - 1).max() <= 1e-11
    # the reported u = j / (rho - delta rho) differs from the populations' velocity j / rho that
    # the Zou-He wall prescribes by the flow-induced density delta rho = -3/2 N1
    lin = uw * (np.arange(ny) + 0.5) / H
    assert np.abs(u[..., 0] - lin[:, None]).max() <= (2 * np.abs(st.drho).max() + 1e-12) * uw
