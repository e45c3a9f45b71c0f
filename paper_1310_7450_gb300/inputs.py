"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the lattice-Boltzmann method itself: it only draws random
numbers and turns the paper's dimensionless run parameters into lattice parameters.

* ``splitmix64`` -- the counter-based SplitMix64 generator (Steele, Lea & Flood, OOPSLA 2014;
  the 64-bit finaliser as published by Vigna).  Output k >= 1 of the stream with seed s is
  mix(s + k * 0x9E3779B97F4A7C15).  The CUDA library implements the same published definition
  on its own for the seeded density perturbation of ``lb_create``; tests check the two agree.
* ``initial_density`` -- rho(r) = rho0 (1 + a U(-1,1)) with U from output (node index + 1).
* parameter recipes for the channel workloads (low-shear viscosity matched to tau_LB).
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters) -> np.ndarray:
    """Output number ``counters`` (array, >= 1) of the SplitMix64 stream seeded with ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + np.asarray(counters, dtype=np.uint64) * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, counters) -> np.ndarray:
    """U(-1, 1) from the top 53 bits: 2 * (z >> 11) * 2^-53 - 1 (exact in FP64)."""
    z = splitmix64(seed, counters)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0


def initial_density(nx: int, ny: int, rho0: float, amp: float, seed: int, node_offset: int = 0) -> np.ndarray:
    """rho[y, x] = rho0 * (1 + amp * U(-1,1)), U drawn at counter node_offset + y*nx + x + 1."""
    k = np.arange(nx * ny, dtype=np.uint64) + np.uint64(node_offset + 1)
    if amp == 0.0:
        return np.full((ny, nx), float(rho0))
    return (rho0 * (1.0 + amp * uniform_pm1(seed, k))).reshape(ny, nx)


def linear_density(nx: int, ny: int, rho_in: float, rho_out: float, rho0: float = 1.0, amp: float = 0.0,
                   seed: int = 0) -> np.ndarray:
    """Start of a pressure-driven channel: the straight line between the densities held at the ghost
    columns x = -1 (rho_in) and x = nx (rho_out), plus rho0 * amp * U(-1,1) at the counters of
    ``initial_density``."""
    x = np.arange(nx, dtype=np.float64)
    lin = rho_in + (rho_out - rho_in) * (x + 1.0) / (nx + 1.0)
    rho = np.repeat(lin[None, :], ny, axis=0)
    if amp != 0.0:
        k = np.arange(nx * ny, dtype=np.uint64) + np.uint64(1)
        rho = rho + (rho0 * (amp * uniform_pm1(seed, k))).reshape(ny, nx)
    return rho


# --------------------------------------------------------------------------------------------
# Parameter recipes.  Lattice units dx = dt = 1, c_s^2 = 1/3.  The Newtonian viscosity carried
# by the BGK collision, eta^N = rho0 (tau_LB - 1/2)/3, is matched to the low-shear viscosity of
# the Maxwell model, G_inf (tau + tau0) = G_inf tau0 (1 + theta)  (choice of Sec. IV).

def nu_lb(tau_lb: float, rho0: float = 1.0) -> float:
    return rho0 * (tau_lb - 0.5) / 3.0


def matched_params(tau_lb: float, theta: float, gamma_c: float, G_inf: float, g_x: float,
                   rho0: float = 1.0, stress_mode: int = 0) -> dict:
    """tau0 from the matching rule; everything else as given."""
    tau0 = nu_lb(tau_lb, rho0) / (G_inf * (1.0 + theta))
    return dict(tau_lb=tau_lb, g_x=g_x, G_inf=G_inf, tau0=tau0, theta=theta, gamma_c=gamma_c,
                rho0=rho0, stress_mode=stress_mode)


def yield_stress_channel(ny: int, tau_lb: float = 0.9, theta: float = 100.0, gamma_c: float = 0.1,
                         wpH: float = 0.5, tau: float | None = None, g_x: float | None = None) -> dict:
    """Channel whose driving is wp*H = g H / G_inf (wpH = 1/2: the paper's Delta p = G_inf/(2H),
    plug half-width gamma_c/(wp H) = 0.2).  Either tau = theta*tau0 (then G_inf follows from the
    matching rule and g from wpH) or g_x is given (then G_inf = g H / wpH)."""
    H = ny / 2.0
    nu = nu_lb(tau_lb)
    if tau is not None:
        tau0 = tau / theta
        G = nu / (tau0 * (1.0 + theta))
        g = wpH * G / H
    else:
        g = g_x
        G = g * H / wpH
    return matched_params(tau_lb, theta, gamma_c, G, g)


# The workloads (sizes and parameters) of the runs -----------------------------------------

def oracle_channel_newtonian() -> dict:
    """4 x 64 channel, theta = 0, tau_LB = 0.9, g = 1e-6 from rest (20000 steps)."""
    return dict(nx=4, ny=64, steps=20000,
                params=matched_params(0.9, 0.0, 0.1, 1e-3, 1e-6))


def oracle_channel_yield() -> dict:
    """4 x 64 channel at theta = 100, tau = theta*tau0 = 1e4 steps, gamma_c = 0.1, wpH = 1/2."""
    return dict(nx=4, ny=64, steps=20000,
                params=yield_stress_channel(64, tau=1e4))


def single_large_channel(nx: int = 4096, ny: int = 4096) -> dict:
    """Start-up of a 4096 x 4096 channel: theta = 100, gamma_c = 0.1, tau_LB = 0.9, g = 1e-6,
    G_inf = 1e-3, rho = 1 + 1e-6 U(-1,1) with seed 1."""
    return dict(nx=nx, ny=ny, params=matched_params(0.9, 100.0, 0.1, 1e-3, 1e-6),
                rho_pert_amp=1e-6, seed=1)


def reduced_precision_channel(nx: int = 8192, ny: int = 2048) -> dict:
    """8192 x 2048 channel with the dimensionless parameters of the 4 x 64 yield-stress run
    (theta = 100, gamma_c = 0.1, wpH = 1/2), g scaled by (32/H)^2 to keep the peak speed."""
    H = ny / 2.0
    g = 2.0 * 1.3201320132013201e-5 / 64.0 / 2.0 * (32.0 / H) ** 2
    return dict(nx=nx, ny=ny, params=yield_stress_channel(ny, g_x=g))


def sweep_draws(n_channels: int, seed: int, ny_lo: int = 32, ny_hi: int = 1024):
    """Per-channel draws of the batched sweep: Ny ~ U{ny_lo..ny_hi}, b ~ logU[1e-8, 1e-5],
    eps ~ U[-0.1, 0.1].  Independent SplitMix64 streams per quantity (counters 3c+1..3c+3)."""
    c = np.arange(n_channels, dtype=np.uint64)
    u0 = (uniform_pm1(seed, 3 * c + 1) + 1.0) / 2.0
    u1 = (uniform_pm1(seed, 3 * c + 2) + 1.0) / 2.0
    u2 = uniform_pm1(seed, 3 * c + 3)
    ny = np.minimum(ny_lo + np.floor(u0 * (ny_hi - ny_lo + 1)).astype(np.int64), ny_hi)
    b = 10.0 ** (-8.0 + 3.0 * u1)
    eps = 0.1 * u2
    return ny, b, eps


def theta_of_eps(eps):
    """Distance to the glass transition -> theta = 10^(2 + 10 eps) (an invented mapping: the paper
    has no eps; this spans its theta range 10..1000)."""
    return 10.0 ** (2.0 + 10.0 * np.asarray(eps))


def steady_peak_speed(ny: int, g: float, G: float, tau0: float, theta: float, gamma_c: float,
                      n: int = 2000) -> float:
    """Peak speed of the steady profile (Eq. maxwellpoiseuille integrated by the trapezoid rule)
    used only to choose G_inf in the sweep recipe."""
    H = ny / 2.0
    wpH = g * H / G
    d = np.linspace(0.0, 1.0, n + 1)
    a = wpH * d / 2.0
    b = gamma_c * (1.0 + theta) / (2.0 * theta)
    dv = -a + b - np.sqrt((a - b) ** 2 + wpH * d * gamma_c / theta)
    v0 = -np.trapezoid(dv, d)
    return float(H / tau0 * v0)


def sweep_channel_params(n_channels: int, seed: int, tau_lb: float = 0.9, gamma_c: float = 0.1,
                         u_max: float = 0.05, ny_lo: int = 32, ny_hi: int = 1024):
    """Parameters of the batched sweep: g = b (32/Ny)^2; G_inf the smallest value >= 1e-6 whose
    steady peak speed is <= u_max (bisection in log G)."""
    ny, b, eps = sweep_draws(n_channels, seed, ny_lo, ny_hi)
    theta = theta_of_eps(eps)
    out = []
    for k in range(n_channels):
        g = float(b[k] * (32.0 / ny[k]) ** 2)
        th = float(theta[k])

        def peak(G):
            tau0 = nu_lb(tau_lb) / (G * (1.0 + th))
            return steady_peak_speed(int(ny[k]), g, G, tau0, th, gamma_c)

        lo, hi = math.log(1e-6), math.log(1.0)
        if peak(math.exp(lo)) > u_max:
            for _ in range(60):
                mid = 0.5 * (lo + hi)
                if peak(math.exp(mid)) > u_max:
                    lo = mid
                else:
                    hi = mid
            G = math.exp(hi)
        else:
            G = math.exp(lo)
        out.append(dict(ny=int(ny[k]), **matched_params(tau_lb, th, gamma_c, G, g)))
    return out
