"""Closed forms of the paper used to pin the oracle -- TEST INFRASTRUCTURE (see ``oracle/__init__``).

Channel geometry in lattice units (reading of the wall location): fluid rows y = 0..Ny-1,
half-way bounce-back walls at y = -1/2 and y = Ny - 1/2, so the channel width is 2H = Ny and
the centre is y_c = (Ny - 1)/2; the dimensionless coordinate of Sec. III B is d = (y - y_c)/H.

Dimensionless channel problem (Sec. III B, Eq. nspoiseuille): s = t/tau0, d = y/H,
v = u_x tau0 / H, wp = Delta p / G_inf with Delta p the pressure drop per unit length, which
for body-force driving is the force density g.  So wp*H = g*H/G_inf and u_x = (H/tau0) v.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate


def dvdd(d: float, wpH: float, theta: float, gamma_c: float) -> float:
    """Eq. (maxwellpoiseuille): steady shear rate d v/d d at d >= 0 (odd in d).  theta = 0 is the
    Newtonian limit -wpH*d (Sec. III B)."""
    s = 1.0 if d >= 0 else -1.0
    d = abs(d)
    if theta == 0.0:
        return -s * wpH * d
    a = wpH * d / 2.0
    b = gamma_c * (1.0 + theta) / (2.0 * theta)
    return s * (-a + b - math.sqrt((a - b) ** 2 + wpH * d * gamma_c / theta))


def quadratic_residual(d: float, x: float, wpH: float, theta: float, gamma_c: float) -> float:
    """Right-hand side of the quadratic for d v/d d printed above Eq. (maxwellpoiseuille)."""
    return wpH * d + (1.0 + theta - wpH * d * theta / gamma_c) * x - (theta / gamma_c) * x * x


def v_of_d(d: float, wpH: float, theta: float, gamma_c: float) -> float:
    """v(d) = -int_{|d|}^1 dv/dd, so that v(1) = 0 (text below Eq. maxwellpoiseuille); adaptive
    Gauss-Kronrod (QUADPACK) with the plug edge d_c as a break point."""
    d = abs(d)
    pts = []
    if theta > 0 and wpH > 0:
        dc = gamma_c / wpH
        if d < dc < 1.0:
            pts = [dc]
    val, _ = integrate.quad(lambda s: dvdd(s, wpH, theta, gamma_c), d, 1.0, points=pts or None,
                            epsabs=1e-15, epsrel=1e-13, limit=400)
    return -val


def channel_profile(ny: int, g: float, G_inf: float, tau0: float, theta: float, gamma_c: float):
    """Analytic steady u_x(y) on the lattice rows y = 0..ny-1 (Eq. maxwellpoiseuille).  For
    theta = 0 the Newtonian parabola g/(2 nu) (H^2 - (y-y_c)^2) with nu = G_inf tau0."""
    H = ny / 2.0
    yc = (ny - 1) / 2.0
    wpH = g * H / G_inf
    out = np.empty(ny)
    for y in range(ny):
        d = (y - yc) / H
        out[y] = (H / tau0) * v_of_d(d, wpH, theta, gamma_c)
    return out


def channel_shear_rate(ny: int, g: float, G_inf: float, tau0: float, theta: float, gamma_c: float):
    """Analytic d u_x / d y on the rows: (1/tau0) dv/dd."""
    H = ny / 2.0
    yc = (ny - 1) / 2.0
    wpH = g * H / G_inf
    return np.array([dvdd((y - yc) / H, wpH, theta, gamma_c) / tau0 for y in range(ny)])


def newtonian_parabola(ny: int, g: float, nu: float):
    """Plane Poiseuille profile g/(2 nu) (H^2 - (y - y_c)^2) for walls at -1/2 and ny - 1/2."""
    H = ny / 2.0
    y = np.arange(ny) - (ny - 1) / 2.0
    return g / (2.0 * nu) * (H * H - y * y)


def newtonian_startup(ny: int, g: float, nu: float, t: float, nterms: int = 400):
    """Start-up of plane Poiseuille flow from rest (the Newtonian solution the paper cites in
    Sec. IV B, derived here from the 1-D diffusion equation u_t = g + nu u_yy, u(+-H) = 0):
    u = g/(2nu)(H^2-y^2) - sum_n 16 g H^2 (-1)^n/(nu pi^3 (2n+1)^3) cos((2n+1) pi y/(2H))
        exp(-(2n+1)^2 pi^2 nu t / (4 H^2))."""
    H = ny / 2.0
    y = np.arange(ny) - (ny - 1) / 2.0
    u = g / (2.0 * nu) * (H * H - y * y)
    for n in range(nterms):
        k = 2 * n + 1
        u -= (16.0 * g * H * H * (-1) ** n / (nu * math.pi ** 3 * k ** 3) *
              np.cos(k * math.pi * y / (2.0 * H)) * math.exp(-k * k * math.pi ** 2 * nu * t / (4 * H * H)))
    return u


def plug_half_width(wpH: float, gamma_c: float) -> float:
    """d_c = gamma_c / (wp H), the plug edge of Eq. (plug)."""
    return gamma_c / wpH


def plug_asymptote(d: float, wpH: float, theta: float, gamma_c: float) -> float:
    """Eq. (plug), theta -> infinity, d >= 0; the inner branch reads p H d as wp H d."""
    dc = gamma_c / wpH
    if d > dc:
        return -wpH * d + gamma_c
    return wpH * d * gamma_c / (wpH * d - gamma_c) / theta


def normal_stress_asymptote(d: float, wpH: float, G_inf: float, gamma_c: float) -> float:
    """Eq. (mwnd): sigma_xx - sigma_yy for theta -> infinity."""
    dc = gamma_c / wpH
    return 2.0 * G_inf * gamma_c ** 2 if d > dc else 2.0 * G_inf * (wpH * d) ** 2


def yield_pressure_drop(G_inf: float, gamma_c: float, H: float) -> float:
    """Delta p_c = 2 G_inf gamma_c / (2H): below it no flow (Sec. III B)."""
    return 2.0 * G_inf * gamma_c / (2.0 * H)


def simple_shear(gdot: float, G: float, tau: float, gamma_c: float):
    """Simple shear kappa_xy = gdot (Sec. III A): returns (sigma_xy, N1, tau_M) with
    sigma_xy = G gdot tau_M, N1 = 2 G gdot^2 tau_M^2 and tau_M of Eq. (nlmaxwell), II_D = gdot^2."""
    inv_gc = 0.0 if math.isinf(gamma_c) else 1.0 / gamma_c
    tau_M = tau / (1.0 + tau * abs(gdot) * inv_gc) if tau > 0 else 0.0
    return G * gdot * tau_M, 2.0 * G * gdot * gdot * tau_M * tau_M, tau_M


def planar_extension_xx(edot: float, G: float, tau_M: float) -> float:
    """Planar extension kappa_xx = -kappa_yy = edot: sigma_xx = 2 G edot tau_M/(1 - 2 edot tau_M)
    (Sec. III A, valid for edot tau_M < 1/2)."""
    return 2.0 * G * edot * tau_M / (1.0 - 2.0 * edot * tau_M)


def simple_shear_yield_stress(G: float, gamma_c: float):
    """Eq. (yieldstress) for simple shear kappa_0 = e_x e_y (II_D0 = 1): only n = 1, 2 survive,
    sigma_y = G gamma_c D_0 + 2 G gamma_c^2 kappa_0 kappa_0^T -> (xx, xy, yy)."""
    return np.array([2.0 * G * gamma_c ** 2, G * gamma_c, 0.0])
