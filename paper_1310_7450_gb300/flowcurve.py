"""Flow curves sigma_xy(gdot), N1(gdot) from the lattice-Boltzmann runs (the paper's flow-curve
figure and its channel-data comparison, Sec. III A and Sec. IV).

* ``couette``: one handle of planar Couette channels (Zou-He moving wall, Sec. IV C), one channel
  per target shear rate; each channel starts from its linear steady profile and steps until the
  residual falls below ``tol``; per channel the imposed shear rate u_wall / H (what the stress
  sees: the velocity gradients use the populations' velocity j / sum n, which the wall fixes),
  the slope of the reported velocity between the second and the second-last rows (it differs by
  the flow-induced density factor rho / (rho - delta rho)), and the row means of sigma_xy and
  N1 = sigma_xx - sigma_yy.
* ``from_channel``: local (gdot, sigma_xy, N1) triples of a channel state, gdot from the three-point
  difference of u_x across the rows (the stencils of the step).

Host-side marshalling and post-processing only; every step runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import lbnlm


def couette(gdots, params, ny: int = 16, nx: int = 1, precision: str = "f64", stream=None, tol: float = 1e-12,
            chunk: int = 2000, max_steps: int = 400_000):
    """Returns (gdot imposed, gdot from the reported velocity, sigma_xy, N1, steps), one entry per
    requested shear rate."""
    gdots = np.asarray(gdots, dtype=np.float64)
    n = gdots.size
    H = ny - 0.5                    # half-way wall at y = -1/2, moving wall on row ny-1
    uw = gdots * H
    y = np.arange(ny) + 0.5
    plist = [dict(params) for _ in range(n)]
    with lbnlm.Channels(nx, [ny] * n, plist, precision, stream=stream, walls="couette") as sim:
        for c in range(n):
            lbnlm.lb_set_wall_velocity(sim.h, c, float(uw[c]))
        u = np.zeros((n, ny, nx, 2))
        u[..., 0] = (uw[:, None] * y[None, :] / H)[:, :, None]
        lbnlm.lb_set_fields(sim.h, np.ascontiguousarray(u.reshape(-1)), np.ones(n * ny * nx))
        steps = 0
        while True:
            sim.step(chunk)
            steps += chunk
            r = sim.residual()
            if np.all(r <= tol) or steps >= max_steps:
                break
        fl = sim.fields()
    g = np.array([(f[0][-2, :, 0].mean() - f[0][1, :, 0].mean()) / (ny - 3) for f in fl])
    sxy = np.array([f[1][..., 3].mean() for f in fl])
    n1 = np.array([(f[1][..., 0] - f[1][..., 1]).mean() for f in fl])
    return uw / H, g, sxy, n1, steps


def from_channel(u: np.ndarray, sigma: np.ndarray):
    """u [ny, nx, 2], sigma [ny, nx, 4] (xx, yy, zz, xy) -> per interior row (gdot, sigma_xy, N1),
    averaged over x."""
    ux = u[..., 0].mean(axis=1)
    gd = 0.5 * (ux[2:] - ux[:-2])
    sxy = sigma[1:-1, :, 3].mean(axis=1)
    n1 = (sigma[1:-1, :, 0] - sigma[1:-1, :, 1]).mean(axis=1)
    return gd, sxy, n1
