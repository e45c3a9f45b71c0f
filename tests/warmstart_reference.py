"""NumPy reference of the warm start's profile arithmetic, which the library runs on the device
(lb_warmstart_apply, lb_warmstart_targets): the closed-form steady channel profile of Sec. III B
(trapezoid rule), the linear resampling between a channel's rows and the 256-point network grid
(end values held), and the target encoding / decoding.  Test infrastructure: the GPU tests compare
the kernels with it, and it is pinned to the oracle's adaptive quadrature on the CPU."""
import numpy as np


NPTS = 256
D_GRID = (np.arange(NPTS) + 0.5) / NPTS * 2.0 - 1.0


def rows_d(ny: int) -> np.ndarray:
    return (np.arange(ny) - (ny - 1) / 2.0) / (ny / 2.0)


def to_grid(profile_rows: np.ndarray, ny: int) -> np.ndarray:
    """Linear interpolation of a profile on the ny rows onto the 256-point grid (end values held)."""
    return np.interp(D_GRID, rows_d(ny), profile_rows)


def to_rows(profile_grid: np.ndarray, ny: int) -> np.ndarray:
    return np.interp(rows_d(ny), D_GRID, profile_grid)


def closed_form_grid(ny: int, p: dict):
    """Closed-form (u, sxy, N1) of the channel on the 256-point grid and the per-field scales."""
    prof = [to_grid(f, ny) for f in analytic_rows(ny, p)]
    sc = [max(np.abs(f).max(), 1e-300) for f in prof]
    return prof, sc


def encode_targets(nys, params, u_rows, sxy_rows, n1_rows) -> np.ndarray:
    """Per channel: [(LB - closed form)/scale for u, sxy, N1 on the 256 points]."""
    out = np.zeros((len(nys), 3 * NPTS))
    for k, (ny, p) in enumerate(zip(nys, params)):
        ref, sc = closed_form_grid(ny, p)
        lb = [to_grid(u_rows[k], ny), to_grid(sxy_rows[k], ny), to_grid(n1_rows[k], ny)]
        for j in range(3):
            out[k, j * NPTS:(j + 1) * NPTS] = (lb[j] - ref[j]) / sc[j]
    return out


def decode(nys, params, pred: np.ndarray):
    """Inverse of encode_targets on the 256-point grid: lists of (u, sxy, N1) arrays per channel."""
    res = []
    for k, (ny, p) in enumerate(zip(nys, params)):
        ref, sc = closed_form_grid(ny, p)
        res.append(tuple(ref[j] + sc[j] * pred[k, j * NPTS:(j + 1) * NPTS] for j in range(3)))
    return res


def analytic_rows(ny: int, p: dict, n: int = 4001):
    """Closed-form steady channel (the quadratic for dv/dd of Sec. III B, integrated with the
    trapezoid rule on n points so that v(1) = 0): u_x, sigma_xy, N1 on the rows."""
    H = ny / 2.0
    G, tau0, theta, gc = p["G_inf"], p["tau0"], p["theta"], p.get("gamma_c", 0.1)
    wpH = p["g_x"] * H / G
    d = np.linspace(0.0, 1.0, n)
    if theta == 0.0:
        dv = -wpH * d
    else:
        a = wpH * d / 2.0
        b = gc * (1.0 + theta) / (2.0 * theta)
        dv = -a + b - np.sqrt((a - b) ** 2 + wpH * d * gc / theta)
    v = np.concatenate([[0.0], np.cumsum(0.5 * (dv[1:] + dv[:-1]) * np.diff(d))])
    v = v - v[-1]
    dd = np.abs(rows_d(ny))
    u = (H / tau0) * np.interp(dd, d, v)
    gdot = np.interp(dd, d, dv) / tau0 * np.sign(rows_d(ny))
    tau = theta * tau0
    tau_m = tau / (1.0 + tau * np.abs(gdot) / gc) if tau > 0 else np.zeros_like(gdot)
    sxy = G * tau_m * gdot
    n1 = 2.0 * G * gdot ** 2 * tau_m ** 2
    return u, sxy, n1
