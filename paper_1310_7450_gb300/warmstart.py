"""Warm starts for the channel runs: the learned surrogate and the closed-form profile.

The surrogate is the library's perceptron (``lbnlm.lb_mlp_*``; forward, backward and Adam run in its
CUDA kernels).  It maps a channel's parameters to its steady profiles u_x, sigma_xy and N1 on 256
points across the channel; ``apply`` writes a profile into a handle with ``lb_set_fields`` and the
lattice-Boltzmann scheme then relaxes to its own steady state (it stays the judge of the result).

Encoding (host-side marshalling only):
  features  log10 Ny, log10 g, log10 G_inf, log10 theta, standardised with the training statistics;
  targets   the steady LB profiles minus the closed-form steady profile (the discretisation error
            of the lattice, which the network learns), each divided by the maximum |value| of the
            closed-form field, on 256 points (d = (y - y_c)/H at the centres of 256 equal cells):
            3 x 256 outputs.  Prediction = closed form + scale x network output.
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs, lbnlm

NPTS = 256
D_GRID = (np.arange(NPTS) + 0.5) / NPTS * 2.0 - 1.0


def scales(ny: int, p: dict):
    H = ny / 2.0
    nu = inputs.nu_lb(p["tau_lb"], p.get("rho0", 1.0))
    us = p["g_x"] * H * H / (2.0 * nu)
    ss = p["g_x"] * H
    ns = ss * ss / p["G_inf"]
    return us, ss, ns


def features(nys, params) -> np.ndarray:
    return np.array([[math.log10(ny), math.log10(p["g_x"]), math.log10(p["G_inf"]), math.log10(max(p["theta"], 1e-12))]
                     for ny, p in zip(nys, params)], dtype=np.float64)


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


class Surrogate:
    """Feature / target standardisation around an lb_mlp handle."""

    def __init__(self, width=256, max_batch=512, seed=0, stream=None):
        self.n_in, self.n_out, self.width = 4, 3 * NPTS, width
        self.m = lbnlm.lb_mlp_create(self.n_in, width, self.n_out, max_batch, seed, stream)
        self.max_batch = max_batch
        self.fmu = self.fsd = self.tmu = self.tsd = None

    def close(self):
        if self.m:
            lbnlm.lb_mlp_destroy(self.m)
            self.m = None

    def fit(self, X, Y, epochs=200, batch=256, lr=1e-3, seed=0, log=None):
        import torch
        self.fmu, self.fsd = X.mean(0), X.std(0) + 1e-12
        self.tmu, self.tsd = Y.mean(0), Y.std(0) + 1e-6
        xs = torch.tensor((X - self.fmu) / self.fsd, dtype=torch.float32, device="cuda")
        ys = torch.tensor((Y - self.tmu) / self.tsd, dtype=torch.float32, device="cuda")
        n = xs.shape[0]
        rng = np.random.default_rng(seed)
        losses = []
        batch = min(batch, self.max_batch, n)
        for ep in range(epochs):
            perm = torch.tensor(rng.permutation(n), device="cuda")
            rate = lr * 0.5 * (1 + math.cos(math.pi * ep / epochs))  # cosine schedule
            tot = 0.0
            nb = 0
            for s in range(0, n - batch + 1, batch):
                idx = perm[s:s + batch]
                xb = xs.index_select(0, idx).contiguous()
                yb = ys.index_select(0, idx).contiguous()
                tot += lbnlm.lb_mlp_train_step(self.m, xb, yb, batch, max(rate, 1e-6))
                nb += 1
            losses.append(tot / max(nb, 1))
            if log and (ep % 50 == 0 or ep == epochs - 1):
                log(f"epoch {ep} loss {losses[-1]:.3e}")
        return losses

    def predict(self, X) -> np.ndarray:
        import torch
        out = np.zeros((X.shape[0], self.n_out))
        for s in range(0, X.shape[0], self.max_batch):
            xb = torch.tensor((X[s:s + self.max_batch] - self.fmu) / self.fsd, dtype=torch.float32, device="cuda")
            yb = torch.zeros((xb.shape[0], self.n_out), dtype=torch.float32, device="cuda")
            lbnlm.lb_mlp_forward(self.m, xb.contiguous(), xb.shape[0], yb)
            torch.cuda.synchronize()
            out[s:s + xb.shape[0]] = yb.cpu().numpy() * self.tsd + self.tmu
        return out


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


def judge(nx, nys, params, candidates, precision="f32", stream=None, check=1000):
    """The lattice-Boltzmann scheme as the judge of the starts: every candidate (a list of per-channel
    (u_x, sigma_xy, N1) row profiles) runs two check intervals of the batched sweep; per channel the
    candidate with the smallest check-interval residual wins.  Returns (chosen rows, index of the
    winning candidate per channel)."""
    res = []
    for rows in candidates:
        sim = lbnlm.Channels(nx, nys, params, precision, stream=stream)
        try:
            apply(sim, rows)
            _, r = sim.run_until_steady(0.0, check_every=check, max_steps=2 * check)
        finally:
            sim.close()
        res.append(np.where(np.isfinite(r), r, np.inf))
    pick = np.argmin(np.array(res), axis=0)
    return [candidates[k][c] for c, k in enumerate(pick)], pick


def apply(sim, rows_by_channel):
    """Write (u_x, sigma_xy, N1) row profiles into every channel of ``sim`` (an lbnlm.Channels):
    u = (u_x, 0), rho = 1 and the stored flow-induced density delta rho = -(3/2) tr sigma with
    tr sigma = N1 in a simple-shear profile."""
    nx = sim.nx
    u = np.zeros((sim.nodes, 2))
    rho = np.ones(sim.nodes)
    drho = np.zeros(sim.nodes)
    o = 0
    for ny, (ux, sxy, n1) in zip(sim.ny, rows_by_channel):
        n = ny * nx
        u[o:o + n, 0] = np.repeat(ux, nx)
        drho[o:o + n] = np.repeat(-1.5 * n1, nx)
        o += n
    lbnlm.lb_set_fields(sim.h, np.ascontiguousarray(u.reshape(-1)), rho, drho)
