"""Warm starts for the channel runs: the learned surrogate and the closed-form profile.

The surrogate is the library's perceptron (``lbnlm.lb_mlp_*``; forward, backward and Adam run in its
CUDA kernels).  It maps a channel's parameters to its steady profiles u_x, sigma_xy and N1 on 256
points across the channel; the library decodes its outputs and writes the start state on the device
(``lbnlm.lb_warmstart_apply``), and the lattice-Boltzmann scheme then relaxes to its own steady state
(it stays the judge of the result).  Training targets come from steady LB states the same way
(``lbnlm.lb_warmstart_targets``).

Encoding (the arithmetic runs in the library's kernels; this module marshals):
  features  log10 Ny, log10 g, log10 G_inf, log10 theta, standardised with the training statistics;
  targets   the steady LB profiles minus the closed-form steady profile (the discretisation error
            of the lattice, which the network learns), each divided by the maximum |value| of the
            closed-form field, on 256 points (d = (y - y_c)/H at the centres of 256 equal cells):
            3 x 256 outputs.  Prediction = closed form + scale x network output.
"""
from __future__ import annotations

import math

import numpy as np

from . import lbnlm

NPTS = 256
N_OUT = 3 * NPTS


def features(nys, params) -> np.ndarray:
    return np.array([[math.log10(ny), math.log10(p["g_x"]), math.log10(p["G_inf"]), math.log10(max(p["theta"], 1e-12))]
                     for ny, p in zip(nys, params)], dtype=np.float64)


def steady_targets(sim):
    """Network targets of the current (steady) state of every channel of ``sim`` (an
    lbnlm.Channels): a CUDA float32 tensor [n_channels, 768]."""
    import torch
    y = torch.empty((len(sim.ny), N_OUT), dtype=torch.float32, device="cuda")
    lbnlm.lb_warmstart_targets(sim.h, y)
    return y


def start_closed_form(sim):
    """Start every channel of ``sim`` from the closed-form steady profile (on the device)."""
    lbnlm.lb_warmstart_apply(sim.h)


class Surrogate:
    """Feature / target standardisation around an lb_mlp handle."""

    def __init__(self, width=256, max_batch=512, seed=0, stream=None):
        self.n_in, self.n_out, self.width = 4, N_OUT, width
        self.m = lbnlm.lb_mlp_create(self.n_in, width, self.n_out, max_batch, seed, stream)
        self.max_batch = max_batch
        self.fmu = self.fsd = self.tmu = self.tsd = None

    def close(self):
        if self.m:
            lbnlm.lb_mlp_destroy(self.m)
            self.m = None

    def fit(self, X, Y, epochs=200, batch=256, lr=1e-3, seed=0, log=None):
        """X: host features [n, 4]; Y: targets [n, 768], a CUDA tensor (steady_targets) or host array.
        Returns the loss of each epoch's last batch."""
        import torch
        self.fmu, self.fsd = X.mean(0), X.std(0) + 1e-12
        ys = Y if isinstance(Y, torch.Tensor) else torch.tensor(Y, dtype=torch.float32, device="cuda")
        ys = ys.to(device="cuda", dtype=torch.float32)
        self.tmu = ys.mean(0).contiguous()
        self.tsd = (ys.std(0) + 1e-6).contiguous()
        ys = ((ys - self.tmu) / self.tsd).contiguous()
        xs = torch.tensor((X - self.fmu) / self.fsd, dtype=torch.float32, device="cuda")
        n = xs.shape[0]
        rng = np.random.default_rng(seed)
        losses = []
        batch = min(batch, self.max_batch, n)
        self.steps_done, self.batch_used = 0, batch
        for ep in range(epochs):
            perm = torch.tensor(rng.permutation(n), device="cuda")
            rate = lr * 0.5 * (1 + math.cos(math.pi * ep / epochs))  # cosine schedule
            starts = range(0, n - batch + 1, batch)
            last = None
            for s in starts:
                idx = perm[s:s + batch]
                xb = xs.index_select(0, idx).contiguous()
                yb = ys.index_select(0, idx).contiguous()
                # the loss comes back (and the stream is waited for) on the epoch's last batch only
                last = lbnlm.lb_mlp_train_step(self.m, xb, yb, batch, max(rate, 1e-6), want_loss=(s == starts[-1]))
                self.steps_done += 1
            losses.append(last)
            if log and (ep % 50 == 0 or ep == epochs - 1):
                log(f"epoch {ep} loss {losses[-1]:.3e}")
        return losses

    def flops_per_step(self, batch):
        """Multiply-add FLOPs of one training step (forward, the three weight gradients and the two
        input gradients of the hidden layers)."""
        i, h, o = self.n_in, self.width, self.n_out
        return 2 * batch * ((i * h + h * h + h * o) + (i * h + h * h + h * o) + (h * h + h * o))

    def predict_device(self, X):
        """Standardised network outputs for host features X [n, 4]: a CUDA float32 tensor [n, 768]."""
        import torch
        out = torch.empty((X.shape[0], self.n_out), dtype=torch.float32, device="cuda")
        for s in range(0, X.shape[0], self.max_batch):
            xb = torch.tensor((X[s:s + self.max_batch] - self.fmu) / self.fsd, dtype=torch.float32, device="cuda")
            lbnlm.lb_mlp_forward(self.m, xb.contiguous(), xb.shape[0], out[s:s + xb.shape[0]])
        return out

    def start(self, sim, nys, params):
        """Start every channel of ``sim`` from the surrogate's prediction (decoded on the device)."""
        pred = self.predict_device(features(nys, params))
        lbnlm.lb_warmstart_apply(sim.h, pred, self.tmu, self.tsd)


def judge(nx, nys, params, starts, precision="f32", stream=None, check=1000):
    """The lattice-Boltzmann scheme as the judge of the starts: every candidate start (a function
    that writes a start state into an lbnlm.Channels) runs two check intervals of the batched sweep;
    per channel the candidate with the smallest check-interval residual wins.  Returns the index of
    the winning candidate per channel."""
    res = []
    for start in starts:
        sim = lbnlm.Channels(nx, nys, params, precision, stream=stream)
        try:
            start(sim)
            _, r = sim.run_until_steady(0.0, check_every=check, max_steps=2 * check)
        finally:
            sim.close()
        res.append(np.where(np.isfinite(r), r, np.inf))
    return np.argmin(np.array(res), axis=0)


def apply_fields(sim, ux_rows_by_channel, n1_rows_by_channel):
    """Write given row profiles (host arrays) into every channel of ``sim``: u = (u_x, 0), rho = 1,
    delta rho = -(3/2) N1 (the trace of a simple-shear stress is N1), through lb_set_fields."""
    nx = sim.nx
    u = np.zeros((sim.nodes, 2))
    rho = np.ones(sim.nodes)
    drho = np.zeros(sim.nodes)
    o = 0
    for ny, ux, n1 in zip(sim.ny, ux_rows_by_channel, n1_rows_by_channel):
        n = ny * nx
        u[o:o + n, 0] = np.repeat(ux, nx)
        drho[o:o + n] = np.repeat(-1.5 * n1, nx)
        o += n
    lbnlm.lb_set_fields(sim.h, np.ascontiguousarray(u.reshape(-1)), rho, drho)
