"""Brute-force NumPy twin of the oracle for tiny grids -- TEST INFRASTRUCTURE.

A second, independently written FP64 implementation of the same scheme, used only to check
``lb_oracle.c`` on grids of a few dozen nodes.  It differs from the C oracle in every place
where a different but equivalent route exists:
  * streaming is done in PUSH form (each node sends n*_i to r + c_i; a population that would
    cross a wall is reflected into the opposite direction at its own node);
  * tensors are full 2x2 arrays; the polymer stress solves the linear steady-state equation
    behind Eq. (sigtsum), sigma/tau_M - kappa sigma - sigma kappa^T = G D, as a 4x4 Kronecker
    system with numpy.linalg.solve (no series, no symmetric reduction);
  * n^eq and F_i are evaluated with einsum over the velocity tensors Q_i;
  * pressure-driven channels (x_mode "gpbc", Sec. II B): a population pushed across x = -1/2 or
    x = nx - 1/2 arrives at the other end rebuilt from the node it leaves, with that node's
    density shifted to p_+- / c_s^2 plus its deviation from its column's mean;
  * planar Couette flow (top_wall "moving"): after streaming, the last row's unknown populations
    solve the four conditions of Zou and He as a linear system (density unknown, wall velocity
    (u_wall, 0), non-equilibrium bounce-back of the wall-normal population).
Same readings of the paper as the C oracle (listed in its header).
"""
from __future__ import annotations

import numpy as np

C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.int64)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CS2 = 1.0 / 3.0
Q = np.einsum("ia,ib->iab", C, C).astype(np.float64) - CS2 * np.eye(2)[None]


def _opposite(i):
    for o in range(9):
        if C[o, 0] == -C[i, 0] and C[o, 1] == -C[i, 1]:
            return o
    raise AssertionError


OPP = [_opposite(i) for i in range(9)]


def _neq(rho, u):
    cu = C @ u
    return W * rho * (1 + cu / CS2 + np.einsum("iab,a,b->i", Q, u, u) / (2 * CS2 ** 2))


def _stream_push(nstar, gpbc=None):
    """gpbc = (rho_plus, rho_minus) for generalized periodic boundaries, None for periodic x."""
    _, ny, nx = nstar.shape
    n = np.zeros_like(nstar)
    if gpbc is not None:
        rho_node = nstar.sum(axis=0)
        j_node = np.einsum("ia,iyx->yxa", C.astype(np.float64), nstar)
        col_mean = rho_node.mean(axis=0)  # [nx]
    for i in range(9):
        for y in range(ny):
            for x in range(nx):
                yd = y + C[i, 1]
                xd = x + C[i, 0]
                v = nstar[i, y, x]
                if not 0 <= yd < ny:
                    n[OPP[i], y, x] += v
                    continue
                if gpbc is not None and not 0 <= xd < nx:
                    # leaves through the outlet (xd = nx) -> enters at the inlet with p_+, and vice versa
                    target = gpbc[0] if xd >= nx else gpbc[1]
                    r, jv = rho_node[y, x], j_node[y, x]
                    r_new = target + r - col_mean[x]
                    v = _neq(r_new, jv / r_new)[i] + (v - _neq(r, jv / r)[i])
                n[i, yd, xd % nx] += v
    return n


def _zou_he_top(n, u_wall):
    """Unknowns (rho, n_4, n_7, n_8) at every node of the last row from: sum_i n_i = rho,
    sum_i c_iy n_i = 0, sum_i c_ix n_i = rho u_wall, n_4 - n_2 = n^eq_4 - n^eq_2 (= 0 for u_y = 0)."""
    _, ny, nx = n.shape
    y = ny - 1
    unk = [4, 7, 8]
    for x in range(nx):
        known = [i for i in range(9) if i not in unk]
        # rows: mass, y-momentum, x-momentum, normal bounce-back; columns: rho, n4, n7, n8
        A = np.zeros((4, 4))
        b = np.zeros(4)
        A[0] = [-1.0, 1.0, 1.0, 1.0]
        b[0] = -sum(n[i, y, x] for i in known)
        A[1] = [0.0] + [float(C[i, 1]) for i in unk]
        b[1] = -sum(C[i, 1] * n[i, y, x] for i in known)
        A[2] = [-u_wall] + [float(C[i, 0]) for i in unk]
        b[2] = -sum(C[i, 0] * n[i, y, x] for i in known)
        A[3] = [0.0, 1.0, 0.0, 0.0]
        b[3] = n[2, y, x]
        sol = np.linalg.solve(A, b)
        for k, i in enumerate(unk):
            n[i, y, x] = sol[k + 1]


def _grad(u):
    """u[ny, nx, 2] -> kappa[ny, nx, 2, 2] with kappa[a, b] = d_b u_a (three-point stencils)."""
    ny, nx, _ = u.shape
    k = np.zeros((ny, nx, 2, 2))
    k[:, :, :, 0] = 0.5 * (np.roll(u, -1, axis=1) - np.roll(u, 1, axis=1))
    k[1:-1, :, :, 1] = 0.5 * (u[2:] - u[:-2])
    k[0, :, :, 1] = 0.5 * (-3 * u[0] + 4 * u[1] - u[2])
    k[-1, :, :, 1] = 0.5 * (3 * u[-1] - 4 * u[-2] + u[-3])
    return k


def _sigma_kron(kap, tau_M, G):
    if tau_M == 0.0:
        return np.zeros((2, 2))
    I = np.eye(2)
    # vec(kappa S) = (kappa (x) I) vec(S), vec(S kappa^T) = (I (x) kappa) vec(S) in row-major vec
    A = np.eye(4) / tau_M - np.kron(kap, I) - np.kron(I, kap)
    D = kap + kap.T
    return np.linalg.solve(A, G * D.reshape(4)).reshape(2, 2)


def step(p, nstar, drho):
    """One step; returns (new nstar, new drho, fields dict of this update)."""
    _, ny, nx = nstar.shape
    gp = p.get("x_mode", "periodic") == "gpbc"
    if gp:
        dp = 1.5 * p["g_x"] * (nx + 1)          # c_s^-2 (p_+ - p_-)/2 with p_+ - p_- = g (nx + 1)
        rho0 = p.get("rho0", 1.0)
        n = _stream_push(nstar, (rho0 + dp, rho0 - dp))
    else:
        n = _stream_push(nstar)
    if p.get("top_wall", "bounce_back") == "moving":
        _zou_he_top(n, p.get("u_wall", 0.0))
    f = np.array([0.0 if gp else p["g_x"], 0.0])
    R0 = n.sum(axis=0)
    j = np.einsum("ia,iyx->yxa", C.astype(np.float64), n) + 0.5 * f
    ug = j / R0[..., None]
    kap = _grad(ug)
    tau = p["theta"] * p["tau0"]
    gc = p.get("gamma_c", np.inf)
    eta_inf = p["G_inf"] * p["tau0"]
    eta_N = p.get("rho0", 1.0) * CS2 * (p["tau_lb"] - 0.5)
    new = np.zeros_like(n)
    new_drho = np.zeros_like(drho)
    sig_out = np.zeros((ny, nx, 2, 2))
    rho_h = np.zeros((ny, nx))
    u_out = np.zeros((ny, nx, 2))
    t = p["tau_lb"]
    for y in range(ny):
        for x in range(nx):
            K = kap[y, x]
            D = K + K.T
            II = 0.5 * np.trace(D @ D)
            tm = 0.0 if tau == 0 else 1.0 / (1.0 / tau + (0.0 if np.isinf(gc) else np.sqrt(II) / gc))
            sig = _sigma_kron(K, tm, p["G_inf"])
            snn = sig + (eta_inf - eta_N) * D
            dr = 0.0 if gp else -np.trace(snn) / (CS2 * 2)
            S = 0.0 if gp else dr - drho[y, x]
            sbar = snn - 0.5 * np.trace(snn) * np.eye(2)
            rho = R0[y, x] + 0.5 * S
            u = j[y, x] / rho
            neq = _neq(rho, u)
            Y = -S * np.outer(u, u) + np.outer(f, u) + np.outer(u, f)
            F = W * (-np.einsum("iab,ab->i", Q, sbar) / (2 * CS2 ** 2 * t)
                     + (1 - 1 / (2 * t)) * (S + (C @ f) / CS2 + np.einsum("iab,ab->i", Q, Y) / (2 * CS2 ** 2)))
            new[:, y, x] = n[:, y, x] - (n[:, y, x] - neq) / t + F
            new_drho[y, x] = dr
            sig_out[y, x] = sig
            rho_h[y, x] = rho - dr
            u_out[y, x] = j[y, x] / rho_h[y, x]
    return new, new_drho, {"u": u_out, "sigma": sig_out, "rho": rho_h}


def run(p, nstar, drho, nsteps):
    nstar = nstar.copy()
    drho = drho.copy()
    for _ in range(nsteps):
        nstar, drho, _ = step(p, nstar, drho)
    return nstar, drho


def fields(p, nstar, drho):
    _, _, fl = step(p, nstar, drho)
    return fl
