"""FP64 CPU oracle of the nlM lattice-Boltzmann scheme (arXiv:1310.7450) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  The product library (``paper_1310_7450_gb300``) never imports it and shares no
code with it: the oracle is plain C (``lb_oracle.c``), compiled here with gcc, plus a NumPy
brute-force twin (``bruteforce.py``) and the paper's closed forms (``analytic.py``).

State layout used by every function here:
    dev[9, ny, nx]    post-collision populations of the last step as offsets from the lattice
                      weights, n*_i - w_i (D2Q9, numbering 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0)
                      4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1)); ``State.nstar`` gives n*_i
    drho[ny, nx]      flow-induced density change delta rho of the last collision (Sec. II A)
    sig[3, ny, nx]    carried polymer stress (xx, xy, yy); only stress mode 1 reads it

Parity status of each function (what pins it, see ``tests/test_oracle_*.py``):
    equilibrium      pinned: moments of Eq. (neq) against Eq. (pieq) / Eq. (rhoj)
    forcing          pinned: zeroth/first/second moments against the conditions below Eq. (lbfab)
    stress_series    pinned: simple-shear / extension / yield-stress closed forms of Sec. III A,
                     and against the separately written elimination
    stress_step      pinned: its fixed point is the steady solution of Eq. (sigtsum)
    intermediates    pinned directly: the three-point gradients (Sec. II C) are exact on a planted
                     quadratic velocity, wall rows included; the delta rho of Eq. (rhoplus) makes
                     the hydrodynamic density uniform in a steady channel while rho_eq + 3/2 N1 is
                     constant (tests/test_oracle_gradients_density.py)
    run / fields     pinned: Newtonian parabola and start-up series, analytic nlM channel profile
                     (Eq. maxwellpoiseuille), mass conservation, mirror symmetry, Newtonian
                     equivalence of the forcing (below Eq. bodyforce), brute-force twin
    GPBC runs        pinned: brute-force twin (push form), Newtonian parabola and linear pressure,
                     continuity of the mass flux, equality with the body-force run (Sec. II B)
    Couette runs     pinned: brute-force twin, exact linear Newtonian profile, start-up Fourier
                     series, homogeneous nlM shear (Sec. III A closed forms), mass invariance
    comparison       generalized-Newtonian scheme: steady channel against Eq. (maxwellpoiseuille)
    schemes          with second-order convergence, theta = 0 equal to the paper's scheme, no
    (Sec. II C)      normal stresses; stress-divergence scheme: steady channel against the
                     paper's scheme to O(H^-2) and against Eq. (maxwellpoiseuille), Newtonian
                     cross-check (a Delta eta D stress acts as the viscosity Delta eta)
                     (tests/test_oracle_schemes.py)
    relaxation       tau(rho): homogeneous Couette shear at a uniform density equals the Sec. III A
    extensions       closed form at tau exp(beta (rho - rho_ref)/rho_ref); fluidity memory: the
                     backward-Euler recursion against its closed form, steady states unchanged,
                     start-up stress overshoot with a long memory
                     (tests/test_oracle_relaxation_models.py)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_SO = os.path.join(_HERE, "liblboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``lb_oracle.c`` with gcc (no fast-math, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class OrcParams(ctypes.Structure):
    _fields_ = [("tau_lb", ctypes.c_double), ("g_x", ctypes.c_double), ("G_inf", ctypes.c_double),
                ("tau0", ctypes.c_double), ("theta", ctypes.c_double), ("gamma_c", ctypes.c_double),
                ("rho0", ctypes.c_double), ("stress_mode", ctypes.c_int), ("boundary", ctypes.c_int),
                ("rho_in", ctypes.c_double), ("rho_out", ctypes.c_double), ("top_wall", ctypes.c_int),
                ("scheme", ctypes.c_int), ("u_wall", ctypes.c_double), ("beta_rho", ctypes.c_double),
                ("rho_ref", ctypes.c_double), ("tau_f", ctypes.c_double)]


SCHEMES = {"paper": 0, "generalized_newtonian": 1, "stress_divergence": 2}


_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_equilibrium.argtypes = [ctypes.c_double] * 3 + [_D]
        lib.orc_equilibrium_offset.argtypes = [ctypes.c_double] * 3 + [_D]
        lib.orc_forcing.argtypes = [ctypes.c_double, _D, ctypes.c_double, _D, _D, _D]
        lib.orc_relaxation_time.argtypes = [ctypes.c_double] * 3
        lib.orc_relaxation_time.restype = ctypes.c_double
        lib.orc_stress_series.argtypes = [_D, ctypes.c_double, ctypes.c_double, _D]
        lib.orc_stress_gauss.argtypes = [_D, ctypes.c_double, ctypes.c_double, _D]
        lib.orc_stress_step.argtypes = [_D, ctypes.c_double, ctypes.c_double, _D, _D]
        lib.orc_init.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
        lib.orc_run.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_int, ctypes.c_int, _D, _D, _D, _D,
                                ctypes.c_long, ctypes.c_int]
        lib.orc_fields.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_int, ctypes.c_int, _D, _D, _D,
                                   _D, _D, _D, _D]
        lib.orc_node_intermediates.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_int, ctypes.c_int,
                                               _D, _D, _D, _D, _D]
        lib.orc_fluidity_step.argtypes = [ctypes.c_double] * 3
        lib.orc_fluidity_step.restype = ctypes.c_double
        lib.orc_fallback_count.restype = ctypes.c_long
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _vec(x, n):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(n))
    return a


def gpbc_density_offsets(p, nx: int):
    """Inlet / outlet lattice densities c_s^-2 p_+- of a pressure-driven channel (Sec. II B), minus 1.
    Reading: the imposed pressure gradient equals the body force g_x it replaces, with p_+ and p_-
    held at the ghost columns x = -1 and x = nx, so p_+ - p_- = g_x (nx + 1), centred on rho0."""
    get = (lambda k, d=None: p.get(k, d)) if isinstance(p, dict) else (lambda k, d=None: getattr(p, k, d))
    rho0, g = float(get("rho0", 1.0)), float(get("g_x", 0.0))
    half = 0.5 * g * (nx + 1) * 3.0
    return (rho0 - 1.0) + half, (rho0 - 1.0) - half


def gpbc_densities(p, nx: int):
    """The same densities as full values."""
    a, b = gpbc_density_offsets(p, nx)
    return 1.0 + a, 1.0 + b


def to_params(p, nx: int | None = None) -> OrcParams:
    """Accepts a mapping (or object) with tau_lb, g_x, G_inf, tau0, theta, gamma_c, rho0,
    stress_mode and optionally x_mode ("periodic" or "gpbc"; GPBC needs nx), top_wall
    ("bounce_back" or "moving": planar Couette flow with a Zou-He wall on the last row) and
    u_wall; scheme ("paper", "generalized_newtonian" or "stress_divergence", the comparison
    schemes of Sec. II C); beta_rho, rho_ref (density-dependent tau) and tau_f (memory time of the
    fluidity 1/tau_M), the relaxation-time extensions of the paper's outlook (off by default)."""
    get = (lambda k, d=None: p.get(k, d)) if isinstance(p, dict) else (lambda k, d=None: getattr(p, k, d))
    gpbc = get("x_mode", "periodic") == "gpbc"
    rin, rout = gpbc_density_offsets(p, nx) if gpbc else (0.0, 0.0)
    return OrcParams(float(get("tau_lb")), float(get("g_x", 0.0)), float(get("G_inf", 0.0)),
                     float(get("tau0", 0.0)), float(get("theta", 0.0)), float(get("gamma_c", np.inf)),
                     float(get("rho0", 1.0)), int(get("stress_mode", 0)), 1 if gpbc else 0, rin, rout,
                     1 if get("top_wall", "bounce_back") == "moving" else 0,
                     SCHEMES[get("scheme", "paper")], float(get("u_wall", 0.0)),
                     float(get("beta_rho", 0.0)), float(get("rho_ref", 1.0)), float(get("tau_f", 0.0)))


# --- per-node functions ---------------------------------------------------------------------

def equilibrium(rho: float, ux: float, uy: float) -> np.ndarray:
    """Eq. (neq) for one node -> n^eq_i, i = 0..8."""
    out = np.zeros(9)
    _load().orc_equilibrium(rho, ux, uy, _p(out))
    return out


def equilibrium_offset(rho_m1: float, ux: float, uy: float) -> np.ndarray:
    """Eq. (neq) minus the weights, from rho - 1 (the form the stepping uses)."""
    out = np.zeros(9)
    _load().orc_equilibrium_offset(rho_m1, ux, uy, _p(out))
    return out


WEIGHTS = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def forcing(tau_lb: float, sbar, S: float, u, f) -> np.ndarray:
    """Eq. (bodyforce) for one node; sbar = traceless Sigma^nN (xx, xy, yy), S = dt d_t delta rho."""
    out = np.zeros(9)
    _load().orc_forcing(tau_lb, _p(_vec(sbar, 3)), S, _p(_vec(u, 2)), _p(_vec(f, 2)), _p(out))
    return out


def relaxation_time(tau: float, gamma_c: float, II_D: float) -> float:
    """Eq. (nlmaxwell)."""
    return _load().orc_relaxation_time(tau, gamma_c, II_D)


def stress_series(kappa, tau_M: float, G: float):
    """Eq. (sigtsum) summed with Eq. (smalld); kappa = (xx, xy, yx, yy).  Returns (sigma(xx,xy,yy),
    number of terms), terms = -1 if the series is not used (not convergent)."""
    out = np.zeros(3)
    n = _load().orc_stress_series(_p(_vec(kappa, 4)), tau_M, G, _p(out))
    return out, n


def stress_gauss(kappa, tau_M: float, G: float) -> np.ndarray:
    out = np.zeros(3)
    rc = _load().orc_stress_gauss(_p(_vec(kappa, 4)), tau_M, G, _p(out))
    if rc != 0:
        raise ArithmeticError("singular stress system")
    return out


def stress_step(kappa, tau_M: float, G: float, s_old) -> np.ndarray:
    """Stress mode 1: one backward-Euler step (dt = 1) of Eq. (gkder) with the Maxwell memory."""
    out = np.zeros(3)
    rc = _load().orc_stress_step(_p(_vec(kappa, 4)), tau_M, G, _p(_vec(s_old, 3)), _p(out))
    if rc == -2:
        raise ArithmeticError("singular stress system")
    return out


def fallback_count() -> int:
    return int(_load().orc_fallback_count())


# --- whole-grid state -----------------------------------------------------------------------

def fluidity_step(phi_old: float, phi_ss: float, tau_f: float) -> float:
    """One backward-Euler step of the fluidity memory d phi/dt = (phi_ss - phi)/tau_f (dt = 1)."""
    return _load().orc_fluidity_step(phi_old, phi_ss, tau_f)


@dataclass
class State:
    dev: np.ndarray    # [9, ny, nx]  n*_i - w_i
    drho: np.ndarray   # [ny, nx]
    sig: np.ndarray    # [3, ny, nx]
    step: int = 0
    phi: np.ndarray = None  # [ny, nx] fluidity 1/tau_M of the memory model (0: not yet set)

    def __post_init__(self):
        if self.phi is None:
            self.phi = np.zeros(self.drho.shape)

    @property
    def shape(self):
        return self.drho.shape

    @property
    def nstar(self) -> np.ndarray:
        """Full post-collision populations n*_i (a new array)."""
        return self.dev + WEIGHTS[:, None, None]

    def copy(self) -> "State":
        return State(self.dev.copy(), self.drho.copy(), self.sig.copy(), self.step, self.phi.copy())


def init_state(rho: np.ndarray) -> State:
    """Rest equilibrium n*_i = w_i rho(r), drho = 0, sigma = 0 (initial state of the runs)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = rho.shape
    st = State(np.zeros((9, ny, nx)), np.zeros((ny, nx)), np.zeros((3, ny, nx)))
    _load().orc_init(nx, ny, _p(rho), _p(st.dev), _p(st.drho), _p(st.sig))
    return st


def state_from_populations(nstar: np.ndarray, drho: np.ndarray) -> State:
    nstar = np.asarray(nstar, dtype=np.float64)
    st = State(np.ascontiguousarray(nstar - WEIGHTS[:, None, None]), np.ascontiguousarray(drho, dtype=np.float64),
               np.zeros((3,) + nstar.shape[1:]))
    return st


def flow_state(rho: np.ndarray, ux: np.ndarray, uy: np.ndarray, g_x: float) -> State:
    """Equilibrium state whose current j = sum c n + f/2 equals rho*u (warm starts in tests)."""
    rho = np.asarray(rho, dtype=np.float64)
    ny, nx = rho.shape
    st = State(np.zeros((9, ny, nx)), np.zeros((ny, nx)), np.zeros((3, ny, nx)))
    for y in range(ny):
        for x in range(nx):
            st.dev[:, y, x] = equilibrium_offset(rho[y, x] - 1.0, ux[y, x] - 0.5 * g_x / rho[y, x], uy[y, x])
    return st


def run(params, st: State, nsteps: int, nthreads: int = 1) -> State:
    """Advance ``st`` in place by ``nsteps`` steps; returns it."""
    ny, nx = st.shape
    pp = to_params(params, nx)
    rc = _load().orc_run(ctypes.byref(pp), nx, ny, _p(st.dev), _p(st.drho), _p(st.sig), _p(st.phi),
                         int(nsteps), int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the grid or parameters")
    st.step += int(nsteps)
    return st


def fields(params, st: State):
    """(u[ny,nx,2], sigma[ny,nx,4] as xx,yy,zz,xy, rho[ny,nx]) of the state: the velocity,
    polymer stress and hydrodynamic density the next collision uses."""
    ny, nx = st.shape
    u = np.zeros((ny, nx, 2))
    sg = np.zeros((ny, nx, 4))
    rho = np.zeros((ny, nx))
    pp = to_params(params, nx)
    rc = _load().orc_fields(ctypes.byref(pp), nx, ny, _p(st.dev), _p(st.drho), _p(st.sig), _p(st.phi),
                            _p(u), _p(sg), _p(rho))
    if rc != 0:
        raise ValueError("oracle rejected the grid or parameters")
    return u, sg, rho


def intermediates(params, st: State) -> np.ndarray:
    """[ny, nx, 9]: kxx, kxy, kyx, kyy, tau_M, drho, S, rho_eq, tau_LB of the next update."""
    ny, nx = st.shape
    out = np.zeros((ny, nx, 9))
    pp = to_params(params, nx)
    rc = _load().orc_node_intermediates(ctypes.byref(pp), nx, ny, _p(st.dev), _p(st.drho),
                                        _p(st.sig), _p(st.phi), _p(out))
    if rc != 0:
        raise ValueError("oracle rejected the grid or parameters")
    return out


def mass(st: State) -> float:
    """Invariant of the scheme with periodic x and bounce-back walls, sum_r (sum_i n*_i - drho),
    minus the number of nodes (sum of the offsets, to keep the precision)."""
    return float(st.dev.sum() - st.drho.sum())


def residual(u_now: np.ndarray, u_prev: np.ndarray) -> float:
    """||u^t - u^{t-1}||_2 / ||u^t||_2 over a channel (the convergence measure of the runs)."""
    den = np.sqrt(np.sum(u_now * u_now))
    return float(np.sqrt(np.sum((u_now - u_prev) ** 2)) / den) if den > 0 else float("inf")


def run_to_steady(params, st: State, tol: float, check_every: int = 100, max_steps: int = 10**7,
                  nthreads: int = 1):
    """Step until the one-step velocity residual is <= tol (checked every ``check_every``)."""
    while st.step < max_steps:
        run(params, st, check_every - 1, nthreads)
        u_prev, _, _ = fields(params, st)
        run(params, st, 1, nthreads)
        u_now, _, _ = fields(params, st)
        r = residual(u_now, u_prev)
        if r <= tol:
            return st, r
    return st, r
