"""Thin ctypes binding of the C ABI in ``include/lbnlm.h`` (same names, argument marshalling only).

Every computation happens in ``liblbnlm.so`` (CUDA, sm_103a).  If the library has not been built
the import-time ``load()`` raises: there is no CPU fallback.

Functions mirror the C calls; a non-OK status raises :class:`LBError` (``lb_step`` returns
``LB_EUNSTABLE`` instead of raising, since the other channels keep running).  Arrays are NumPy
(host) or anything with a ``data_ptr()`` (device tensors) where the C call takes device memory.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, c_double, c_int, c_long, c_size_t, c_uint64, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblbnlm.so")

LB_OK, LB_EINVAL, LB_ENOMEM, LB_ECUDA, LB_EUNSTABLE, LB_ETIMEOUT, LB_ESTATE = range(7)
LB_PREC_F64, LB_PREC_F32, LB_PREC_BF16 = 0, 1, 2
LB_STRESS_INLM, LB_STRESS_TIMESTEPPED = 0, 1
LB_GRID_STORE_SIGMA, LB_GRID_TILE_ONLY, LB_GRID_BF16_STOCHASTIC, LB_GRID_NO_GRAPH = 1, 2, 4, 8
LB_GRID_GENERALIZED_NEWTONIAN, LB_GRID_STRESS_DIVERGENCE, LB_GRID_RELAXATION_MODEL = 16, 32, 64
SCHEME_FLAGS = {"paper": 0, "generalized_newtonian": LB_GRID_GENERALIZED_NEWTONIAN,
                "stress_divergence": LB_GRID_STRESS_DIVERGENCE}
LB_X_PERIODIC, LB_X_GPBC = 1, 2
X_MODES = {"periodic": LB_X_PERIODIC, "gpbc": LB_X_GPBC}
LB_WALLS_BOUNCE_BACK, LB_WALLS_COUETTE = 1, 2
LB_MONITOR_RESIDUAL, LB_MONITOR_FLUX_MAX = 0, 1
WALLS = {"bounce_back": LB_WALLS_BOUNCE_BACK, "couette": LB_WALLS_COUETTE}
LB_PREC_F64S_F32M, LB_PREC_F32S_F64M = 3, 4
PRECISIONS = {"f64": LB_PREC_F64, "f32": LB_PREC_F32, "bf16": LB_PREC_BF16, "f64s_f32m": LB_PREC_F64S_F32M,
              "f32s_f64m": LB_PREC_F32S_F64M}


class lb_grid(ctypes.Structure):
    _fields_ = [("n_channels", c_int), ("nx", c_int), ("ny", POINTER(c_int)), ("precision", c_int),
                ("stress_mode", c_int), ("flags", c_int)]


class lb_params(ctypes.Structure):
    _fields_ = [("tau_lb", c_double), ("g_x", c_double), ("G_inf", c_double), ("tau0", c_double),
                ("theta", c_double), ("gamma_c", c_double), ("rho0", c_double), ("rho_pert_amp", c_double),
                ("seed", c_uint64)]


class lb_boundary(ctypes.Structure):
    _fields_ = [("walls", c_int), ("x_mode", c_int)]


class LBError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


_lib = None
_D = POINTER(c_double)
_H = c_void_p


def load():
    """Load ``liblbnlm.so``; raises if it is missing (build it with ``paper_1310_7450_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing; run paper_1310_7450_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "lb_create": ([POINTER(lb_grid), POINTER(lb_params), POINTER(lb_boundary), c_void_p, POINTER(c_void_p)], c_int),
        "lb_step": ([_H, c_long], c_int),
        "lb_get_fields": ([_H, c_void_p, c_void_p, c_void_p, c_int, c_int], c_int),
        "lb_residual": ([_H, _D], c_int),
        "lb_monitor": ([_H, _D], c_int),
        "lb_monitor_async": ([_H, c_void_p], c_int),
        "lb_set_body_force": ([_H, c_int, c_double], c_int),
        "lb_set_wall_velocity": ([_H, c_int, c_double], c_int),
        "lb_set_fields": ([_H, _D, _D, _D], c_int),
        "lb_set_populations": ([_H, _D, _D, _D], c_int),
        "lb_get_populations": ([_H, _D, _D, _D], c_int),
        "lb_state_bytes": ([_H], c_size_t),
        "lb_get_state": ([_H, c_void_p, c_size_t], c_int),
        "lb_set_state": ([_H, c_void_p, c_size_t], c_int),
        "lb_channel_status": ([_H, POINTER(c_int)], c_int),
        "lb_set_wait_limit": ([_H, c_double], c_int),
        "lb_set_monitor_mode": ([_H, c_int], c_int),
        "lb_set_relaxation_model": ([_H, c_int, c_double, c_double, c_double], c_int),
        "lb_warmstart_apply": ([_H, c_void_p, c_void_p, c_void_p], c_int),
        "lb_warmstart_targets": ([_H, c_void_p], c_int),
        "lb_step_count": ([_H], c_long),
        "lb_mlp_create": ([c_int, c_int, c_int, c_int, c_uint64, c_void_p, POINTER(c_void_p)], c_int),
        "lb_mlp_destroy": ([_H], None),
        "lb_mlp_num_params": ([_H], ctypes.c_longlong),
        "lb_mlp_forward": ([_H, c_void_p, c_int, c_void_p], c_int),
        "lb_mlp_gradients": ([_H, c_void_p, c_void_p, c_int, c_void_p, POINTER(c_double)], c_int),
        "lb_mlp_train_step": ([_H, c_void_p, c_void_p, c_int, ctypes.c_float, POINTER(c_double)], c_int),
        "lb_mlp_get_params": ([_H, c_void_p], c_int),
        "lb_mlp_set_params": ([_H, c_void_p], c_int),
        "lb_run_until_steady": ([_H, c_double, c_long, c_long, c_void_p, c_void_p], c_int),
        "lb_sweep_config": ([_H, POINTER(c_int), POINTER(c_int), POINTER(c_double)], c_int),
        "lb_sweep_variant": ([_H], c_int),
        "lb_sweep_groups": ([_H, POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int), c_int], c_int),
        "lb_sweep_set_config": ([_H, c_int, c_int, c_int], c_int),
        "lb_sweep_tune": ([_H], c_int),
        "lb_field_monitor_static": ([c_void_p, c_void_p, c_int, c_int, c_void_p, c_int, c_void_p, c_void_p], c_int),
        "lb_uses_row_march": ([_H], c_int),
        "lb_row_march_plan": ([c_int, c_int, c_int, c_int, c_int, c_int, c_void_p, c_int], c_int),
        "lb_graph_replays": ([_H], c_long),
        "lb_num_nodes": ([_H], c_size_t),
        "lb_destroy": ([_H], None),
        "lb_strerror": ([c_int], ctypes.c_char_p),
        "lb_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != LB_OK:
        raise LBError(status, where, load().lb_last_error().decode())
    return status


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "expected a C-contiguous float64 array"
    return a.ctypes.data_as(_D)


def _ptr(a):
    """Host NumPy array or device tensor -> void*."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return c_void_p(a.ctypes.data)
    return c_void_p(a.data_ptr())


def make_params(p: dict, rho_pert_amp: float = 0.0, seed: int = 0) -> lb_params:
    return lb_params(float(p["tau_lb"]), float(p.get("g_x", 0.0)), float(p.get("G_inf", 0.0)),
                     float(p.get("tau0", 0.0)), float(p.get("theta", 0.0)), float(p.get("gamma_c", math.inf)),
                     float(p.get("rho0", 1.0)), float(p.get("rho_pert_amp", rho_pert_amp)),
                     int(p.get("seed", seed)))


# ---- the C calls ---------------------------------------------------------------------------

def lb_create(nx: int, ny, params, precision: int = LB_PREC_F64, stress_mode: int = LB_STRESS_INLM,
              flags: int = 0, stream: int | None = None, x_mode: int = LB_X_PERIODIC,
              walls: int = LB_WALLS_BOUNCE_BACK) -> int:
    """ny: int or list per channel; params: dict / lb_params or a list of them (one per channel);
    x_mode: LB_X_PERIODIC (body-force driven) or LB_X_GPBC (pressure-driven); walls:
    LB_WALLS_BOUNCE_BACK or LB_WALLS_COUETTE (moving top wall)."""
    lib = load()
    nys = [int(ny)] if np.isscalar(ny) else [int(v) for v in ny]
    plist = params if isinstance(params, (list, tuple)) else [params] * len(nys)
    arr = (lb_params * len(nys))(*[p if isinstance(p, lb_params) else make_params(p) for p in plist])
    nyarr = (c_int * len(nys))(*nys)
    grid = lb_grid(len(nys), int(nx), nyarr, int(precision), int(stress_mode), int(flags))
    bnd = lb_boundary(int(walls), int(x_mode))
    h = c_void_p()
    _check(lib.lb_create(ctypes.byref(grid), arr, ctypes.byref(bnd), c_void_p(stream or 0), ctypes.byref(h)),
           "lb_create")
    return h.value


def lb_step(h: int, n: int) -> int:
    st = load().lb_step(h, int(n))
    if st not in (LB_OK, LB_EUNSTABLE):
        _check(st, "lb_step")
    return st


def lb_get_fields(h: int, u=None, sigma=None, rho=None, out_dtype: int = 0, on_device: bool = False):
    _check(load().lb_get_fields(h, _ptr(u), _ptr(sigma), _ptr(rho), int(out_dtype), int(bool(on_device))),
           "lb_get_fields")


def lb_residual(h: int, out: np.ndarray):
    _check(load().lb_residual(h, _dp(out)), "lb_residual")


def lb_monitor(h: int, out: np.ndarray):
    _check(load().lb_monitor(h, _dp(out)), "lb_monitor")


def lb_monitor_async(h: int, out):
    """out: a pinned host tensor / array or a device tensor of n_channels * 4 doubles."""
    _check(load().lb_monitor_async(h, _ptr(out)), "lb_monitor_async")


def lb_set_body_force(h: int, channel: int, g_x: float):
    _check(load().lb_set_body_force(h, int(channel), float(g_x)), "lb_set_body_force")


def lb_set_wall_velocity(h: int, channel: int, u_wall: float):
    _check(load().lb_set_wall_velocity(h, int(channel), float(u_wall)), "lb_set_wall_velocity")


def lb_set_fields(h: int, u: np.ndarray, rho: np.ndarray, drho: np.ndarray | None = None):
    _check(load().lb_set_fields(h, _dp(u), _dp(rho), _dp(drho)), "lb_set_fields")


def lb_set_populations(h: int, n: np.ndarray, drho: np.ndarray, sig3: np.ndarray | None = None):
    _check(load().lb_set_populations(h, _dp(n), _dp(drho), _dp(sig3)), "lb_set_populations")


def lb_get_populations(h: int, n: np.ndarray, drho: np.ndarray, sig3: np.ndarray | None = None):
    _check(load().lb_get_populations(h, _dp(n), _dp(drho), _dp(sig3)), "lb_get_populations")


def lb_state_bytes(h: int) -> int:
    return int(load().lb_state_bytes(h))


def lb_get_state(h: int, buf: np.ndarray):
    _check(load().lb_get_state(h, c_void_p(buf.ctypes.data), buf.nbytes), "lb_get_state")


def lb_set_state(h: int, buf: np.ndarray):
    _check(load().lb_set_state(h, c_void_p(buf.ctypes.data), buf.nbytes), "lb_set_state")


def _dev(t):
    """Device address of a CUDA tensor (or None)."""
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous()
    return c_void_p(t.data_ptr())


def lb_warmstart_apply(h: int, pred=None, t_mu=None, t_sd=None):
    """pred: CUDA float32 [n_channels, 768] network outputs (or None: the closed form); t_mu, t_sd:
    CUDA float32 [768] de-standardisation (both or neither)."""
    _check(load().lb_warmstart_apply(h, _dev(pred), _dev(t_mu), _dev(t_sd)), "lb_warmstart_apply")


def lb_warmstart_targets(h: int, targets):
    """targets: CUDA float32 [n_channels, 768], filled on the handle's stream."""
    _check(load().lb_warmstart_targets(h, _dev(targets)), "lb_warmstart_targets")


def lb_set_relaxation_model(h: int, channel: int, beta_rho: float, rho_ref: float, tau_f: float):
    _check(load().lb_set_relaxation_model(h, int(channel), float(beta_rho), float(rho_ref), float(tau_f)),
           "lb_set_relaxation_model")


def lb_set_monitor_mode(h: int, mode: int):
    _check(load().lb_set_monitor_mode(h, int(mode)), "lb_set_monitor_mode")


def lb_set_wait_limit(h: int, seconds: float):
    _check(load().lb_set_wait_limit(h, float(seconds)), "lb_set_wait_limit")


def lb_channel_status(h: int, out: np.ndarray):
    assert out.dtype == np.int32
    _check(load().lb_channel_status(h, out.ctypes.data_as(POINTER(c_int))), "lb_channel_status")


def lb_field_monitor_static(u_now, u_prev, dtype: int, n_channels: int, node_offsets, nx: int, out, stream=None):
    """Device tensors in, device tensor out (see include/lbnlm.h); allocates nothing."""
    _check(load().lb_field_monitor_static(_ptr(u_now), _ptr(u_prev), int(dtype), int(n_channels), _ptr(node_offsets),
                                          int(nx), _ptr(out), c_void_p(stream or 0)), "lb_field_monitor_static")


def lb_run_until_steady(h: int, tol: float, check_every: int, max_steps: int, steps_out=None, residual_out=None):
    """steps_out: int64 [n_channels], residual_out: float64 [n_channels] (host NumPy, optional)."""
    if steps_out is not None:
        assert steps_out.dtype == np.int64
    _check(load().lb_run_until_steady(h, float(tol), int(check_every), int(max_steps), _ptr(steps_out),
                                      _ptr(residual_out)), "lb_run_until_steady")


def lb_sweep_tune(h: int):
    _check(load().lb_sweep_tune(h), "lb_sweep_tune")


def lb_sweep_config(h: int):
    nt, cl, ms = c_int(), c_int(), c_double()
    _check(load().lb_sweep_config(h, ctypes.byref(nt), ctypes.byref(cl), ctypes.byref(ms)), "lb_sweep_config")
    return nt.value, cl.value, ms.value


def lb_sweep_variant(h: int) -> int:
    return int(load().lb_sweep_variant(h))


def lb_sweep_groups(h: int):
    """[(kernel variant, threads, cluster, channels)] per width class of the sweep."""
    n = int(load().lb_sweep_groups(h, None, None, None, None, 0))
    if n <= 0:
        return []
    v, t, c, k = (c_int * n)(), (c_int * n)(), (c_int * n)(), (c_int * n)()
    load().lb_sweep_groups(h, v, t, c, k, n)
    return [(v[i], t[i], c[i], k[i]) for i in range(n)]


def lb_sweep_set_config(h: int, variant: int, threads: int, cluster: int):
    _check(load().lb_sweep_set_config(h, int(variant), int(threads), int(cluster)), "lb_sweep_set_config")


def lb_mlp_create(n_in: int, width: int, n_out: int, max_batch: int, seed: int = 0, stream=None) -> int:
    m = c_void_p()
    _check(load().lb_mlp_create(int(n_in), int(width), int(n_out), int(max_batch), int(seed), c_void_p(stream or 0),
                                ctypes.byref(m)), "lb_mlp_create")
    return m.value


def lb_mlp_destroy(m: int):
    load().lb_mlp_destroy(m)


def lb_mlp_num_params(m: int) -> int:
    return int(load().lb_mlp_num_params(m))


def lb_mlp_forward(m: int, x, batch: int, y):
    _check(load().lb_mlp_forward(m, _ptr(x), int(batch), _ptr(y)), "lb_mlp_forward")


def lb_mlp_gradients(m: int, x, target, batch: int, grads=None) -> float:
    loss = c_double()
    _check(load().lb_mlp_gradients(m, _ptr(x), _ptr(target), int(batch), _ptr(grads), ctypes.byref(loss)),
           "lb_mlp_gradients")
    return loss.value


def lb_mlp_train_step(m: int, x, target, batch: int, lr: float, want_loss: bool = True):
    loss = c_double()
    _check(load().lb_mlp_train_step(m, _ptr(x), _ptr(target), int(batch), ctypes.c_float(lr),
                                    ctypes.byref(loss) if want_loss else None), "lb_mlp_train_step")
    return loss.value if want_loss else None


def lb_mlp_get_params(m: int, host: np.ndarray):
    assert host.dtype == np.float32
    _check(load().lb_mlp_get_params(m, c_void_p(host.ctypes.data)), "lb_mlp_get_params")


def lb_mlp_set_params(m: int, host: np.ndarray):
    assert host.dtype == np.float32 and host.flags["C_CONTIGUOUS"]
    _check(load().lb_mlp_set_params(m, c_void_p(host.ctypes.data)), "lb_mlp_set_params")


def lb_step_count(h: int) -> int:
    return int(load().lb_step_count(h))


def lb_uses_row_march(h: int) -> bool:
    return bool(load().lb_uses_row_march(h))


def lb_row_march_plan(nx: int, ny: int, ctas_per_sm: int, n_sm: int, precision="f32", gpbc: bool = False) -> np.ndarray:
    """The row-march kernel's work items for a single nx x ny channel: an int32 array [n, 3] of
    (x0, y0, y1) (host computation; no GPU needed)."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    lib = load()
    n = lib.lb_row_march_plan(nx, ny, ctas_per_sm, n_sm, prec, int(bool(gpbc)), None, 0)
    if n < 0:
        _check(-n, "lb_row_march_plan")
    out = np.zeros((max(n, 1), 3), dtype=np.int32)
    m = lib.lb_row_march_plan(nx, ny, ctas_per_sm, n_sm, prec, int(bool(gpbc)), out.ctypes.data, n)
    if m < 0:
        _check(-m, "lb_row_march_plan")
    return out[:m]


def lb_graph_replays(h: int) -> int:
    return int(load().lb_graph_replays(h))


def lb_num_nodes(h: int) -> int:
    return int(load().lb_num_nodes(h))


def lb_destroy(h: int):
    load().lb_destroy(h)


def lb_strerror(status: int) -> str:
    return load().lb_strerror(int(status)).decode()


def lb_last_error() -> str:
    return load().lb_last_error().decode()


# ---- convenience (marshalling only) ----------------------------------------------------------

class Channels:
    """Owns one handle; returns fields as NumPy arrays shaped per channel."""

    def __init__(self, nx, ny, params, precision="f64", stress_mode=0, flags=0, stream=None, x_mode="periodic",
                 walls="bounce_back", scheme="paper"):
        self.nx = int(nx)
        self.ny = [int(ny)] if np.isscalar(ny) else [int(v) for v in ny]
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        xm = X_MODES[x_mode] if isinstance(x_mode, str) else int(x_mode)
        wl = WALLS[walls] if isinstance(walls, str) else int(walls)
        flags = int(flags) | SCHEME_FLAGS[scheme]
        self.h = lb_create(self.nx, self.ny, params, prec, stress_mode, flags, stream, xm, wl)
        self.nodes = lb_num_nodes(self.h)

    def close(self):
        if self.h:
            lb_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n):
        return lb_step(self.h, n)

    def _split(self, flat, k):
        out, o = [], 0
        for ny in self.ny:
            n = ny * self.nx
            out.append(flat[o:o + n].reshape((ny, self.nx) + ((k,) if k > 1 else ())))
            o += n
        return out

    def fields(self):
        """Per channel: (u [ny,nx,2], sigma [ny,nx,4] as xx,yy,zz,xy, rho [ny,nx]) in float64."""
        u = np.zeros(2 * self.nodes)
        s = np.zeros(4 * self.nodes)
        r = np.zeros(self.nodes)
        lb_get_fields(self.h, u, s, r, 0, False)
        return list(zip(self._split(u.reshape(-1, 2), 2), self._split(s.reshape(-1, 4), 4), self._split(r, 1)))

    def populations(self):
        """Per channel: (n [9,ny,nx] full FP64 values, drho [ny,nx])."""
        n = np.zeros(9 * self.nodes)
        d = np.zeros(self.nodes)
        lb_get_populations(self.h, n, d, None)
        out, o, k = [], 0, 0
        for ny in self.ny:
            m = ny * self.nx
            out.append((n[o:o + 9 * m].reshape(9, ny, self.nx), d[k:k + m].reshape(ny, self.nx)))
            o += 9 * m
            k += m
        return out

    def set_populations(self, pops, drhos, sig3s=None):
        n = np.concatenate([np.ascontiguousarray(p, dtype=np.float64).reshape(-1) for p in pops])
        d = np.concatenate([np.ascontiguousarray(x, dtype=np.float64).reshape(-1) for x in drhos])
        s = None
        if sig3s is not None:
            s = np.concatenate([np.ascontiguousarray(x, dtype=np.float64).reshape(-1) for x in sig3s])
        lb_set_populations(self.h, n, d, s)

    def run_until_steady(self, tol, check_every=100, max_steps=10**7):
        """Per channel (steps, residual) of the persistent sweep."""
        steps = np.zeros(len(self.ny), dtype=np.int64)
        res = np.zeros(len(self.ny))
        lb_run_until_steady(self.h, tol, check_every, max_steps, steps, res)
        return steps, res

    def monitor(self):
        m = np.zeros(4 * len(self.ny))
        lb_monitor(self.h, m)
        return m.reshape(-1, 4)

    def residual(self):
        r = np.zeros(len(self.ny))
        lb_residual(self.h, r)
        return r

    def status(self):
        s = np.zeros(len(self.ny), dtype=np.int32)
        lb_channel_status(self.h, s)
        return s
