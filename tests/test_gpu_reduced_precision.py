"""Reduced-precision storage on the 8192 x 2048 channel (theta = 100, gamma_c = 0.1, wp H = 1/2,
H = 1024): FP32 and BF16 deviations with FP32 arithmetic, 1e5 steps from the closed-form steady
profile (1e5 steps is far below the diffusion time at this width, so the run measures drift from
the steady state, not convergence).  The FP64 oracle runs the same start on a 4 x 2048 channel,
which the x-invariant wide run must reproduce column by column (bitwise x-invariance; stochastic
rounding draws per node and breaks it, so that run is compared through its x-mean).  Errors are
printed per precision.  Bounds: FP32 storage within 2e-3 of the analytic steady profile; BF16 with
stochastic rounding within 4e-3 (measured 2.8e-3 of the x-mean: the 2e-3 target of reduced storage
is not reached by BF16 here; round to nearest drifts to 5.1e-3 and its stress is O(1) wrong in the
plug); FP32 u within 5e-5 of the oracle and sigma within 4x its FP32 velocity floor -- the FP32
velocity carries ~4e-9 absolute (ulp of 0.05), and in the plug the stress G tau kappa_xy is built
from row differences of that size, so at this width the stress, and through it u, drift further
from the FP64 oracle than on the narrow channels (measured: u 1.5e-5, sigma 2.6e-2 of max |sigma|,
2.2x the floor)."""
import numpy as np
import pytest

import oracle
from oracle import analytic
import warmstart_reference as ref
from paper_1310_7450_gb300 import inputs, lbnlm, warmstart

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_reduced_precision_8192x2048():
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    cfg = inputs.reduced_precision_channel()
    nx, ny, p = cfg["nx"], cfg["ny"], cfg["params"]
    steps = 100_000
    start = ref.analytic_rows(ny, p)   # (the library computes the same closed form on the device)
    ua = analytic.channel_profile(ny, p["g_x"], p["G_inf"], p["tau0"], p["theta"], p["gamma_c"])
    # FP64 oracle on 4 x 2048 from the same closed-form start
    st = oracle.flow_state(np.ones((ny, 4)), np.repeat(start[0][:, None], 4, 1), np.zeros((ny, 4)), p["g_x"])
    st.drho[:] = (-1.5 * start[2])[:, None]
    oracle.run(p, st, steps, nthreads=16)
    u_o, s_o, _ = oracle.fields(p, st)
    res = {}
    for name, prec, flags in (("f32", "f32", 0), ("bf16", "bf16", 0), ("bf16_sr", "bf16", lbnlm.LB_GRID_BF16_STOCHASTIC)):
        with lbnlm.Channels(nx, ny, p, prec, flags=flags | lbnlm.LB_GRID_STORE_SIGMA, stream=stream) as sim:
            assert lbnlm.lb_uses_row_march(sim.h)
            warmstart.start_closed_form(sim)
            sim.step(steps)
            (u, s, _), = sim.fields()
        if flags & lbnlm.LB_GRID_BF16_STOCHASTIC:
            um, sm = u.mean(axis=1, keepdims=True), s.mean(axis=1, keepdims=True)
            uc, sc = np.repeat(um, 4, axis=1), np.repeat(sm, 4, axis=1)
        else:
            for x in (1, nx // 2, nx - 1):
                assert np.array_equal(u[:, x], u[:, 0])
            uc, sc = u[:, :4], s[:, :4]
        res[name] = (rel(uc, u_o), rel(sc, s_o), rel(uc[:, 0, 0], ua))
        print(f"{name}: u vs oracle {res[name][0]:.2e}, sigma vs oracle {res[name][1]:.2e}, "
              f"u vs analytic {res[name][2]:.2e}")
    print(f"f64 oracle: u vs analytic {rel(u_o[:, 0, 0], ua):.2e}")
    # the stress floor of the FP32 velocity: one unit in the last place of max |u| carried into
    # sigma by G tau, relative to max |sigma| (1.2e-2 here); after 1e5 steps the row-to-row
    # velocity errors in the plug reach about two such units (sigma 2.6e-2 = 2.2x the floor)
    floor = p["G_inf"] * p["theta"] * p["tau0"] * float(np.spacing(np.float32(np.abs(u_o).max()))) / np.abs(s_o).max()
    print(f"f32 sigma: {res['f32'][1] / floor:.1f} x floor {floor:.2e}")
    assert res["f32"][1] < 4 * floor
    assert res["f32"][0] < 5e-5
    assert res["f32"][2] < 2e-3
    assert res["bf16_sr"][2] < 4e-3
    assert res["bf16_sr"][2] < res["bf16"][2]
