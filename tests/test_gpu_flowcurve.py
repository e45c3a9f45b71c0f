"""Flow curves from the GPU runs against the closed forms of Sec. III A: homogeneous planar Couette
shear reproduces sigma_xy = G gdot tau_M and N1 = 2 G gdot^2 tau_M^2 over five decades of shear
rate (exact for a linear profile), and the local (gdot, sigma_xy) data of a steady yield-stress
channel collapse onto the same flow curve (the paper's channel-data comparison)."""
import numpy as np
import pytest

import oracle
from oracle import analytic
from paper_1310_7450_gb300 import flowcurve, inputs, lbnlm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stream():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("theta", [0.0, 10.0, 100.0])
def test_couette_flow_curve_matches_closed_form(stream, theta):
    G = 1e-3
    p = inputs.matched_params(0.9, theta, 0.1, G, 0.0)
    gdots = np.logspace(-8, -3, 11)
    g, g_rep, sxy, n1, steps = flowcurve.couette(gdots, p, stream=stream)
    assert np.abs(g / gdots - 1).max() < 1e-14
    assert np.abs(g_rep / g - 1).max() < 1e-4       # flow-induced density factor (~1.5 N1)
    ref = np.array([analytic.simple_shear(gd, G, theta * p["tau0"], 0.1) for gd in g])
    if theta == 0.0:
        assert np.abs(sxy).max() < 1e-15 and np.abs(n1).max() < 1e-15
    else:
        assert np.abs(sxy / ref[:, 0] - 1).max() < 1e-9
        assert np.abs(n1 / ref[:, 1] - 1).max() < 1e-8


def test_channel_data_collapse_onto_the_flow_curve(stream):
    """Steady 4 x 64 yield-stress channel (theta = 100) started from the closed-form profile: in the
    yielded rows, sigma_xy(gdot) of the LB fields lies on the simple-shear flow curve."""
    cfg = inputs.oracle_channel_yield()
    nx, ny, p = cfg["nx"], cfg["ny"], cfg["params"]
    ua = analytic.channel_profile(ny, p["g_x"], p["G_inf"], p["tau0"], p["theta"], p["gamma_c"])
    with lbnlm.Channels(nx, ny, p, "f64", stream=stream) as sim:
        u0 = np.zeros((ny, nx, 2))
        u0[..., 0] = ua[:, None]
        lbnlm.lb_set_fields(sim.h, np.ascontiguousarray(u0.reshape(-1)), np.ones(nx * ny))
        sim.step(400000)
        (u, s, _), = sim.fields()
    gd, sxy, n1 = flowcurve.from_channel(u, s)
    tau = p["theta"] * p["tau0"]
    yielded = np.abs(gd) * tau > 10.0      # well outside the plug
    assert yielded.sum() >= 20
    ref = np.array([analytic.simple_shear(x, p["G_inf"], tau, p["gamma_c"])[0] for x in gd[yielded]])
    assert np.abs(sxy[yielded] / ref - 1).max() < 1e-3
