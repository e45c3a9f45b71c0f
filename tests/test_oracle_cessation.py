"""Cessation of the yield-stress channel (Sec. IV B, the stopping-time phenomenon): qualitative pin
(the paper's stopping time 0.016 tau0 has no stated units, so its value stays unpinned).

A channel relaxed to its steady state is let go (g = 0).  A Newtonian fluid decays exponentially:
each factor of 100 in the mid-channel velocity takes the same time.  The yield-stress fluid
(theta = 100, and already theta = 10) keeps decelerating under a wall stress near the yield
stress and then drops to rest: the last two decades take a small fraction of the time the first
two took."""
import numpy as np
import pytest

from oracle import analytic
from paper_1310_7450_gb300 import inputs


def decay_times(oracle_mod, p, ny=32, every=500, levels=(1e-2, 1e-4), cap=400000):
    ua = analytic.channel_profile(ny, p["g_x"], p["G_inf"], p["tau0"], p["theta"], p["gamma_c"])
    st = oracle_mod.flow_state(np.ones((ny, 1)), ua[:, None], np.zeros((ny, 1)), p["g_x"])
    oracle_mod.run(p, st, 200000)                  # steady (residual < 1e-12 at this width)
    u0 = oracle_mod.fields(p, st)[0][ny // 2, 0, 0]
    pc = dict(p, g_x=0.0)
    out, T = {}, 0
    while T < cap and len(out) < len(levels):
        oracle_mod.run(pc, st, every)
        T += every
        um = oracle_mod.fields(pc, st)[0][ny // 2, 0, 0]
        for lv in levels:
            if lv not in out and um < lv * u0:
                out[lv] = T
    return out


def yield_channel(ny, theta):
    return inputs.yield_stress_channel(ny, theta=theta, tau=theta * 100.0, wpH=0.5)


@pytest.mark.parametrize("theta", [10.0, 100.0])
def test_yield_stress_channel_stops_while_newtonian_decays_exponentially(oracle_mod, theta):
    t = decay_times(oracle_mod, yield_channel(32, theta))
    p100 = yield_channel(32, 100.0)
    tn = decay_times(oracle_mod, inputs.matched_params(0.9, 0.0, 0.1, p100["G_inf"], p100["g_x"]))
    # Newtonian: the second pair of decades takes as long as the first (exponential)
    assert 0.6 <= (tn[1e-4] - tn[1e-2]) / tn[1e-2] <= 1.5
    # yield stress: the second pair takes a small fraction of the first (finite-time stop)
    assert (t[1e-4] - t[1e-2]) / t[1e-2] <= 0.35
