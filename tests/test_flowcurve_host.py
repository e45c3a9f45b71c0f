"""flowcurve.from_channel (host post-processing of a channel state into local flow-curve points) on
an oracle channel.  In stress mode A the nlM stress is an instantaneous function of kappa
(Eq. sigtsum), and a channel is in simple shear row by row (kappa_xy = d_y u_x, the other
components 0), so every interior row must satisfy the Sec. III A closed forms sigma_xy = G gdot
tau_M(gdot) and N1 = 2 G gdot^2 tau_M^2 at any time of the start-up -- a wrong stress component, a
wrong stencil or an off-by-one row fails it."""
import numpy as np
import pytest

import oracle
from oracle import analytic
from paper_1310_7450_gb300 import flowcurve, inputs


@pytest.mark.parametrize("theta", [10.0, 100.0])
def test_from_channel_points_lie_on_the_flow_curve(theta):
    p = inputs.matched_params(0.9, theta, 0.1, 1e-3, 1e-6)
    nx, ny = 4, 32
    st = oracle.init_state(np.ones((ny, nx)))
    oracle.run(p, st, 3000)
    u, sigma, _ = oracle.fields(p, st)
    gd, sxy, n1 = flowcurve.from_channel(u, sigma)
    assert gd.shape == sxy.shape == n1.shape == (ny - 2,)
    # the start-up has developed a shear profile, antisymmetric about the centre line
    assert np.abs(gd).max() > 1e-7
    np.testing.assert_allclose(gd, -gd[::-1], rtol=0, atol=1e-12 * np.abs(gd).max())
    tau = p["theta"] * p["tau0"]
    for g, s, n in zip(gd, sxy, n1):
        want_s, want_n, _ = analytic.simple_shear(g, p["G_inf"], tau, p["gamma_c"])
        # gdot here is the difference of the reported velocity j / (rho - delta rho); the stress
        # saw the gradient velocity j / sum n: they differ by the flow-induced density, ~1e-6
        assert s == pytest.approx(want_s, rel=1e-5, abs=1e-9 * abs(sxy).max())
        assert n == pytest.approx(want_n, rel=2e-5, abs=1e-9 * abs(n1).max())
