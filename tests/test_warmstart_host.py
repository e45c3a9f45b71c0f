"""The NumPy reference of the warm start's profile arithmetic (the library runs it on the device;
tests/warmstart_reference.py): its closed-form initial profile (a trapezoid evaluation of the steady
channel solution) against the oracle's adaptive quadrature, and the target encoding round trip;
the network features."""
import numpy as np
import pytest

import warmstart_reference as ref
from oracle import analytic
from paper_1310_7450_gb300 import inputs, warmstart


@pytest.mark.parametrize("theta,wpH", [(0.0, 0.5), (10.0, 0.5), (100.0, 0.5), (500.0, 3.0), (20.0, 0.02)])
def test_closed_form_start_matches_oracle_quadrature(theta, wpH):
    ny = 64
    G = 1e-4
    p = inputs.matched_params(0.9, theta, 0.1, G, wpH * G / (ny / 2))
    u, sxy, n1 = ref.analytic_rows(ny, p)
    ua = analytic.channel_profile(ny, p["g_x"], G, p["tau0"], theta, 0.1)
    assert np.abs(u - ua).max() <= 2e-4 * np.abs(ua).max()
    gd = analytic.channel_shear_rate(ny, p["g_x"], G, p["tau0"], theta, 0.1)
    for k in range(ny):
        s_ref, n1_ref, _ = analytic.simple_shear(gd[k], G, theta * p["tau0"], 0.1)
        assert sxy[k] == pytest.approx(s_ref, rel=1e-3, abs=1e-3 * G * 0.1)
        assert n1[k] == pytest.approx(n1_ref, rel=2e-3, abs=1e-4 * G * 0.01)


def test_encode_decode_roundtrip():
    rng = np.random.default_rng(2)
    nys = [33, 200, 1024]
    ps = [inputs.matched_params(0.9, 50.0, 0.1, 1e-4, 1e-7) for _ in nys]
    us = [rng.uniform(0, 1, n) for n in nys]
    ss = [rng.uniform(-1, 1, n) for n in nys]
    ns = [rng.uniform(0, 1, n) for n in nys]
    Y = ref.encode_targets(nys, ps, us, ss, ns)
    assert Y.shape == (3, 3 * warmstart.NPTS) and ref.NPTS == warmstart.NPTS
    back = ref.decode(nys, ps, Y)
    for k, ny in enumerate(nys):
        for j, src in enumerate((us, ss, ns)):
            np.testing.assert_allclose(back[k][j], ref.to_grid(src[k], ny), rtol=1e-10, atol=1e-12 * np.abs(src[k]).max())
    # a zero prediction is the closed-form start
    zero = ref.decode(nys, ps, np.zeros_like(Y))
    for k, ny in enumerate(nys):
        np.testing.assert_allclose(zero[k][0], ref.to_grid(ref.analytic_rows(ny, ps[k])[0], ny), rtol=1e-12)
    X = warmstart.features(nys, ps)
    assert X.shape == (3, 4) and np.all(np.isfinite(X))
