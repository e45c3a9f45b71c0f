"""GPU parity of the comparison schemes of Sec. II C (generalized-Newtonian tau_LB(gdot); the
divergence of Sigma^nN as a force density) against the FP64 oracle, through the C ABI.

FP64 within 1e-12 on random states over grids with several tiles, ragged tails and the degenerate
widths nx = 1, 2, and on channels from rest; FP32 within 1e-5 on u, and on the stress within 1e-5
or 1.5x the stress floor of the FP32 velocity (one unit in the last place of max |u| carried into
sigma by G tau, relative to max |sigma|), whichever is larger.
"""
import numpy as np
import pytest

import oracle
from paper_1310_7450_gb300 import inputs, lbnlm

pytestmark = pytest.mark.gpu
SCHEMES = ["generalized_newtonian", "stress_divergence"]


@pytest.fixture(scope="module")
def stream():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch.cuda.current_stream().cuda_stream


def rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def random_state(nx, ny, seed, amp=1e-2):
    rng = np.random.default_rng(seed)
    st = oracle.init_state(1.0 + amp * rng.uniform(-1, 1, (ny, nx)))
    w = oracle.equilibrium(1.0, 0.0, 0.0)
    st.dev += amp * rng.uniform(-1, 1, st.dev.shape) * w[:, None, None]
    return st


def nlm(theta=10.0, g=1e-5, G=1e-3):
    return inputs.matched_params(0.9, theta, 0.1, G, g)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("nx,ny", [(4, 200), (40, 13), (70, 29), (1, 10), (2, 3), (129, 7)])
def test_fp64_random_state_matches_oracle(stream, scheme, nx, ny):
    p = dict(nlm(), scheme=scheme)
    st = random_state(nx, ny, 500 + nx * 3 + ny)
    with lbnlm.Channels(nx, ny, p, "f64", stream=stream, scheme=scheme) as sim:
        assert not lbnlm.lb_uses_row_march(sim.h)
        sim.set_populations([st.nstar], [st.drho])
        sim.step(30)
        (n_g, d_g), = sim.populations()
        (u_g, s_g, r_g), = sim.fields()
    oracle.run(p, st, 30)
    u_o, s_o, r_o = oracle.fields(p, st)
    assert rel(n_g, st.nstar) < 1e-14
    assert np.all(d_g == 0.0) and np.all(st.drho == 0.0)
    assert rel(u_g, u_o) < 1e-12
    assert rel(s_g, s_o) < 1e-11
    assert np.abs(r_g - r_o).max() < 1e-14


@pytest.mark.parametrize("scheme", SCHEMES)
def test_fp64_channels_from_rest_match_oracle(stream, scheme):
    """Three channels of different widths and parameters in one handle, 3000 steps from rest (runs
    of plain steps replay a captured graph, which for the divergence scheme holds both launches)."""
    nys = [24, 37, 64]
    ps = [dict(nlm(10.0, 2e-6), scheme=scheme), dict(nlm(100.0, 1e-6, 2e-3), scheme=scheme),
          dict(nlm(0.0, 3e-6), scheme=scheme)]
    with lbnlm.Channels(4, nys, ps, "f64", stream=stream, scheme=scheme) as sim:
        sim.step(3000)
        assert lbnlm.lb_graph_replays(sim.h) > 0
        fields = sim.fields()
    for ny, p, (u_g, s_g, _) in zip(nys, ps, fields):
        st = oracle.init_state(np.ones((ny, 4)))
        oracle.run(p, st, 3000)
        u_o, s_o, _ = oracle.fields(p, st)
        assert np.abs(u_o).max() > 1e-5
        assert rel(u_g, u_o) < 1e-12
        if p["theta"] > 0:
            assert rel(s_g, s_o) < 1e-11


@pytest.mark.parametrize("scheme", SCHEMES)
def test_fp32_yield_stress_channel(stream, scheme):
    """4 x 64 yield-stress channel (theta = 100, tau = 1e4), 20000 steps from rest, FP32."""
    cfg = inputs.oracle_channel_yield()
    p = dict(cfg["params"], scheme=scheme)
    nx, ny, steps = cfg["nx"], cfg["ny"], cfg["steps"]
    with lbnlm.Channels(nx, ny, p, "f32", stream=stream, scheme=scheme) as sim:
        sim.step(steps)
        (u_g, s_g, _), = sim.fields()
    st = oracle.init_state(np.ones((ny, nx)))
    oracle.run(p, st, steps)
    u_o, s_o, _ = oracle.fields(p, st)
    floor = p["G_inf"] * p["theta"] * p["tau0"] * float(np.spacing(np.float32(np.abs(u_o).max()))) / np.abs(s_o).max()
    print(f"{scheme} FP32: u {rel(u_g, u_o):.2e}, sigma {rel(s_g, s_o):.2e} = {rel(s_g, s_o) / floor:.2f} x floor")
    assert np.abs(u_o).max() > 1e-3
    assert rel(u_g, u_o) < 1e-5
    assert rel(s_g, s_o) < max(1e-5, 1.5 * floor)


def test_generalized_newtonian_relaxation_time_reaches_the_wall_layers(stream):
    """The GN channel's steady velocity is faster than the Newtonian one at the low-shear
    viscosity (shear thinning lowers tau_LB near the walls); the FP64 GPU state equals the
    oracle's after 20000 steps, and neither has normal stresses."""
    cfg = inputs.oracle_channel_yield()
    p = dict(cfg["params"], scheme="generalized_newtonian")
    with lbnlm.Channels(4, 64, p, "f64", stream=stream, scheme="generalized_newtonian") as gn, \
            lbnlm.Channels(4, 64, dict(p, theta=0.0, tau0=p["tau0"] * (1 + p["theta"])), "f64", stream=stream) as nw:
        gn.step(20000)
        nw.step(20000)
        (u_gn, s_gn, _), = gn.fields()
        (u_nw, _, _), = nw.fields()
    assert u_gn[:, :, 0].max() > 1.2 * u_nw[:, :, 0].max()
    assert np.abs(s_gn[..., 0] - s_gn[..., 1]).max() <= 1e-12 * np.abs(s_gn[..., 3]).max()


def test_comparison_schemes_are_refused_where_not_implemented(stream):
    p = nlm()
    for kw in (dict(stress_mode=1), dict(x_mode="gpbc"), dict(walls="couette")):
        with pytest.raises(lbnlm.LBError) as e:
            lbnlm.Channels(4, 16, p, "f32", stream=stream, scheme="generalized_newtonian", **kw)
        assert e.value.status == lbnlm.LB_EINVAL
    with lbnlm.Channels(4, [16, 20], [p, p], "f32", stream=stream, scheme="stress_divergence") as sim:
        with pytest.raises(lbnlm.LBError) as e:
            sim.run_until_steady(1e-8, check_every=100, max_steps=200)
        assert e.value.status == lbnlm.LB_EINVAL
    # wide FP32 channels: the generalized-Newtonian scheme has a row-march variant, the divergence
    # scheme (two passes per step) stays on the tile kernel
    with lbnlm.Channels(256, 32, p, "f32", stream=stream, scheme="generalized_newtonian") as sim:
        assert lbnlm.lb_uses_row_march(sim.h)
    with lbnlm.Channels(256, 32, p, "f32", stream=stream, scheme="stress_divergence") as sim:
        assert not lbnlm.lb_uses_row_march(sim.h)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_generalized_newtonian_row_march_equals_tile_kernel_and_oracle(stream, prec):
    """Wide single FP32/BF16 channels of the generalized-Newtonian scheme step on the row-march
    kernel's scheme variant: bitwise equal to the tile kernel's, and in FP32 within 1e-5 of the
    oracle on u (BF16: a few units of its roundoff 2^-9)."""
    nx, ny = 256, 48
    scheme = "generalized_newtonian"
    p = dict(nlm(), scheme=scheme)
    st = random_state(nx, ny, 901, amp=1e-3)
    res = {}
    for flags in (0, lbnlm.LB_GRID_TILE_ONLY):
        with lbnlm.Channels(nx, ny, p, prec, flags=flags | lbnlm.LB_GRID_STORE_SIGMA, stream=stream,
                            scheme=scheme) as sim:
            assert lbnlm.lb_uses_row_march(sim.h) == (flags == 0)
            sim.set_populations([st.nstar], [st.drho])
            sim.step(40)
            (u, s, r), = sim.fields()
            (n, d), = sim.populations()
            res[flags] = (u, s, n, d)
    u_m, s_m, n_m, d_m = res[0]
    u_t, s_t, n_t, d_t = res[lbnlm.LB_GRID_TILE_ONLY]
    assert np.array_equal(n_m, n_t) and np.array_equal(u_m, u_t) and np.array_equal(s_m, s_t)
    assert np.all(d_m == 0.0)
    oracle.run(p, st, 40)
    u_o, s_o, _ = oracle.fields(p, st)
    print(f"{prec} row march GN vs oracle: u {rel(u_m, u_o):.2e}, sigma {rel(s_m, s_o):.2e}")
    assert rel(u_m, u_o) < (1e-5 if prec == "f32" else 4 * 2.0 ** -9)
