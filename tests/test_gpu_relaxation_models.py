"""GPU parity of the relaxation-time extensions (density-dependent Maxwell time tau(rho); fluidity
memory of tau_M) against the FP64 oracle, through the C ABI (LB_GRID_RELAXATION_MODEL +
lb_set_relaxation_model).

FP64 within 1e-12 on Couette flow at a uniform density away from rho_ref, on start-up with the
fluidity memory in both stress modes, and on random states (several tiles, ragged tails, body
force and pressure-driven ends); FP32 within 1e-5 on u and within the stress floor of the FP32
velocity on sigma; checkpoint / resume carries the fluidity plane bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1310_7450_gb300 import inputs, lbnlm

pytestmark = pytest.mark.gpu
RX = lbnlm.LB_GRID_RELAXATION_MODEL


@pytest.fixture(scope="module")
def stream():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch.cuda.current_stream().cuda_stream


def rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def couette(theta=10.0, G=1e-3, uw=0.01, **kw):
    p = dict(inputs.matched_params(0.9, theta, 0.1, G, 0.0), top_wall="moving", u_wall=uw)
    p.update(kw)
    return p


def test_fp64_density_dependent_tau_in_couette_flow(stream):
    ny, nx = 16, 2
    p = couette(beta_rho=5.0, rho_ref=1.0)
    st = oracle.init_state(np.full((ny, nx), 1.02))
    with lbnlm.Channels(nx, ny, p, "f64", flags=RX, stream=stream, walls="couette") as sim:
        lbnlm.lb_set_wall_velocity(sim.h, -1, p["u_wall"])
        lbnlm.lb_set_relaxation_model(sim.h, -1, 5.0, 1.0, 0.0)
        sim.set_populations([st.nstar], [st.drho])
        sim.step(4000)
        (u_g, s_g, r_g), = sim.fields()
    oracle.run(p, st, 4000)
    u_o, s_o, r_o = oracle.fields(p, st)
    assert rel(u_g, u_o) < 1e-12 and rel(s_g, s_o) < 1e-12
    assert np.abs(r_g - r_o).max() < 1e-14


@pytest.mark.parametrize("mode", [0, 1])
def test_fp64_fluidity_memory_startup(stream, mode):
    ny, nx = 16, 2
    p = couette(tau_f=800.0, stress_mode=mode)
    with lbnlm.Channels(nx, ny, p, "f64", stress_mode=mode, flags=RX, stream=stream, walls="couette") as sim:
        lbnlm.lb_set_wall_velocity(sim.h, -1, p["u_wall"])
        lbnlm.lb_set_relaxation_model(sim.h, -1, 0.0, 1.0, 800.0)
        sim.step(3000)
        (u_g, s_g, _), = sim.fields()
    st = oracle.init_state(np.ones((ny, nx)))
    oracle.run(p, st, 3000)
    u_o, s_o, _ = oracle.fields(p, st)
    assert np.all(st.phi > 0)
    assert rel(u_g, u_o) < 1e-12 and rel(s_g, s_o) < 1e-12


@pytest.mark.parametrize("x_mode", ["periodic", "gpbc"])
@pytest.mark.parametrize("nx,ny", [(40, 13), (70, 29), (1, 10), (129, 7)])
def test_fp64_random_state_matches_oracle(stream, x_mode, nx, ny):
    p = dict(inputs.matched_params(0.9, 10.0, 0.1, 1e-3, 1e-5), beta_rho=-3.0, rho_ref=0.999, tau_f=25.0,
             x_mode=x_mode)
    rng = np.random.default_rng(90 + nx + ny)
    st = oracle.init_state(1.0 + 1e-2 * rng.uniform(-1, 1, (ny, nx)))
    w = oracle.equilibrium(1.0, 0.0, 0.0)
    st.dev += 1e-2 * rng.uniform(-1, 1, st.dev.shape) * w[:, None, None]
    if x_mode == "periodic":
        st.drho[:] = 1e-4 * rng.uniform(-1, 1, (ny, nx))
    with lbnlm.Channels(nx, ny, p, "f64", flags=RX, stream=stream, x_mode=x_mode) as sim:
        lbnlm.lb_set_relaxation_model(sim.h, -1, p["beta_rho"], p["rho_ref"], p["tau_f"])
        sim.set_populations([st.nstar], [st.drho])
        sim.step(30)
        (n_g, d_g), = sim.populations()
        (u_g, s_g, _), = sim.fields()
    oracle.run(p, st, 30)
    u_o, s_o, _ = oracle.fields(p, st)
    assert rel(n_g, st.nstar) < 1e-14
    assert rel(u_g, u_o) < 1e-12 and rel(s_g, s_o) < 1e-11


def test_fp32_yield_stress_channel_with_memory(stream):
    """4 x 64 yield-stress channel (theta = 100), stress mode 1, fluidity memory tau_f = 2000 and a
    density dependence, 20000 steps from rest in FP32."""
    cfg = inputs.oracle_channel_yield()
    p = dict(cfg["params"], stress_mode=1, beta_rho=2.0, rho_ref=1.0, tau_f=2000.0)
    with lbnlm.Channels(4, 64, p, "f32", stress_mode=1, flags=RX, stream=stream) as sim:
        lbnlm.lb_set_relaxation_model(sim.h, -1, 2.0, 1.0, 2000.0)
        sim.step(20000)
        (u_g, s_g, _), = sim.fields()
    st = oracle.init_state(np.ones((64, 4)))
    oracle.run(p, st, 20000)
    u_o, s_o, _ = oracle.fields(p, st)
    floor = p["G_inf"] * p["theta"] * p["tau0"] * float(np.spacing(np.float32(np.abs(u_o).max()))) / np.abs(s_o).max()
    print(f"relaxation extensions FP32: u {rel(u_g, u_o):.2e}, sigma {rel(s_g, s_o):.2e} = {rel(s_g, s_o) / floor:.2f} x floor")
    assert np.abs(u_o).max() > 1e-3
    assert rel(u_g, u_o) < 1e-5
    assert rel(s_g, s_o) < max(1e-5, 1.5 * floor)


def test_checkpoint_carries_the_fluidity(stream):
    nx, ny = 6, 11
    p = dict(inputs.matched_params(0.9, 10.0, 0.1, 1e-3, 1e-5), rho_pert_amp=1e-3, seed=3)
    with lbnlm.Channels(nx, ny, p, "f32", stress_mode=1, flags=RX, stream=stream) as a:
        lbnlm.lb_set_relaxation_model(a.h, -1, 1.0, 1.0, 50.0)
        a.step(40)
        buf = np.zeros(lbnlm.lb_state_bytes(a.h), dtype=np.uint8)
        lbnlm.lb_get_state(a.h, buf)
        a.step(30)
        (na, da), = a.populations()
        with lbnlm.Channels(nx, ny, p, "f32", stress_mode=1, flags=RX, stream=stream) as b:
            lbnlm.lb_set_relaxation_model(b.h, -1, 1.0, 1.0, 50.0)
            lbnlm.lb_set_state(b.h, buf)
            b.step(30)
            (nb, db), = b.populations()
        with lbnlm.Channels(nx, ny, p, "f32", stress_mode=1, stream=stream) as c:   # no fluidity plane
            with pytest.raises(lbnlm.LBError):
                lbnlm.lb_set_state(c.h, buf)
    assert np.array_equal(na, nb) and np.array_equal(da, db)


def test_relaxation_model_refusals(stream):
    p = inputs.matched_params(0.9, 10.0, 0.1, 1e-3, 1e-5)
    with lbnlm.Channels(4, 16, p, "f32", stream=stream) as sim:
        with pytest.raises(lbnlm.LBError):
            lbnlm.lb_set_relaxation_model(sim.h, -1, 1.0, 1.0, 0.0)   # created without the flag
    with lbnlm.Channels(256, 32, p, "f32", flags=RX, stream=stream, x_mode="gpbc") as sim:
        assert not lbnlm.lb_uses_row_march(sim.h)   # (pressure-driven ends: the tile kernel)
    with lbnlm.Channels(256, 32, p, "f32", flags=RX, stream=stream) as sim:
        assert lbnlm.lb_uses_row_march(sim.h)
        for bad in ((0, 1.0, 0.0, 0.0), (0, 1.0, 1.0, -1.0), (5, 1.0, 1.0, 0.0)):
            with pytest.raises(lbnlm.LBError):
                lbnlm.lb_set_relaxation_model(sim.h, *bad)
    with lbnlm.Channels(4, [16, 20], [p, p], "f32", flags=RX, stream=stream) as sim:
        with pytest.raises(lbnlm.LBError):
            sim.run_until_steady(1e-8, check_every=100, max_steps=200)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("smode", [0, 1])
def test_row_march_variant_equals_tile_kernel_and_oracle(stream, prec, smode):
    """Wide single FP32/BF16 channels with the relaxation-time extensions (density-dependent tau and
    a fluidity memory) step on the row-march kernel's scheme variant, whose fluidity is loaded a row
    ahead: bitwise equal to the tile kernel (populations, fields and the fluidity through the
    checkpoint image), and in FP32 within 1e-5 of the oracle on u."""
    nx, ny, steps = 256, 40, 40
    p = dict(inputs.matched_params(0.9, 10.0, 0.1, 1e-3, 1e-5), rho_pert_amp=1e-3, seed=9, stress_mode=smode,
             beta_rho=2.0, rho_ref=1.0, tau_f=50.0)
    res = {}
    for flags in (0, lbnlm.LB_GRID_TILE_ONLY):
        with lbnlm.Channels(nx, ny, p, prec, stress_mode=smode, flags=flags | RX | lbnlm.LB_GRID_STORE_SIGMA,
                            stream=stream) as sim:
            assert lbnlm.lb_uses_row_march(sim.h) == (flags == 0)
            lbnlm.lb_set_relaxation_model(sim.h, -1, 2.0, 1.0, 50.0)
            sim.step(steps)
            (u, s, r), = sim.fields()
            (n, d), = sim.populations()
            buf = np.zeros(lbnlm.lb_state_bytes(sim.h), dtype=np.uint8)
            lbnlm.lb_get_state(sim.h, buf)
            res[flags] = (u, s, n, d, buf)
    u_m, s_m, n_m, d_m, b_m = res[0]
    u_t, s_t, n_t, d_t, b_t = res[lbnlm.LB_GRID_TILE_ONLY]
    assert np.array_equal(n_m, n_t) and np.array_equal(d_m, d_t)
    assert np.array_equal(u_m, u_t) and np.array_equal(s_m, s_t)
    assert np.array_equal(b_m, b_t)              # (the image carries the fluidity plane)
    if prec == "f32":
        st = oracle.init_state(inputs.initial_density(nx, ny, 1.0, 1e-3, 9))
        oracle.run(p, st, steps)
        u_o, _, _ = oracle.fields(p, st)
        print(f"relaxation row march {prec} smode {smode}: u {rel(u_m, u_o):.2e}")
        assert rel(u_m, u_o) < 1e-5
