"""GPU parity of planar Couette flow (Zou-He moving wall on the last row, Sec. IV C) against the
FP64 oracle: FP64 within 1e-12, FP32 within 1e-5 on u and sigma; start-up and cessation through
lb_set_wall_velocity; combined with the pressure-driven ends."""
import numpy as np
import pytest

import oracle
from paper_1310_7450_gb300 import inputs, lbnlm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stream():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch.cuda.current_stream().cuda_stream


def rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def nlm(theta=10.0, g=0.0, G=1e-3):
    return inputs.matched_params(0.9, theta, 0.1, G, g)


def cou(p, uw):
    return dict(p, top_wall="moving", u_wall=uw)


@pytest.mark.parametrize("nx,ny", [(4, 37), (1, 5), (40, 13), (96, 21), (129, 10)])
def test_couette_fp64_random_state_matches_oracle(stream, nx, ny):
    rng = np.random.default_rng(900 + nx + ny)
    p = nlm()
    st = oracle.flow_state(1 + 1e-2 * rng.uniform(-1, 1, (ny, nx)), 1e-2 * rng.uniform(-1, 1, (ny, nx)),
                           1e-2 * rng.uniform(-1, 1, (ny, nx)), 0.0)
    st.drho[:] = 1e-4 * rng.uniform(-1, 1, (ny, nx))
    with lbnlm.Channels(nx, ny, p, "f64", stream=stream, walls="couette") as sim:
        lbnlm.lb_set_wall_velocity(sim.h, -1, 0.02)
        sim.set_populations([st.nstar], [st.drho])
        sim.step(40)
        (n_g, d_g), = sim.populations()
        (u_g, s_g, _), = sim.fields()
    oracle.run(cou(p, 0.02), st, 40)
    u_o, s_o, _ = oracle.fields(cou(p, 0.02), st)
    assert rel(n_g, st.nstar) < 1e-14
    assert rel(d_g, st.drho) < 1e-10
    assert rel(u_g, u_o) < 1e-12
    assert rel(s_g, s_o) < 1e-11


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_couette_startup_and_cessation(stream, prec, tol):
    """theta = 100: the wall starts at u_wall = 0.01, runs 6000 steps, then stops for 4000."""
    nx, ny = 4, 64
    p = nlm(100.0)
    with lbnlm.Channels(nx, ny, p, prec, stream=stream, walls="couette") as sim:
        lbnlm.lb_set_wall_velocity(sim.h, -1, 0.01)
        sim.step(6000)
        (u1, s1, _), = sim.fields()
        lbnlm.lb_set_wall_velocity(sim.h, -1, 0.0)
        sim.step(4000)
        (u2, s2, _), = sim.fields()
    st = oracle.init_state(np.ones((ny, nx)))
    oracle.run(cou(p, 0.01), st, 6000)
    uo1, so1, _ = oracle.fields(cou(p, 0.01), st)
    oracle.run(cou(p, 0.0), st, 4000)
    uo2, so2, _ = oracle.fields(cou(p, 0.0), st)
    print(f"Couette {prec}: start-up u {rel(u1, uo1):.2e} sigma {rel(s1, so1):.2e}; "
          f"cessation u {rel(u2, uo2):.2e} sigma {rel(s2, so2):.2e}")
    assert rel(u1, uo1) < tol and rel(s1, so1) < tol
    assert rel(u2, uo2) < tol and rel(s2, so2) < tol


def test_couette_with_pressure_driven_ends(stream):
    nx, ny = 6, 20
    p = nlm(10.0, 2e-6)
    with lbnlm.Channels(nx, ny, p, "f64", stream=stream, walls="couette", x_mode="gpbc") as sim:
        lbnlm.lb_set_wall_velocity(sim.h, -1, 0.005)
        sim.step(3000)
        (u_g, s_g, r_g), = sim.fields()
    pg = dict(cou(p, 0.005), x_mode="gpbc")
    rin, rout = oracle.gpbc_densities(pg, nx)
    st = oracle.init_state(inputs.linear_density(nx, ny, rin, rout))
    oracle.run(pg, st, 3000)
    u_o, s_o, r_o = oracle.fields(pg, st)
    assert rel(u_g, u_o) < 1e-12 and rel(s_g, s_o) < 1e-11
    assert np.abs(r_g - r_o).max() < 2e-15   # rho ~ 1: a few units of its last place


def test_wall_velocity_needs_a_moving_wall(stream):
    with lbnlm.Channels(4, 16, nlm(), "f64", stream=stream) as sim:
        with pytest.raises(lbnlm.LBError) as e:
            lbnlm.lb_set_wall_velocity(sim.h, -1, 0.01)
        assert e.value.status == lbnlm.LB_EINVAL
    with lbnlm.Channels(4, [16, 24], nlm(), "f32", stream=stream, walls="couette") as sim:
        with pytest.raises(lbnlm.LBError) as e:
            sim.run_until_steady(1e-8, check_every=100, max_steps=1000)
        assert e.value.status == lbnlm.LB_EINVAL
