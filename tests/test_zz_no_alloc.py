"""lb_field_monitor_static: the allocation-free form of the channel monitor.

It serves callers that must not allocate device memory when they read the convergence measures
(for example a monitoring loop that cannot take cudaMalloc's implicit device synchronisation
mid-run, or a process whose device memory is fully reserved by another allocator).  Its scratch
is a fixed array inside the library.  The test feeds it velocity fields read from the device and
checks it against lb_monitor, which evaluates the same measures inside the step with
handle-owned scratch, on two calls in a row (the second call reuses the array the first one
filled); float fields against a host evaluation, with the device memory unchanged across a call;
and channels holding NaN or Inf, which must read as NaN.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1310_7450_gb300 import inputs, lbnlm

pytestmark = pytest.mark.gpu


def test_static_monitor_matches_lb_monitor_on_two_calls():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    nx, nys = 8, [24, 40]
    ps = [dict(inputs.matched_params(0.9, 10.0, 0.1, 1e-3, 1e-5), rho_pert_amp=1e-4, seed=s) for s in (5, 6)]
    nodes = nx * sum(nys)
    offsets = torch.tensor([0, nx * nys[0], nodes], dtype=torch.int64, device="cuda")

    def device_u(sim):
        u = torch.zeros(2 * nodes, dtype=torch.float64, device="cuda")
        lbnlm.lb_get_fields(sim.h, u, None, None, 0, True)
        return u

    with lbnlm.Channels(nx, nys, ps, "f64", stream=stream) as a, lbnlm.Channels(nx, nys, ps, "f64", stream=stream) as b:
        a.step(50)                 # monitor: velocity of state 49 against state 48
        want1 = a.monitor()
        b.step(48)
        u48 = device_u(b)
        b.step(1)
        u49 = device_u(b)
        out = torch.full((len(nys), 3), float("nan"), dtype=torch.float64, device="cuda")
        lbnlm.lb_field_monitor_static(u49, u48, 0, len(nys), offsets, nx, out, stream)
        torch.cuda.synchronize()
        got1 = out.cpu().numpy()

        a.step(2)                  # monitor: state 51 against state 50
        want2 = a.monitor()
        b.step(1)
        u50 = device_u(b)
        b.step(1)
        u51 = device_u(b)
        lbnlm.lb_field_monitor_static(u51, u50, 0, len(nys), offsets, nx, out, stream)
        torch.cuda.synchronize()
        got2 = out.cpu().numpy()

    for got, want in ((got1, want1), (got2, want2)):
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, want[:, :3], rtol=1e-12, atol=0)
    assert not np.array_equal(got1, got2)


def host_monitor(u_now, u_prev, offsets, nx):
    """The three measures in FP64 on the host, per channel, from the same (float) inputs."""
    u_now = np.asarray(u_now, dtype=np.float64).reshape(-1, 2)
    u_prev = np.asarray(u_prev, dtype=np.float64).reshape(-1, 2)
    out = []
    for a, b in zip(offsets[:-1], offsets[1:]):
        un, up = u_now[a:b], u_prev[a:b]
        s1 = np.sum(un * un)
        out.append([np.sqrt(np.sum((un - up) ** 2) / s1) if s1 > 0 else 0.0, un[:, 0].sum() / nx,
                    np.sqrt(np.max(np.sum(un * un, axis=1)))])
    return np.array(out)


def test_static_monitor_float_fields_and_no_allocation():
    """dtype 1 (float fields) against a host FP64 evaluation of the same float inputs, on two calls
    in a row; the device's free memory and torch's reserved pool do not change across the second
    call (the first call may load the library's module, which places the fixed array)."""
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    nx, nys = 16, [3, 61, 200]
    offs = np.concatenate([[0], np.cumsum([nx * n for n in nys])]).astype(np.int64)
    offsets = torch.tensor(offs, dtype=torch.int64, device="cuda")
    g = torch.Generator(device="cpu").manual_seed(11)
    out = torch.full((len(nys), 3), float("nan"), dtype=torch.float64, device="cuda")
    results = []
    for call in range(2):
        un = (1e-2 * torch.randn(2 * int(offs[-1]), generator=g)).float()
        up = un + (1e-6 * torch.randn(un.shape, generator=g)).float()
        un_d, up_d = un.cuda(), up.cuda()
        torch.cuda.synchronize()
        free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        lbnlm.lb_field_monitor_static(un_d, up_d, 1, len(nys), offsets, nx, out, stream)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_reserved() == reserved0
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, host_monitor(un.numpy(), up.numpy(), offs, nx), rtol=1e-12, atol=1e-300)
        results.append(got)
    assert not np.array_equal(results[0], results[1])


@pytest.mark.parametrize("where", ["nan_now", "inf_prev", "inf_now"])
def test_static_monitor_non_finite_channel_reads_nan(where):
    """A NaN or Inf in one channel's fields gives NaN residual, flux and max |u| for that channel
    (a diverged field must never read as converged); the other channel's numbers are unchanged."""
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    nx, nys = 8, [24, 40]
    offs = np.array([0, nx * nys[0], nx * sum(nys)], dtype=np.int64)
    offsets = torch.tensor(offs, dtype=torch.int64, device="cuda")
    g = torch.Generator(device="cpu").manual_seed(3)
    un = 1e-2 * torch.randn(2 * int(offs[-1]), generator=g, dtype=torch.float64)
    up = un + 1e-7 * torch.randn(un.shape, generator=g, dtype=torch.float64)
    out = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    lbnlm.lb_field_monitor_static(un.cuda(), up.cuda(), 0, 2, offsets, nx, out, stream)
    torch.cuda.synchronize()
    clean = out.cpu().numpy()
    k = 2 * (nx * 5 + 3)                     # a node of channel 0
    if where == "nan_now":
        un[k] = float("nan")
    elif where == "inf_prev":
        up[k + 1] = float("inf")
    else:
        un[k] = -float("inf")
    lbnlm.lb_field_monitor_static(un.cuda(), up.cuda(), 0, 2, offsets, nx, out, stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.isnan(got[0]).all()
    assert np.array_equal(got[1], clean[1])


def test_static_monitor_rejects_oversize_requests():
    import torch
    torch.cuda.set_device(0)
    u = torch.zeros(2 * 8, dtype=torch.float64, device="cuda")
    offsets = torch.zeros(2000, dtype=torch.int64, device="cuda")
    out = torch.zeros(1999 * 3, dtype=torch.float64, device="cuda")
    with pytest.raises(lbnlm.LBError) as e:
        lbnlm.lb_field_monitor_static(u, u, 0, 1999, offsets, 4, out, None)
    assert e.value.status == lbnlm.LB_EINVAL
    assert "1024" in lbnlm.lb_last_error()
