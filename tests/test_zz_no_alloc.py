"""lb_field_monitor_static: the allocation-free form of the channel monitor.

It serves callers that must not allocate device memory when they read the convergence measures
(for example a monitoring loop that cannot take cudaMalloc's implicit device synchronisation
mid-run, or a process whose device memory is fully reserved by another allocator).  Its scratch
is a fixed array inside the library.  The test feeds it velocity fields read from the device and
checks it against lb_monitor, which evaluates the same measures inside the step with
handle-owned scratch, on two calls in a row (the second call reuses the array the first one
filled).  This file is collected last on purpose.
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
