"""The warm start's profile arithmetic on the device (lb_warmstart_apply, lb_warmstart_targets)
against its NumPy reference (tests/warmstart_reference.py, pinned to the oracle's quadrature):
the closed-form start and a decoded prediction give the same populations as the reference rows
written through lb_set_fields (FP64 handle: to 1e-13 of the populations' offsets), and the training
targets of a state equal the reference encoding at FP32 rounding.  Channel widths 33 to 4096 rows
(grid finer and coarser than the rows), several channels per handle."""
import numpy as np
import pytest

import oracle
import warmstart_reference as ref
from paper_1310_7450_gb300 import inputs, lbnlm, warmstart

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stream():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch.cuda.current_stream().cuda_stream


NYS = [33, 200, 256, 1024, 4096]


def channels():
    ps = [inputs.matched_params(0.9, th, 0.1, G, g) for th, G, g in
          [(0.0, 1e-4, 1e-7), (10.0, 1e-4, 2e-7), (100.0, 3e-5, 5e-9), (500.0, 1e-5, 2e-10), (31.6, 2e-5, 1e-11)]]
    return NYS, ps


def offsets(pops):
    w = oracle.WEIGHTS[:, None, None]
    return np.concatenate([(n - w).ravel() for n, _ in pops]), np.concatenate([d.ravel() for _, d in pops])


def test_closed_form_start_equals_reference_rows(stream):
    nys, ps = channels()
    with lbnlm.Channels(2, nys, ps, "f64", stream=stream) as a, lbnlm.Channels(2, nys, ps, "f64", stream=stream) as b:
        warmstart.start_closed_form(a)
        rows = [ref.analytic_rows(ny, p) for ny, p in zip(nys, ps)]
        warmstart.apply_fields(b, [r[0] for r in rows], [r[2] for r in rows])
        na, da = offsets(a.populations())
        nb, db = offsets(b.populations())
    assert np.abs(na - nb).max() <= 1e-13 * np.abs(nb).max()
    assert np.abs(da - db).max() <= 1e-13 * np.abs(db).max()


def test_decoded_prediction_equals_reference_decoding(stream):
    import torch
    nys, ps = channels()
    rng = np.random.default_rng(12)
    raw = rng.normal(0.0, 1.0, (len(nys), 3 * ref.NPTS)).astype(np.float32)
    mu = rng.normal(0.0, 0.05, 3 * ref.NPTS).astype(np.float32)
    sd = rng.uniform(0.01, 0.1, 3 * ref.NPTS).astype(np.float32)
    with lbnlm.Channels(3, nys, ps, "f64", stream=stream) as a, lbnlm.Channels(3, nys, ps, "f64", stream=stream) as b:
        lbnlm.lb_warmstart_apply(a.h, torch.tensor(raw, device="cuda"), torch.tensor(mu, device="cuda"),
                                 torch.tensor(sd, device="cuda"))
        pred = raw.astype(np.float64) * sd.astype(np.float64) + mu.astype(np.float64)
        prof = ref.decode(nys, ps, pred)
        warmstart.apply_fields(b, [ref.to_rows(f[0], ny) for f, ny in zip(prof, nys)],
                               [ref.to_rows(f[2], ny) for f, ny in zip(prof, nys)])
        na, da = offsets(a.populations())
        nb, db = offsets(b.populations())
    assert np.abs(na - nb).max() <= 1e-13 * np.abs(nb).max()
    assert np.abs(da - db).max() <= 1e-13 * np.abs(db).max()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_targets_equal_reference_encoding(stream, prec):
    """Targets of a developed (not steady) state: the device encoding of the handle's own fields
    against the reference encoding of the same fields read back (float32 outputs)."""
    nys, ps = channels()
    nys, ps = nys[:4], ps[:4]
    with lbnlm.Channels(4, nys, ps, prec, stream=stream) as sim:
        warmstart.start_closed_form(sim)
        sim.step(500)
        y = warmstart.steady_targets(sim).cpu().numpy()
        fl = sim.fields()
    want = ref.encode_targets(nys, ps, [f[0][:, 0, 0] for f in fl], [f[1][:, 0, 3] for f in fl],
                              [f[1][:, 0, 0] - f[1][:, 0, 1] for f in fl])
    assert y.dtype == np.float32
    np.testing.assert_allclose(y, want, rtol=0, atol=2e-6 * np.abs(want).max() + 1e-6)


def test_warmstart_needs_a_closed_form(stream):
    p = inputs.matched_params(0.9, 10.0, 0.1, 1e-3, 0.0)   # no body force: no closed form
    with lbnlm.Channels(4, 16, p, "f32", stream=stream) as sim:
        with pytest.raises(lbnlm.LBError) as e:
            warmstart.start_closed_form(sim)
        assert e.value.status == lbnlm.LB_EINVAL
