"""What the learned warm start gains over the plain scheme (the method without it), end to end on
the GPU: steady states of the batched solver train the perceptron with the library's kernels;
held-out channels started from its prediction reach the steady residual in far fewer steps, and
more of them within the cap, than the same channels started from rest.  Small channels (Ny 32-96)
keep the test short; the full-size comparison is bench.py --workload warmstart."""
import numpy as np
import pytest

from paper_1310_7450_gb300 import inputs, lbnlm, warmstart

pytestmark = pytest.mark.gpu

TOL, CHECK, CAP, TRAIN_CAP = 1e-8, 1000, 1_000_000, 3_000_000


@pytest.fixture(scope="module")
def stream():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch.cuda.current_stream().cuda_stream


def draw(n, seed):
    ps = inputs.sweep_channel_params(n, seed, ny_lo=32, ny_hi=96)
    return [q.pop("ny") for q in ps], ps


def steady(nys, ps, start, stream, cap=CAP):
    with lbnlm.Channels(4, nys, ps, "f32", stream=stream) as sim:
        if start is not None:
            warmstart.apply(sim, start)
        steps, _ = sim.run_until_steady(TOL, check_every=CHECK, max_steps=cap)
        return steps, sim.fields()


def test_trained_surrogate_gains_over_the_plain_scheme(stream):
    nys_t, ps_t = draw(320, 5)
    cf_t = [warmstart.analytic_rows(ny, q) for ny, q in zip(nys_t, ps_t)]
    st_t, fl_t = steady(nys_t, ps_t, cf_t, stream, TRAIN_CAP)
    ok = st_t > 0
    assert ok.sum() >= 150
    keep = [k for k in range(len(nys_t)) if ok[k]]
    Y = warmstart.encode_targets([nys_t[k] for k in keep], [ps_t[k] for k in keep],
                                 [fl_t[k][0][:, 0, 0] for k in keep], [fl_t[k][1][:, 0, 3] for k in keep],
                                 [fl_t[k][1][:, 0, 0] - fl_t[k][1][:, 0, 1] for k in keep])
    X = warmstart.features([nys_t[k] for k in keep], [ps_t[k] for k in keep])
    sur = warmstart.Surrogate(width=256, max_batch=128, seed=1, stream=stream)
    try:
        losses = sur.fit(X, Y, epochs=400, batch=64, lr=2e-3)
        nys, ps = draw(64, 55)
        pred = warmstart.decode(nys, ps, sur.predict(warmstart.features(nys, ps)))
    finally:
        sur.close()
    assert losses[-1] < 0.5 * losses[0]
    rows = [tuple(warmstart.to_rows(f, ny) for f in prof) for ny, prof in zip(nys, pred)]
    st_mlp, fl_mlp = steady(nys, ps, rows, stream)
    st_rest, _ = steady(nys, ps, None, stream)
    cost = lambda st: int(np.where(st > 0, st, CAP).sum())
    err = [np.abs(r[0] - f[0][:, 0, 0]).max() / np.abs(f[0][:, 0, 0]).max() for r, f, s in zip(rows, fl_mlp, st_mlp) if s > 0]
    print(f"held out 64: surrogate start {int((st_mlp > 0).sum())} converged, {cost(st_mlp)} steps; "
          f"from rest {int((st_rest > 0).sum())} converged, {cost(st_rest)} steps; "
          f"surrogate u error median {np.median(err):.2e}; final loss {losses[-1]:.3e}")
    assert (st_mlp > 0).sum() >= (st_rest > 0).sum()
    assert cost(st_mlp) <= 0.5 * cost(st_rest)
    assert np.median(err) < 0.05
