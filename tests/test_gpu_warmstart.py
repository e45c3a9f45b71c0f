"""What the learned warm start gains over the plain scheme (the method without it), end to end on
the GPU: steady states of the batched solver train the perceptron with the library's kernels;
held-out channels started from its prediction reach the steady residual in far fewer steps, and
more of them within the cap, than the same channels started from rest.  Small channels (Ny 32-96)
keep the test short; the full-size comparison is bench.py --workload warmstart.  The closed-form
start, the training targets and the decoding of the predictions run on the device."""
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
    """start: a function writing the start state into the handle (None: rest)."""
    with lbnlm.Channels(4, nys, ps, "f32", stream=stream) as sim:
        if start is not None:
            start(sim)
        steps, _ = sim.run_until_steady(TOL, check_every=CHECK, max_steps=cap)
        return steps, sim.fields(), (warmstart.steady_targets(sim) if start is not None else None)


def start_fields(nys, ps, start, stream):
    """The velocity field a start writes (read back before any step)."""
    with lbnlm.Channels(4, nys, ps, "f32", stream=stream) as sim:
        start(sim)
        return sim.fields()


def test_trained_surrogate_gains_over_the_plain_scheme(stream):
    nys_t, ps_t = draw(320, 5)
    st_t, _, Y_all = steady(nys_t, ps_t, warmstart.start_closed_form, stream, TRAIN_CAP)
    ok = st_t > 0
    assert ok.sum() >= 150
    keep = [k for k in range(len(nys_t)) if ok[k]]
    import torch
    Y = Y_all[torch.tensor(keep, device="cuda")]
    X = warmstart.features([nys_t[k] for k in keep], [ps_t[k] for k in keep])
    sur = warmstart.Surrogate(width=256, max_batch=128, seed=1, stream=stream)
    try:
        losses = sur.fit(X, Y, epochs=400, batch=64, lr=2e-3)
        nys, ps = draw(64, 55)
        start = lambda sim: sur.start(sim, nys, ps)
        fl_start = start_fields(nys, ps, start, stream)
        st_mlp, fl_mlp, _ = steady(nys, ps, start, stream)
    finally:
        sur.close()
    assert losses[-1] < 0.5 * losses[0]
    st_rest, _, _ = steady(nys, ps, None, stream)
    cost = lambda st: int(np.where(st > 0, st, CAP).sum())
    err = [np.abs(a[0][:, 0, 0] - f[0][:, 0, 0]).max() / np.abs(f[0][:, 0, 0]).max()
           for a, f, s in zip(fl_start, fl_mlp, st_mlp) if s > 0]
    print(f"held out 64: surrogate start {int((st_mlp > 0).sum())} converged, {cost(st_mlp)} steps; "
          f"from rest {int((st_rest > 0).sum())} converged, {cost(st_rest)} steps; "
          f"surrogate u error median {np.median(err):.2e}; final loss {losses[-1]:.3e}")
    assert (st_mlp > 0).sum() >= (st_rest > 0).sum()
    assert cost(st_mlp) <= 0.5 * cost(st_rest)
    assert np.median(err) < 0.05
