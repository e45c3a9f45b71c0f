"""The warm-start perceptron's GPU kernels against the FP64 reference (oracle/mlp.py)."""
import numpy as np
import pytest

from oracle import mlp as ref
from paper_1310_7450_gb300 import lbnlm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    return torch


def make(torch, n_in, H, n_out, B, seed):
    m = lbnlm.lb_mlp_create(n_in, H, n_out, B, seed, torch.cuda.current_stream().cuda_stream)
    p = np.zeros(lbnlm.lb_mlp_num_params(m), dtype=np.float32)
    lbnlm.lb_mlp_get_params(m, p)
    return m, p


@pytest.mark.parametrize("n_in,H,n_out,B", [(5, 256, 768, 64), (3, 17, 5, 9)])
def test_forward_and_gradients_match_fp64_reference(torch_cuda, n_in, H, n_out, B):
    torch = torch_cuda
    rng = np.random.default_rng(7)
    m, p = make(torch, n_in, H, n_out, B, 11)
    try:
        x = rng.normal(0, 1, (B, n_in)).astype(np.float32)
        t = rng.normal(0, 0.3, (B, n_out)).astype(np.float32)
        xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        y = torch.zeros((B, n_out), device="cuda")
        lbnlm.lb_mlp_forward(m, xd, B, y)
        g = torch.zeros(p.size, device="cuda")
        loss = lbnlm.lb_mlp_gradients(m, xd, td, B, g)
        torch.cuda.synchronize()
        # reference with the same bfloat16 working weights, in FP64
        y_ref, _ = ref.forward(p, x, n_in, H, n_out, bf16=True)
        loss_ref, g_ref = ref.loss_and_grad(p, x, t, n_in, H, n_out, bf16=True)
        yg = y.cpu().numpy()
        assert np.abs(yg - y_ref).max() <= 1e-5 * max(1.0, np.abs(y_ref).max())
        assert loss == pytest.approx(loss_ref, rel=1e-5)
        gg = g.cpu().numpy()
        assert np.abs(gg - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
        # and the bfloat16 weights change the FP64 gradient only at the BF16 level
        _, g64 = ref.loss_and_grad(p, x, t, n_in, H, n_out, bf16=False)
        assert np.abs(gg - g64).max() <= 3e-2 * np.abs(g64).max()
    finally:
        lbnlm.lb_mlp_destroy(m)


def test_training_reduces_loss_and_params_roundtrip(torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(8)
    n_in, H, n_out, B = 4, 64, 16, 128
    m, p0 = make(torch, n_in, H, n_out, B, 3)
    try:
        x = rng.uniform(-1, 1, (B, n_in)).astype(np.float32)
        w = rng.normal(0, 1, (n_in, n_out))
        t = np.sin(x @ w).astype(np.float32)
        xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        first = lbnlm.lb_mlp_train_step(m, xd, td, B, 3e-3)
        for _ in range(400):
            last = lbnlm.lb_mlp_train_step(m, xd, td, B, 3e-3)
        assert last < 0.1 * first
        p = np.zeros_like(p0)
        lbnlm.lb_mlp_get_params(m, p)
        m2, _ = make(torch, n_in, H, n_out, B, 99)
        lbnlm.lb_mlp_set_params(m2, p)
        y1 = torch.zeros((B, n_out), device="cuda"); y2 = torch.zeros((B, n_out), device="cuda")
        lbnlm.lb_mlp_forward(m, xd, B, y1)
        lbnlm.lb_mlp_forward(m2, xd, B, y2)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2)
        lbnlm.lb_mlp_destroy(m2)
    finally:
        lbnlm.lb_mlp_destroy(m)
