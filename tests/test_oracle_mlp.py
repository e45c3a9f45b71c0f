"""The FP64 reference of the warm-start perceptron, pinned by central finite differences and by
the bfloat16 rounding rule."""
import numpy as np

from oracle import mlp


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    n_in, H, n_out, B = 5, 7, 4, 6
    n_par = H * n_in + H + H * H + H + n_out * H + n_out
    p = rng.normal(0, 0.5, n_par)
    x = rng.normal(0, 1, (B, n_in))
    t = rng.normal(0, 1, (B, n_out))
    loss, g = mlp.loss_and_grad(p, x, t, n_in, H, n_out)
    h = 1e-6
    for k in rng.choice(n_par, 40, replace=False):
        e = np.zeros(n_par); e[k] = h
        lp, _ = mlp.loss_and_grad(p + e, x, t, n_in, H, n_out)
        lm, _ = mlp.loss_and_grad(p - e, x, t, n_in, H, n_out)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k]))


def test_bf16_rounding_rule():
    v = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 1e-3], dtype=np.float32)
    r = mlp.bf16_round(v)
    # exactly representable values are kept; others land on a bfloat16 (8 significant bits)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125  # 1 + 2^-8 is a tie -> even
    for a, b in zip(v.astype(np.float64), r):
        assert abs(a - b) <= abs(a) * 2.0 ** -8
        m, e = np.frexp(b)
        assert float(m * 2 ** 8) == int(m * 2 ** 8)
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert mlp.bf16_round(np.array([1.0 + 2.0 ** -8], dtype=np.float32))[0] == 1.0
