"""Pins for the CPU reference of the neural operator (CPU only): its hand-written
backward pass against central finite differences of its own loss, and the
convolution against a direct per-pixel sum."""
import numpy as np

from oracle import nn_ref as R


def small_problem(seed=0, H=7, W=6, cin=4, hidden=5, dil=(1, 2, 3, 1)):
    rng = np.random.default_rng(seed)
    shapes, n = R.layer_shapes(cin, hidden, dil)
    params = rng.normal(0, 0.4, n)
    x = rng.normal(0, 1, (2, H, W, cin))
    tgt = rng.normal(0, 1, (2, H, W))
    mask = np.ones((H, W))
    mask[0, :] = mask[-1, :] = mask[:, 0] = mask[:, -1] = 0.0
    return shapes, params, x, tgt, mask


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 5, 6, 3))
    Wt = rng.normal(size=(2, 3, 3, 3))
    d = 2
    out = R.conv(x, Wt, d)
    for yy in range(5):
        for xx in range(6):
            for o in range(2):
                s = 0.0
                for ky in range(3):
                    for kx in range(3):
                        sy, sx = yy + d * (ky - 1), xx + d * (kx - 1)
                        if 0 <= sy < 5 and 0 <= sx < 6:
                            s += Wt[o, ky, kx] @ x[0, sy, sx]
                assert abs(out[0, yy, xx, o] - s) < 1e-12


import pytest


@pytest.mark.parametrize("beta", [0.0, 3.0])
def test_backward_matches_finite_differences(beta):
    shapes, params, x, tgt, mask = small_problem()
    loss, grad = R.loss_and_grad(params, shapes, x, tgt, mask, beta)
    rng = np.random.default_rng(2)
    idx = rng.choice(len(params), 40, replace=False)
    idx = np.concatenate([idx, [shapes[l][4] for l in range(len(shapes))]])  # a bias of every layer
    h = 1e-6
    for i in idx:
        e = np.zeros_like(params)
        e[i] = h
        lp, _ = R.loss_and_grad(params + e, shapes, x, tgt, mask, beta)
        lm, _ = R.loss_and_grad(params - e, shapes, x, tgt, mask, beta)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, grad[i])
