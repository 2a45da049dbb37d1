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


# ---------------------------------------------- Adam (Kingma and Ba 2015, Alg. 1)

def test_adam_first_step_moves_by_lr_times_the_sign():
    # t = 1: m_hat = g and v_hat = g^2 exactly, so the step is lr g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3, -2e-6])
    st = R.AdamState(4)
    out = R.adam_step(np.zeros(4), g, st, lr=0.01, eps=1e-8)
    assert np.allclose(out, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=0)
    assert st.t == 1


def test_adam_constant_gradient_keeps_the_corrected_moments_exact():
    # with g fixed, the bias corrections make m_hat = g and v_hat = g^2 at every t;
    # without them the first steps would be about 3x too long
    g = np.array([0.7, -1.3])
    st = R.AdamState(2)
    th = np.zeros(2)
    for t in range(1, 6):
        th = R.adam_step(th, g, st, lr=1e-2, beta1=0.9, beta2=0.999, eps=0.0)
        assert np.allclose(th, -1e-2 * t * np.sign(g), rtol=1e-13, atol=0)


def test_adam_alternating_gradient_closed_form():
    # g, then -g: m_2 = -(1-b1)^2 g and v_2 = (1-b2)(1+b2) g^2, so m_hat_2 =
    # -(1-b1)/(1+b1) g, v_hat_2 = g^2 and the second step is +lr (1-b1)/(1+b1) sign(g);
    # swapping beta1 and beta2 changes the factor
    b1, b2, lr = 0.9, 0.999, 1e-3
    g = np.array([2.0, -0.25])
    st = R.AdamState(2)
    th1 = R.adam_step(np.zeros(2), g, st, lr, b1, b2, eps=0.0)
    th2 = R.adam_step(th1, -g, st, lr, b1, b2, eps=0.0)
    step2 = th2 - th1
    assert np.allclose(step2, lr * (1 - b1) / (1 + b1) * np.sign(g), rtol=1e-12, atol=0)
    assert np.allclose(st.m, -(1 - b1) ** 2 * g, rtol=1e-14)
    assert np.allclose(st.v, (1 - b2) * (1 + b2) * g * g, rtol=1e-13)
