"""CPU FP64 reference of the convolutional neural operator (TEST INFRASTRUCTURE).

Plain numpy: zero-padded dilated 3x3 convolutions written as nine shifted
channel contractions, SiLU, a masked mean-squared error, the backward pass
written out by hand (chain rule per layer), and the Adam update of Kingma and Ba
(2015, Algorithm 1).  Parameters use the flat layout of the CUDA network: per
layer W[cout][3][3][cin] then b[cout].  Never imported by the product path.
"""
import numpy as np


def layer_shapes(in_channels, hidden, dilations):
    out, off = [], 0
    L = len(dilations)
    for l, d in enumerate(dilations):
        cin = in_channels if l == 0 else hidden
        cout = 1 if l == L - 1 else hidden
        woff = off
        off += cout * 9 * cin
        out.append((cin, cout, d, woff, off))
        off += cout
    return out, off


def _shift(xp, d, ky, kx, H, W):
    return xp[:, d * ky:d * ky + H, d * kx:d * kx + W, :]


def conv(x, Wt, d):
    """out[b,y,x,o] = sum_{ky,kx,c} Wt[o,ky,kx,c] x[b, y+d(ky-1), x+d(kx-1), c], zero outside."""
    B, H, W, C = x.shape
    xp = np.pad(x, ((0, 0), (d, d), (d, d), (0, 0)))
    out = np.zeros((B, H, W, Wt.shape[0]))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("bhwc,oc->bhwo", _shift(xp, d, ky, kx, H, W), Wt[:, ky, kx, :])
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, shapes, x, mask):
    acts, zs = [x], []
    for l, (cin, cout, d, woff, boff) in enumerate(shapes):
        Wt = params[woff:boff].reshape(cout, 3, 3, cin)
        z = conv(acts[-1], Wt, d) + params[boff:boff + cout]
        zs.append(z)
        if l + 1 < len(shapes):
            acts.append(silu(z))
    y = mask[None] * zs[-1][..., 0]
    return y, acts, zs


def loss_and_grad(params, shapes, x, tgt, mask, beta=0.0):
    """Loss [sum mask e^2 + beta * sum over grid edges (e_i - e_j)^2] / sum mask with
    e = y - tgt, and its gradient with respect to params."""
    y, acts, zs = forward(params, shapes, x, mask)
    m = mask[None] * np.ones_like(tgt)
    count = max(m.sum(), 1.0)
    e = y - tgt
    dx, dy = np.diff(e, axis=2), np.diff(e, axis=1)
    loss = float(((m * e ** 2).sum() + beta * ((dx ** 2).sum() + (dy ** 2).sum())) / count)
    grad = np.zeros_like(params)
    gy = 2.0 * m * e
    if beta:
        lap = np.zeros_like(e)
        lap[:, :, :-1] -= dx
        lap[:, :, 1:] += dx
        lap[:, :-1, :] -= dy
        lap[:, 1:, :] += dy
        gy = gy + 2.0 * beta * lap
    dz = (mask[None] * gy / count)[..., None]  # dL/dz of the last layer, y = mask * z
    for l in range(len(shapes) - 1, -1, -1):
        cin, cout, d, woff, boff = shapes[l]
        if l < len(shapes) - 1:
            dz = da * dsilu(zs[l])
        xin = acts[l]
        B, H, W, C = xin.shape
        xp = np.pad(xin, ((0, 0), (d, d), (d, d), (0, 0)))
        Wt = params[woff:boff].reshape(cout, 3, 3, cin)
        gW = np.zeros((cout, 3, 3, cin))
        dxp = np.zeros_like(xp)
        for ky in range(3):
            for kx in range(3):
                gW[:, ky, kx, :] = np.einsum("bhwo,bhwc->oc", dz, _shift(xp, d, ky, kx, H, W))
                dxp[:, d * ky:d * ky + H, d * kx:d * kx + W, :] += np.einsum("bhwo,oc->bhwc", dz, Wt[:, ky, kx, :])
        grad[woff:boff] = gW.reshape(-1)
        grad[boff:boff + cout] = dz.sum(axis=(0, 1, 2))
        da = dxp[:, d:d + H, d:d + W, :]
    return loss, grad


class AdamState:
    """First and second moment estimates m, v (zero at the start) and the step count t."""

    def __init__(self, n):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0


def adam_step(params, grad, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015, Algorithm 1), elementwise:
        t <- t + 1
        m <- beta1 m + (1 - beta1) g          (biased first moment)
        v <- beta2 v + (1 - beta2) g^2        (biased second raw moment)
        m_hat = m / (1 - beta1^t),  v_hat = v / (1 - beta2^t)   (bias corrections)
        theta <- theta - lr m_hat / (sqrt(v_hat) + eps)
    Returns the new parameters; `state` is updated in place."""
    g = np.asarray(grad, dtype=np.float64)
    state.t += 1
    state.m = beta1 * state.m + (1.0 - beta1) * g
    state.v = beta2 * state.v + (1.0 - beta2) * g * g
    m_hat = state.m / (1.0 - beta1 ** state.t)
    v_hat = state.v / (1.0 - beta2 ** state.t)
    return np.asarray(params, dtype=np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps)
