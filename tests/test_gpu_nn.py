"""Neural-operator kernels (BF16 tensor-core GEMMs, FP32 accumulation) against the
CPU FP64 reference, and the gain of a trained initial guess over the zero start."""
import numpy as np
import pytest

from oracle import nn_ref as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_4452_gb300 import build, nn
    build.build()
    return nn


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("shape", [(10, 10, 16, (1, 2, 4, 1), 3, 0.0), (13, 11, 32, (1, 3, 1), 2, 4.0),
                                   (9, 12, 64, (2, 1), 4, 1.0)])
def test_forward_loss_and_gradients_match_cpu_reference(M, shape):
    H, Wd, hidden, dil, B, beta = shape
    net = M.Net(H, Wd, hidden=hidden, dilations=dil, max_batch=4, seed=3)
    net.set_h1_weight(beta)
    shapes, n = R.layer_shapes(4, hidden, dil)
    assert n == net.nparams
    rng = np.random.default_rng(7)
    params = net.get_params().astype(np.float64)
    params[[s[4] for s in shapes]] = rng.normal(0, 0.1, len(shapes))  # nonzero first biases too
    net.set_params(params.astype(np.float32))
    params = net.get_params().astype(np.float64)
    x = rng.normal(0, 1, (B, H, Wd, 4)).astype(np.float32)
    tgt = rng.normal(0, 0.3, (B, H, Wd)).astype(np.float32)
    mask = np.ones((H, Wd), np.float32)
    mask[0, :] = mask[-1, :] = mask[:, 0] = mask[:, -1] = 0
    xd, td, md = (torch.tensor(a, device="cuda") for a in (x, tgt, mask))
    y = net.forward(xd, md).cpu().numpy()
    grads = torch.zeros(net.nparams, dtype=torch.float32, device="cuda")
    loss = net.loss_grad(xd, td, md, grads)
    yr, _, _ = R.forward(params, shapes, x.astype(np.float64), mask.astype(np.float64))
    lr, gr = R.loss_and_grad(params, shapes, x.astype(np.float64), tgt.astype(np.float64), mask.astype(np.float64), beta)
    # BF16 operands (8-bit significands) with FP32 accumulation
    assert rel(y, yr) < 2e-2
    assert abs(loss - lr) < 2e-2 * lr
    g = grads.cpu().numpy().astype(np.float64)
    for cin, cout, d, woff, boff in shapes:
        gw, gwr = g[woff:boff], gr[woff:boff]
        assert rel(gw, gwr) < 6e-2, (woff, rel(gw, gwr))
        assert np.dot(gw, gwr) / (np.linalg.norm(gw) * np.linalg.norm(gwr)) > 0.998
        assert rel(g[boff:boff + cout], gr[boff:boff + cout]) < 6e-2
    net.close()


def test_loss_grad_is_deterministic(M):
    net = M.Net(12, 12, hidden=16, dilations=(1, 2, 1), max_batch=2, seed=1)
    x = torch.randn(2, 12, 12, 4, device="cuda", generator=torch.Generator(device="cuda").manual_seed(0))
    t = torch.zeros(2, 12, 12, device="cuda")
    g1 = torch.zeros(net.nparams, device="cuda")
    g2 = torch.zeros_like(g1)
    l1 = net.loss_grad(x, t, None, g1)
    l2 = net.loss_grad(x, t, None, g2)
    assert l1 == l2 and torch.equal(g1, g2)
    net.close()


def test_adam_steps_match_the_cpu_reference(M):
    """iga_nn_adam_step against Kingma and Ba's Algorithm 1 in FP64 (nn_ref.adam_step):
    three steps, each on the gradient the network itself returns at its current
    weights; the update of every parameter is compared element by element."""
    net = M.Net(10, 9, hidden=16, dilations=(1, 2, 1), max_batch=2, seed=5)
    rng = np.random.default_rng(3)
    x = torch.tensor(rng.normal(0, 1, (2, 10, 9, 4)), dtype=torch.float32, device="cuda")
    t = torch.tensor(rng.normal(0, 0.3, (2, 10, 9)), dtype=torch.float32, device="cuda")
    st = R.AdamState(net.nparams)
    g = torch.zeros(net.nparams, dtype=torch.float32, device="cuda")
    for step, (lr, b1, b2, eps) in enumerate([(1e-3, 0.9, 0.999, 1e-8), (2e-3, 0.9, 0.999, 1e-8),
                                              (5e-4, 0.8, 0.99, 1e-6)]):
        w0 = net.get_params().astype(np.float64)
        net.loss_grad(x, t, None, g)
        gh = g.cpu().numpy().astype(np.float64)
        net.adam_step(lr, b1, b2, eps)
        w1 = net.get_params().astype(np.float64)
        ref = R.adam_step(w0, gh, st, lr, b1, b2, eps)
        # FP32 moments and weights: the step agrees to ~1e-6 of lr, the weights to
        # their own rounding
        err = np.abs((w1 - w0) - (ref - w0))
        bound = 1e-5 * lr + 2.0 * np.finfo(np.float32).eps * np.abs(w0)
        assert np.all(err <= bound), (step, float((err / bound).max()))
        assert np.count_nonzero(gh) > 0.9 * net.nparams  # the comparison covers real updates
    net.close()


def test_trained_guess_reduces_newton_iterations(M):
    from paper_1305_4452_gb300 import iga
    nel = 16
    train = M.kappa_instances(range(0, 768), nel=nel)
    test = M.kappa_instances(range(100000, 100064), nel=nel)
    Utr, rtr, _ = M.solve_batch(train)
    keep = rtr["status"] == 0
    train = [t for t, k in zip(train, keep) if k]
    Utr = Utr[keep]
    x, mask = M.features(train)
    tgt = torch.tensor(Utr.reshape(len(train), nel + 2, nel + 2), dtype=torch.float32, device="cuda")
    net = M.Net(nel + 2, nel + 2, hidden=32, max_batch=64, seed=0)
    first = None
    for step in range(600):
        idx = torch.tensor(np.random.default_rng(step).choice(len(train), 64, replace=False), device="cuda")
        loss = net.loss_grad(x[idx], tgt[idx], mask)
        first = loss if first is None else first
        net.adam_step(2e-3 if step < 400 else 5e-4)
    assert loss < 0.1 * first
    # held-out instances: zero start versus the network's guess
    U0, r0, _ = M.solve_batch(test)
    ok = r0["status"] == 0
    xt, _ = M.features(test)
    guess = net.forward(xt, mask).double().cpu().numpy().reshape(len(test), -1)
    U1, r1, _ = M.solve_batch(test, U0=guess)
    assert np.all(r1["status"][ok] == 0)
    assert r1["newton_its"][ok].mean() < r0["newton_its"][ok].mean()
    assert np.abs(U1[ok] - U0[ok]).max() < 1e-7  # same solutions
    net.close()
