"""Pins for the numpy U-Net oracle: torch CPU convolution and autograd as library
routines, adjoint identities, finite differences of the whole network, torch's
Adam and BF16 rounding."""
import numpy as np
import pytest

from oracle import unet_oracle as U

torch = pytest.importorskip("torch")


def test_conv_matches_torch_conv2d_and_autograd():
    g = np.random.default_rng(0)
    x = g.standard_normal((2, 3, 9, 7))
    W = g.standard_normal((5, 3, 3, 3))
    b = g.standard_normal(5)
    out = U.conv3x3(x, W, b)
    xt = torch.tensor(x, requires_grad=True)
    Wt = torch.tensor(W, requires_grad=True)
    bt = torch.tensor(b, requires_grad=True)
    ot = torch.nn.functional.conv2d(xt, Wt, bt, padding=1)
    assert np.max(np.abs(out - ot.detach().numpy())) < 1e-12
    gy = g.standard_normal(out.shape)
    ot.backward(torch.tensor(gy))
    dx, dW, db = U.conv3x3_grads(x, W, gy)
    assert np.max(np.abs(dx - xt.grad.numpy())) < 1e-12
    assert np.max(np.abs(dW - Wt.grad.numpy())) < 1e-11
    assert np.max(np.abs(db - bt.grad.numpy())) < 1e-11


def test_pool_and_up_adjoints():
    g = np.random.default_rng(1)
    x = g.standard_normal((2, 3, 8, 12))
    y = g.standard_normal((2, 3, 4, 6))
    assert abs(np.sum(U.pool(x) * y) - np.sum(x * U.pool_adj(y))) < 1e-12
    assert abs(np.sum(U.up(y) * x) - np.sum(y * U.up_adj(x))) < 1e-12
    assert np.allclose(U.pool(U.up(y)), y)


def test_network_gradient_matches_finite_differences():
    w = 2
    g = np.random.default_rng(2)
    params = g.standard_normal(U.num_params(w)) * 0.3
    C = g.uniform(0, 1, (2, 8, 8))
    T = g.uniform(0, 1, (2, 8, 8))
    loss, grad = U.loss_grad(params, w, C, T, bf16=False)
    idx = g.choice(len(params), 60, replace=False)
    h = 1e-6
    for j in idx:
        pp, pm = params.copy(), params.copy()
        pp[j] += h
        pm[j] -= h
        fd = (U.loss_grad(pp, w, C, T, bf16=False)[0] - U.loss_grad(pm, w, C, T, bf16=False)[0]) / (2 * h)
        assert abs(fd - grad[j]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (j, fd, grad[j])


def test_adam_matches_torch():
    g = np.random.default_rng(3)
    p0 = g.standard_normal(17)
    grads = [g.standard_normal(17) for _ in range(3)]
    pt = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m1, m2 = p0.copy(), np.zeros(17), np.zeros(17)
    for k, gr in enumerate(grads, start=1):
        opt.zero_grad()
        pt.grad = torch.tensor(gr)
        opt.step()
        p, m1, m2 = U.adam_step(p, gr, m1, m2, k, 1e-2)
    assert np.max(np.abs(p - pt.detach().numpy())) < 1e-12


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(4).standard_normal(1000).astype(np.float32) * 10
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16_round(x), ref)


def test_param_count():
    assert U.num_params(20) == 184361
