"""Warm-start U-Net: the library's kernels (forward, both backward passes,
pooling, upsampling, loss, Adam) against the numpy FP64 oracle, and the gain
of the trained network as a starting point for the batched solver."""
import numpy as np
import pytest

import workloads
from oracle import unet_oracle as U

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2408_05444_gb300 as g  # noqa: E402
from paper_2408_05444_gb300 import warmstart as ws  # noqa: E402


def _setup(width, n, h, w, seed, scale=0.3):
    r = np.random.default_rng(seed)
    params = (r.standard_normal(U.num_params(width)) * scale).astype(np.float32)
    C = r.uniform(0, 1, (n, h, w)).astype(np.float32)
    T = r.uniform(0, 1, (n, h, w)).astype(np.float32)
    net = g.grbk_unet_create(width)
    g.grbk_unet_set_params(net, params)
    dev = torch.device("cuda")
    return net, params, C, T, torch.from_numpy(C).to(dev), torch.from_numpy(T).to(dev)


@pytest.mark.parametrize("width,n,h,w", [(4, 3, 16, 24), (20, 2, 32, 32), (3, 1, 36, 20)])
def test_forward_matches_oracle(width, n, h, w):
    net, params, C, T, Ct, Tt = _setup(width, n, h, w, seed=width + h)
    X0 = torch.empty_like(Ct)
    g.grbk_unet_forward(net, Ct, X0)
    ref = U.forward(params, width, C.astype(np.float64))
    err = np.max(np.abs(X0.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < 2e-5, err


@pytest.mark.parametrize("width,n,h,w", [(4, 3, 16, 24), (20, 2, 32, 32)])
def test_loss_and_gradients_match_oracle(width, n, h, w):
    net, params, C, T, Ct, Tt = _setup(width, n, h, w, seed=7 + width)
    loss, grad = g.grbk_unet_loss_grad(net, Ct, Tt)
    lref, gref = U.loss_grad(params, width, C.astype(np.float64), T.astype(np.float64))
    assert abs(loss - lref) <= 1e-5 * lref
    # per layer: relative to the layer's largest gradient entry
    off = 0
    for ci, co in U.layer_io(width):
        for size in (ci * co * 9, co):
            a, b = grad[off:off + size], gref[off:off + size]
            assert np.max(np.abs(a - b)) <= 2e-4 * max(np.max(np.abs(b)), 1e-12), (off, size)
            off += size


def test_adam_step_matches_oracle():
    width = 4
    net, params, C, T, Ct, Tt = _setup(width, 2, 16, 16, seed=3)
    _, grad = g.grbk_unet_loss_grad(net, Ct, Tt)
    g.grbk_unet_train_step(net, Ct, Tt, 1e-3)
    new = g.grbk_unet_get_params(net)
    ref, _, _ = U.adam_step(params.astype(np.float64), grad.astype(np.float64), 0.0, 0.0, 1, 1e-3)
    assert np.max(np.abs(new - ref)) < 1e-6


def test_training_reduces_loss():
    sy = workloads.blur_systems(n_images=22, min_side=32, max_side=32, noise=1e-3, seed=40)
    C = np.stack([s["C"] for s in sy]).astype(np.float32)
    T = np.stack([s["X"] for s in sy]).astype(np.float32)
    net = ws.make_net(12, seed=1)
    dev = torch.device("cuda")
    Ct, Tt = torch.from_numpy(C).to(dev), torch.from_numpy(T).to(dev)
    l0, _ = g.grbk_unet_loss_grad(net, Ct, Tt, want_grad=False)
    losses = ws.train(net, Ct, Tt, epochs=60, batch=16, lr=3e-3)
    l1, _ = g.grbk_unet_loss_grad(net, Ct, Tt, want_grad=False)
    assert np.isfinite(l1) and l1 < 0.5 * l0, (l0, l1, losses[-5:])


def test_warm_start_gain():
    """Train on the solver's own restorations of 64x64 blurred channels, then
    solve held-out channels to the discrepancy stop from X0 = 0, from the
    untrained network and from the trained one: the trained start needs fewer
    iterations than both, and its restorations are as close to the clean
    images."""
    train_sys = workloads.blur_systems(n_images=64, min_side=64, max_side=64, noise=1e-3, seed=50)
    As, Bs, Cs = [s["A"] for s in train_sys], [s["B"] for s in train_sys], [s["C"] for s in train_sys]
    nn_ = [np.linalg.norm(s["E"]) for s in train_sys]
    Xr, _ = ws.restore(As, Bs, Cs, nn_, seed=1)
    dev = torch.device("cuda")
    Ct = torch.tensor(np.stack(Cs), dtype=torch.float32, device=dev)
    Tt = torch.tensor(np.stack(Xr), dtype=torch.float32, device=dev)
    untrained = ws.make_net(20, seed=2)
    net = ws.make_net(20, seed=2)
    ws.train(net, Ct, Tt, epochs=40, batch=32, lr=2e-3)

    test_sys = workloads.blur_systems(n_images=8, min_side=64, max_side=64, noise=1e-3, seed=60)
    As, Bs, Cs = [s["A"] for s in test_sys], [s["B"] for s in test_sys], [s["C"] for s in test_sys]
    nn_ = [np.linalg.norm(s["E"]) for s in test_sys]
    clean = [s["X"] for s in test_sys]

    def run(X0s):
        X, res = ws.restore(As, Bs, Cs, nn_, seed=3, X0s=X0s)
        its = np.array([r["iters"] for r in res])
        err = np.mean([np.linalg.norm(x - c) / np.linalg.norm(c) for x, c in zip(X, clean)])
        return its, err, res

    it0, e0, _ = run(None)
    itu, eu, _ = run([x.astype(np.float64) for x in ws.warm_starts(untrained, Cs)])
    itw, ew, resw = run([x.astype(np.float64) for x in ws.warm_starts(net, Cs)])
    itd, ed, _ = run(ws.warm_starts(net, Cs, on_device=True))   # the same X0 handed over on the device
    assert np.array_equal(itd, itw) and abs(ed - ew) <= 1e-6 * ew
    assert sum(r["x0_rejected"] for r in resw) == 0
    assert itw.mean() < 0.8 * it0.mean(), (itw.mean(), it0.mean())
    assert itw.mean() < itu.mean(), (itw.mean(), itu.mean())
    assert ew <= 1.05 * e0, (ew, e0)


def test_rejected_warm_start_falls_back_to_zero():
    sy = workloads.blur_systems(n_images=1, min_side=48, max_side=48, noise=1e-3, seed=70)
    As, Bs, Cs = [s["A"] for s in sy], [s["B"] for s in sy], [s["C"] for s in sy]
    nn_ = [np.linalg.norm(s["E"]) for s in sy]
    bad = [np.full_like(C, 1e3) for C in Cs]
    X0r, res0 = ws.restore(As, Bs, Cs, nn_, seed=4)
    Xb, resb = ws.restore(As, Bs, Cs, nn_, seed=4, X0s=bad)
    assert all(r["x0_rejected"] == 1 for r in resb)
    assert [r["iters"] for r in resb] == [r["iters"] for r in res0]
    for a, b in zip(X0r, Xb):
        assert np.max(np.abs(a - b)) < 1e-6 * np.max(np.abs(a))


@pytest.mark.parametrize("n,h,w", [(2, 64, 96), (1, 144, 72), (1, 144, 256)])
def test_tensor_core_forward_matches_simt_and_oracle(n, h, w):
    """The tensor-core convolutions (implicit GEMM over a three-term BF16 split of
    the activations, BF16 weights, FP32 accumulation in TMEM) give the forward
    pass of the SIMT kernels to FP32 accuracy: within 3e-5 of the output's scale
    of the SIMT path and of the FP64 oracle (both are FP32 computations of a
    deep network with random weights, summed in different orders).  144 x 72 has
    partial pixel tiles on every level (tiles of 64 x 2, 32 x 4 and 16 x 8
    pixels); 144 x 256 takes the row-halo variant on its two upper levels (rows
    of 256 and 128 pixels, a partial tile in neither), which must agree with
    the one-load-per-tap tiling to 1e-5."""
    width = 20
    net, params, C, T, Ct, Tt = _setup(width, n, h, w, seed=40 + h + w)
    out = {}
    for mode in (1, 2, 0):
        g.grbk_unet_use_tensor_cores(net, mode)
        X = torch.empty_like(Ct)
        g.grbk_unet_forward(net, Ct, X)
        out[mode] = X.cpu().numpy()
    scale = np.max(np.abs(out[0] - C))
    for mode in (1, 2):
        assert np.max(np.abs(out[mode] - out[0])) <= 3e-5 * scale, (mode, np.max(np.abs(out[mode] - out[0])) / scale)
    assert np.max(np.abs(out[1] - out[2])) <= 1e-5 * scale
    ref = U.forward(params, width, C.astype(np.float64))
    assert np.max(np.abs(out[1] - ref)) / np.max(np.abs(ref)) < 3e-5


@pytest.mark.parametrize("n,h,w", [(2, 64, 96), (1, 144, 256)])
def test_tensor_core_input_gradients_match_simt(n, h, w):
    """The gradient with respect to each layer's input runs on the tensor cores
    (the output gradient, masked by the ReLU derivative, convolved with the
    flipped, channel-transposed weights): the parameter gradients of a whole
    backward pass agree with the all-SIMT pass per layer to 2e-4 of the layer's
    largest entry, and the losses (from the two forward passes, which agree to
    3e-5 of the output's scale) to 1e-4; 144 x 256 takes the row-halo variant
    on its two upper levels."""
    width = 20
    net, params, C, T, Ct, Tt = _setup(width, n, h, w, seed=90 + h)
    res = {}
    for mode in (1, 0):
        g.grbk_unet_use_tensor_cores(net, mode)
        res[mode] = g.grbk_unet_loss_grad(net, Ct, Tt)
    (l1, g1), (l0, g0) = res[1], res[0]
    assert abs(l1 - l0) <= 1e-4 * l0
    off = 0
    for ci, co in U.layer_io(width):
        for size in (ci * co * 9, co):
            a, b = g1[off:off + size], g0[off:off + size]
            assert np.max(np.abs(a - b)) <= 2e-4 * max(np.max(np.abs(b)), 1e-12), (off, size)
            off += size
