"""Learned warm start for batched colour-image restoration (Section 6 solves one
A X B = C system per channel): train the library's U-Net on (blurred channel,
restoration) pairs produced by the solver itself, then start each solve from
X0 = U-Net(C), with X0 = 0 as the fallback and the reference it must beat.

Every numerical step runs in the library's kernels (grbk_unet_* and
grbk_batch_*); this module only orders the calls.
"""
from __future__ import annotations

import numpy as np

from . import (grbk_batch_create, grbk_batch_solve, grbk_unet_create, grbk_unet_forward,
               grbk_unet_num_params, grbk_unet_set_params, grbk_unet_train_step)

DISCREPANCY_TAU = 1.05


def init_params(width: int, seed: int = 0) -> np.ndarray:
    """He-normal weights (std sqrt(2 / (9 c_in))), zero biases; the output layer is
    scaled by 1e-2 so that the untrained network gives X0 close to C."""
    io = [(1, width), (width, width), (width, 2 * width), (2 * width, 2 * width), (2 * width, 4 * width),
          (4 * width, 4 * width), (6 * width, 2 * width), (2 * width, 2 * width), (3 * width, width),
          (width, width), (width, 1)]
    g = np.random.default_rng(seed)
    parts = []
    for k, (ci, co) in enumerate(io):
        W = g.standard_normal(co * ci * 9) * np.sqrt(2.0 / (9 * ci))
        if k == len(io) - 1:
            W *= 1e-2
        parts += [W, np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


def restore(As, Bs, Cs, noise_norms, variant="grbk", theta=0.8, maxit=2_000_000, seed=0, X0s=None):
    """Batched solve of every system to the discrepancy stop ||R_s|| <= 1.05 ||E_s||;
    returns (X list, result list).  theta is the relaxation of variant "rgrbk"
    (0.8 is the paper's image setting, Section 6); ME-GRBK fixes it at 1/2."""
    b = grbk_batch_create(As, Bs, Cs)
    Xs = [np.zeros((A.shape[1], B.shape[0])) for A, B in zip(As, Bs)]
    targets = DISCREPANCY_TAU * np.asarray(noise_norms, dtype=np.float64)
    st, res = grbk_batch_solve(b, variant, theta=theta, X0s=X0s, targets=targets, maxit=maxit, seed=seed, X_outs=Xs)
    return Xs, res


def train(net, C, T, epochs=2, batch=64, lr=2e-3, seed=0, log=None):
    """Adam on mean((U-Net(C) - T)^2); C, T: CUDA FP32 tensors [N, h, w].
    Returns the per-step losses."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    N = C.shape[0]
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(N, generator=g).to(C.device)
        for i in range(0, N - batch + 1, batch):
            idx = perm[i:i + batch]
            l = grbk_unet_train_step(net, C[idx].contiguous(), T[idx].contiguous(), lr)
            losses.append(l)
            if log:
                log(ep, i // batch, l)
    return losses


def warm_starts(net, Cs, on_device=False):
    """X0 = U-Net(C) for each channel (equal shapes run batched).  The check of
    each X0 against X0 = 0 happens inside grbk_batch_solve.  on_device=True
    returns FP32 device tensors (views of the batched output), which
    grbk_batch_solve takes without a round trip through the host."""
    import torch
    shapes = {}
    for k, C in enumerate(Cs):
        shapes.setdefault(C.shape, []).append(k)
    out = [None] * len(Cs)
    for shp, ks in shapes.items():
        Ct = torch.from_numpy(np.stack([np.asarray(Cs[k], dtype=np.float32) for k in ks])).to("cuda")
        Xt = torch.empty_like(Ct)
        grbk_unet_forward(net, Ct, Xt)
        if on_device:
            for j, k in enumerate(ks):
                out[k] = Xt[j]
        else:
            Xh = Xt.cpu().numpy()
            for j, k in enumerate(ks):
                out[k] = Xh[j]
    return out


def make_net(width=20, seed=0, stream=None):
    net = grbk_unet_create(width, stream=stream)
    p = init_params(width, seed)
    assert len(p) == grbk_unet_num_params(net)
    grbk_unet_set_params(net, p)
    return net
