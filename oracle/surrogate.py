"""FP64 CPU reference of the warm-start network (test infrastructure only).

The paper has no network; this is the reference the CUDA training kernels are
checked against: the same U-Net written with plain PyTorch CPU operations in
float64 (conv2d, avg_pool2d, nearest upsampling, concatenation, ReLU), and
gradients by autograd.  Parameter order and layout follow clbm_net_create:
each convolution contributes weights [co][ci][k][k] then bias [co], in the
order encoder (two per level), bottleneck (two), decoder (two per level,
deepest first), 1x1 head.  Pinned in tests by finite differences.

The tensor-core arithmetic (CLBM_NET_TENSOR) rounds both operands of every
convolution GEMM to bfloat16 and accumulates exactly enough that only those
roundings matter; ``rnd=bf16`` reproduces it: forward conv(bf16(x), W),
input gradient from bf16(dL/dy) and W, weight gradient from bf16(x) and
bf16(dL/dy), bias gradient from the unrounded dL/dy (W is passed in already
rounded).  With ``rnd=None`` the convolutions are the plain float64 ones.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F


def unpack(params, shapes):
    p = torch.as_tensor(np.asarray(params, np.float64))
    out, off = [], 0
    for ci, co, k in shapes:
        nw = co * ci * k * k
        out.append((p[off:off + nw].reshape(co, ci, k, k), p[off + nw:off + nw + co]))
        off += nw + co
    return out


def bf16(t):
    """Round a float64 tensor as the kernels round their FP32 values: to
    float32, then to the nearest bfloat16 (ties to even); kept in float64."""
    return t.to(torch.float32).to(torch.bfloat16).to(torch.float64)


class _RoundedConv(torch.autograd.Function):
    """conv2d with GEMM operands passed through rnd (see the module docstring)."""

    @staticmethod
    def forward(ctx, x, w, b, pad, rnd):
        xr = rnd(x)
        ctx.save_for_backward(xr, w)
        ctx.pad, ctx.rnd = pad, rnd
        return F.conv2d(xr, w, b, padding=pad)

    @staticmethod
    def backward(ctx, gy):
        xr, w = ctx.saved_tensors
        gyr = ctx.rnd(gy)
        gx = torch.nn.grad.conv2d_input(xr.shape, w, gyr, padding=ctx.pad)
        gw = torch.nn.grad.conv2d_weight(xr, w.shape, gyr, padding=ctx.pad)
        return gx, gw, gy.sum(dim=(0, 2, 3)), None, None


def conv(h, w, b, pad, rnd=None):
    if rnd is None:
        return F.conv2d(h, w, b, padding=pad)
    return _RoundedConv.apply(h, w, b, pad, rnd)


def forward(x, layers, levels: int, rnd=None):
    """x: float64 tensor [N, Cin, G, G]; layers: list of (W, b) tensors."""
    i = 0
    h = x
    skips = []
    for _ in range(levels - 1):
        h = F.relu(conv(h, layers[i][0], layers[i][1], 1, rnd)); i += 1
        h = F.relu(conv(h, layers[i][0], layers[i][1], 1, rnd)); i += 1
        skips.append(h)
        h = F.avg_pool2d(h, 2)
    h = F.relu(conv(h, layers[i][0], layers[i][1], 1, rnd)); i += 1
    h = F.relu(conv(h, layers[i][0], layers[i][1], 1, rnd)); i += 1
    for l in range(levels - 2, -1, -1):
        up = F.interpolate(h, scale_factor=2, mode="nearest")
        h = torch.cat([up, skips[l]], dim=1)
        h = F.relu(conv(h, layers[i][0], layers[i][1], 1, rnd)); i += 1
        h = F.relu(conv(h, layers[i][0], layers[i][1], 1, rnd)); i += 1
    return conv(h, layers[i][0], layers[i][1], 0, rnd)


def loss_fn(y, t, mask):
    """sum mask (y - t)^2 / (sum mask * C); mask [N, G, G] or None."""
    C = y.shape[1]
    if mask is None:
        mask = torch.ones(y.shape[0], y.shape[2], y.shape[3], dtype=y.dtype)
    return (mask[:, None] * (y - t) ** 2).sum() / (mask.sum() * C)


def loss_and_grad(params, shapes, levels, x, t, mask=None, rnd=None):
    """Loss and d loss / d params (flat float64 array) at the given parameters."""
    p = torch.tensor(np.asarray(params, np.float64), requires_grad=True)
    layers, off = [], 0
    for ci, co, k in shapes:
        nw = co * ci * k * k
        layers.append((p[off:off + nw].reshape(co, ci, k, k), p[off + nw:off + nw + co]))
        off += nw + co
    xt = torch.as_tensor(np.asarray(x, np.float64))
    tt = torch.as_tensor(np.asarray(t, np.float64))
    mt = None if mask is None else torch.as_tensor(np.asarray(mask, np.float64))
    y = forward(xt, layers, levels, rnd)
    L = loss_fn(y, tt, mt)
    (g,) = torch.autograd.grad(L, p)
    return float(L.detach()), g.numpy(), y.detach().numpy()
