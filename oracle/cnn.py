"""CPU FP64 oracle of the warm-start surrogate's network (test infrastructure only).

Same architecture as the CUDA library's lbm_cnn: six 3x3 convolutions, channels 12 -> 32 ->
32 -> 32 -> 32 -> 32 -> 4, SiLU between layers, periodic padding in x, zero padding in y,
mean squared error.  Written with plain torch CPU float64 operations (conv2d and autograd
serve as library primitives); pinned by tests/test_cnn_oracle.py against an explicit-loop
convolution and against finite differences.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

CH = (12, 32, 32, 32, 32, 32, 4)


def split_params(flat):
    """Flat parameter vector (per layer: weights [Cout][Cin][3][3], then biases) -> list."""
    flat = torch.as_tensor(np.asarray(flat, dtype=np.float64))
    out, o = [], 0
    for l in range(len(CH) - 1):
        ci, co = CH[l], CH[l + 1]
        w = flat[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = flat[o:o + co]
        o += co
        out.append((w, b))
    assert o == flat.numel()
    return out


def conv3x3(a, w, b):
    """y[b,co,h,x] = bias[co] + sum w[co,ci,dy,dx] a[b,ci,h+dy-1,x+dx-1]; periodic x, zero y."""
    a = F.pad(a, (1, 1, 0, 0), mode="circular")
    a = F.pad(a, (0, 0, 1, 1), mode="constant", value=0.0)
    return F.conv2d(a, w, b)


def forward(layers, x):
    a = x
    for l, (w, b) in enumerate(layers):
        z = conv3x3(a, w, b)
        a = z * torch.sigmoid(z) if l < len(layers) - 1 else z
    return a


def loss_and_grad(flat, x, target):
    """Mean squared error and its gradient with respect to the flat parameter vector."""
    p = torch.tensor(np.asarray(flat, dtype=np.float64), requires_grad=True)
    xt = torch.as_tensor(np.asarray(x, dtype=np.float64))
    tt = torch.as_tensor(np.asarray(target, dtype=np.float64))
    y = forward(split_params_tensor(p), xt)
    loss = ((y - tt) ** 2).mean()
    loss.backward()
    return float(loss.item()), p.grad.numpy().copy(), y.detach().numpy()


def split_params_tensor(p):
    out, o = [], 0
    for l in range(len(CH) - 1):
        ci, co = CH[l], CH[l + 1]
        w = p[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = p[o:o + co]
        o += co
        out.append((w, b))
    return out


def n_params():
    return sum(CH[l + 1] * CH[l] * 9 + CH[l + 1] for l in range(len(CH) - 1))
