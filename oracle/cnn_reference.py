"""CPU reference for the warm-start network's convolutions.

TEST INFRASTRUCTURE ONLY (like the rest of this package).  Plain float64
PyTorch CPU operations, from the definitions: a convolution is the
cross-correlation out[n, p, q, k] = bias[k] + sum_{r, s, c}
in[n, p stride + r - pad, q stride + s - pad, c] w[k, r, s, c] with zero
padding, and its gradients are those torch's autograd derives for that
expression.  Tensors are NHWC / [K][R][S][C] as in the CUDA kernels.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F


def _nchw(x: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).permute(0, 3, 1, 2)


def _kcrs(w: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(w, dtype=np.float64)).permute(0, 3, 1, 2)


def conv_forward(x, w, bias, stride, pad, relu):
    """NHWC output of act(conv(x, w) + bias)."""
    y = F.conv2d(_nchw(x), _kcrs(w), torch.from_numpy(np.asarray(bias, np.float64)),
                 stride=stride, padding=pad)
    if relu:
        y = torch.clamp(y, min=0.0)
    return y.permute(0, 2, 3, 1).numpy()


def conv_grads(x, w, bias, stride, pad, dy):
    """(dx, dw, dbias) of L = sum(dy * conv(x, w) + bias) (no activation)."""
    xt = _nchw(x).clone().requires_grad_(True)
    wt = _kcrs(w).clone().requires_grad_(True)
    bt = torch.from_numpy(np.asarray(bias, np.float64)).clone().requires_grad_(True)
    y = F.conv2d(xt, wt, bt, stride=stride, padding=pad)
    (y * _nchw(dy)).sum().backward()
    return (xt.grad.permute(0, 2, 3, 1).numpy(), wt.grad.permute(0, 2, 3, 1).numpy(),
            bt.grad.numpy())
