"""FP64 CPU reference of the residual 3D CNN initialiser.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).  The paper has no
such network; its definition here is the architecture the library
implements: 3x3x3 convolutions (stride 1, zero padding 1) with ReLU, 2x2x2
average pooling, nearest 2x upsampling with additive skips and a residual
output.  The convolution is torch's CPU ``conv3d`` in float64 (a library
primitive); everything else is written out directly.

Layouts match the library: activations [B, D, H, W, C] (channels last),
weights [27, Cout, Cin] with tap = (dz*3 + dy)*3 + dx.
"""
from __future__ import annotations

import torch
import torch.nn.functional as F

LAYERS = [("c0", 1, 16), ("c1", 16, 16), ("c2", 16, 32), ("c3", 32, 32), ("c4", 32, 64), ("c5", 64, 64),
          ("c6", 64, 64), ("c7", 64, 64), ("c8", 64, 32), ("c9", 32, 16), ("c10", 16, 16), ("c11", 16, 1)]


def to_kernel(w):
    """[27, Cout, Cin] -> torch's [Cout, Cin, 3, 3, 3]."""
    w = torch.as_tensor(w, dtype=torch.float64)
    cout, cin = w.shape[1], w.shape[2]
    return w.reshape(3, 3, 3, cout, cin).permute(3, 4, 0, 1, 2).contiguous()


def conv3d(x, w, bias=None, relu=False):
    """y[v, co] = sum_{tap, ci} w[tap, co, ci] x[v + tap - 1, ci] (+ bias, ReLU); channels last."""
    x = torch.as_tensor(x, dtype=torch.float64)
    y = F.conv3d(x.permute(0, 4, 1, 2, 3), to_kernel(w),
                 None if bias is None else torch.as_tensor(bias, dtype=torch.float64), padding=1)
    y = y.permute(0, 2, 3, 4, 1).contiguous()
    return torch.clamp_min(y, 0.0) if relu else y


def conv3d_wgrad(x, dy):
    """dW[tap, co, ci] = sum_v dy[v, co] x[v + tap - 1, ci]."""
    x = torch.as_tensor(x, dtype=torch.float64).permute(0, 4, 1, 2, 3)
    dy = torch.as_tensor(dy, dtype=torch.float64).permute(0, 4, 1, 2, 3)
    cout, cin = dy.shape[1], x.shape[1]
    g = torch.nn.grad.conv3d_weight(x, (cout, cin, 3, 3, 3), dy, padding=1)
    return g.permute(2, 3, 4, 0, 1).reshape(27, cout, cin)


def avgpool2(x):
    x = torch.as_tensor(x, dtype=torch.float64)
    B, D, H, W, C = x.shape
    return x.reshape(B, D // 2, 2, H // 2, 2, W // 2, 2, C).mean(dim=(2, 4, 6))


def upsample2(x, skip=None):
    x = torch.as_tensor(x, dtype=torch.float64)
    y = x.repeat_interleave(2, 1).repeat_interleave(2, 2).repeat_interleave(2, 3)
    return y if skip is None else y + torch.as_tensor(skip, dtype=torch.float64)


def network(x, params):
    """out = x + net(x) for x [B, N, N, N]; params: name -> (w [27, Cout, Cin], b [Cout])."""
    x = torch.as_tensor(x, dtype=torch.float64)
    c = lambda name, v, relu=True: conv3d(v, params[name][0], params[name][1], relu)
    a0 = c("c0", x[..., None])
    a1 = c("c1", a0)
    a2 = c("c2", avgpool2(a1))
    a3 = c("c3", a2)
    a4 = c("c4", avgpool2(a3))
    a5 = c("c5", a4)
    a6 = c("c6", avgpool2(a5))
    a7 = c("c7", a6)
    a8 = c("c8", upsample2(a7, a5))
    a9 = c("c9", upsample2(a8, a3))
    a10 = c("c10", upsample2(a9, a1))
    a11 = c("c11", a10, relu=False)
    return x + a11[..., 0]
