"""Residual 3D CNN initialiser for sparse-view reconstruction (BF16 weights
and activations, FP32 accumulation and master weights).

The paper reconstructs with known operators (Eq. 4, 5, 7) and outlines
learned parts inside such pipelines (Section "Network Architectures"); this
network is that learned part.  It maps an FDK reconstruction of sparse
projections to an estimate of the object, used as the starting point of the
TV iteration of Eq. 7.  Its training data comes from the library itself
(phantoms -> ray-driven FP -> FDK).

Architecture (out = x + net(x), all convs 3x3x3, stride 1, zero padding 1):
  level 1 (N^3):     conv 1->16, relu; conv 16->16, relu             -> s1
  level 2 (N/2)^3:   avgpool; conv 16->32, relu; conv 32->32, relu   -> s2
  level 3 (N/4)^3:   avgpool; conv 32->64, relu; conv 64->64, relu   -> s3
  level 4 (N/8)^3:   avgpool; conv 64->64, relu; conv 64->64, relu
  up: nearest x2 + s3; conv 64->32, relu; x2 + s2; conv 32->16, relu;
      x2 + s1; conv 16->16, relu; conv 16->1
About 0.51 M parameters.  Every step (convolutions on the tensor cores,
pooling, upsampling, skips, ReLU, loss, Adam) is a library kernel; PyTorch
only allocates the buffers.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np
import torch

from . import binding as B

LAYERS = [("c0", 1, 16), ("c1", 16, 16), ("c2", 16, 32), ("c3", 32, 32), ("c4", 32, 64), ("c5", 64, 64),
          ("c6", 64, 64), ("c7", 64, 64), ("c8", 64, 32), ("c9", 32, 16), ("c10", 16, 16), ("c11", 16, 1)]


def _bf16(shape, dev):
    return torch.empty(shape, device=dev, dtype=torch.bfloat16)


@dataclass
class Param:
    w: torch.Tensor  # [27, cout, cin] f32 master
    b: torch.Tensor  # [cout] f32
    w16: torch.Tensor  # bf16 copy
    mw: torch.Tensor = None
    vw: torch.Tensor = None
    mb: torch.Tensor = None
    vb: torch.Tensor = None


class ResidualCNN:
    def __init__(self, device="cuda", seed: int = 0):
        self.dev = torch.device(device)
        rng = np.random.default_rng(seed)
        self.params: Dict[str, Param] = {}
        for name, cin, cout in LAYERS:
            std = math.sqrt(2.0 / (27 * cin)) * (0.1 if name == "c11" else 1.0)  # He init; small last layer
            w = torch.from_numpy(rng.normal(0.0, std, (27, cout, cin)).astype(np.float32)).to(self.dev)
            b = torch.zeros(cout, device=self.dev, dtype=torch.float32)
            p = Param(w, b, torch.empty_like(w, dtype=torch.bfloat16))
            B.pyro_cnn_op(B.CNN_F32_TO_BF16, w, p.w16)
            p.mw, p.vw = torch.zeros_like(w), torch.zeros_like(w)
            p.mb, p.vb = torch.zeros_like(b), torch.zeros_like(b)
            self.params[name] = p
        self.step_count = 0

    def n_params(self) -> int:
        return sum(p.w.numel() + p.b.numel() for p in self.params.values())

    # ---------------------------------------------------------------- forward --
    def _conv(self, name, x, relu=True):
        p = self.params[name]
        return B.pyro_conv3d(x, p.w16, p.b, relu)

    def _pool(self, x):
        Bn, D, H, W, C = x.shape
        y = _bf16((Bn, D // 2, H // 2, W // 2, C), self.dev)
        return B.pyro_cnn_op(B.CNN_AVGPOOL2, x, y, dims=(D, H, W, C))

    def _up(self, x, skip):
        Bn, D, H, W, C = x.shape
        y = _bf16((Bn, 2 * D, 2 * H, 2 * W, C), self.dev)
        return B.pyro_cnn_op(B.CNN_UPSAMPLE2, x, y, b=skip, dims=(D, H, W, C))

    def forward(self, x: torch.Tensor, keep: bool = False):
        """x: [B, N, N, N] float32 (an FDK volume) -> out float32 of the same shape."""
        x = x.contiguous()
        Bn, D, H, W = x.shape
        if min(D, H, W) < 64 or D % 8 or H % 64 or W % 64:
            raise ValueError(f"volume {D}x{H}x{W}: each side must be >= 64 and H, W multiples of 64, D of 8 "
                             "(the deepest level runs at N/8 and its convolutions tile by 8)")
        a = {}
        a["x16"] = B.pyro_cnn_op(B.CNN_F32_TO_BF16, x, _bf16((Bn, D, H, W, 1), self.dev))
        a["a0"] = self._conv("c0", a["x16"])
        a["a1"] = self._conv("c1", a["a0"])
        a["p1"] = self._pool(a["a1"])
        a["a2"] = self._conv("c2", a["p1"])
        a["a3"] = self._conv("c3", a["a2"])
        a["p2"] = self._pool(a["a3"])
        a["a4"] = self._conv("c4", a["p2"])
        a["a5"] = self._conv("c5", a["a4"])
        a["p3"] = self._pool(a["a5"])
        a["a6"] = self._conv("c6", a["p3"])
        a["a7"] = self._conv("c7", a["a6"])
        a["u3"] = self._up(a["a7"], a["a5"])
        a["a8"] = self._conv("c8", a["u3"])
        a["u2"] = self._up(a["a8"], a["a3"])
        a["a9"] = self._conv("c9", a["u2"])
        a["u1"] = self._up(a["a9"], a["a1"])
        a["a10"] = self._conv("c10", a["u1"])
        a["a11"] = self._conv("c11", a["a10"], relu=False)
        out = torch.empty_like(x)
        B.pyro_cnn_op(B.CNN_RESIDUAL, a["a11"], out, f=x)
        return (out, a) if keep else out

    # --------------------------------------------------------------- backward --
    def _bwd_conv(self, name, x_in, dy, need_dx=True):
        """Gradients of one conv given dy (already through its ReLU)."""
        p = self.params[name]
        gw = B.pyro_conv3d_wgrad(x_in, dy)
        gb = B.pyro_cnn_bias_grad(dy)
        dx = B.pyro_conv3d(dy, B.pyro_conv3d_flip_weights(p.w16), None, False) if need_dx else None
        return gw, gb, dx

    def _relu_bwd(self, dy, y):
        return B.pyro_cnn_op(B.CNN_RELU_BWD, y, dy)

    def _pool_bwd(self, dy, shape):
        y = _bf16(shape, self.dev)
        D, H, W, C = shape[1:]
        return B.pyro_cnn_op(B.CNN_AVGPOOL2_BWD, dy, y, dims=(D, H, W, C))

    def _up_bwd(self, dy, shape):
        y = _bf16(shape, self.dev)
        D, H, W, C = shape[1:]
        return B.pyro_cnn_op(B.CNN_UPSAMPLE2_BWD, dy, y, dims=(D, H, W, C))

    def _add(self, a, b):
        y = torch.empty_like(a)
        return B.pyro_cnn_op(B.CNN_ADD, a, y, b=b)

    def backward(self, a, dout16: torch.Tensor) -> Dict[str, tuple]:
        """dout16: [B, N, N, N, 1] bf16 gradient of the loss w.r.t. the output."""
        g = {}
        g["c11"] = self._bwd_conv("c11", a["a10"], dout16)
        d = self._relu_bwd(g["c11"][2], a["a10"])
        g["c10"] = self._bwd_conv("c10", a["u1"], d)
        d_u1 = g["c10"][2]
        d = self._relu_bwd(self._up_bwd(d_u1, a["a9"].shape), a["a9"])
        g["c9"] = self._bwd_conv("c9", a["u2"], d)
        d_u2 = g["c9"][2]
        d = self._relu_bwd(self._up_bwd(d_u2, a["a8"].shape), a["a8"])
        g["c8"] = self._bwd_conv("c8", a["u3"], d)
        d_u3 = g["c8"][2]
        d = self._relu_bwd(self._up_bwd(d_u3, a["a7"].shape), a["a7"])
        g["c7"] = self._bwd_conv("c7", a["a6"], d)
        d = self._relu_bwd(g["c7"][2], a["a6"])
        g["c6"] = self._bwd_conv("c6", a["p3"], d)
        d = self._relu_bwd(self._add(self._pool_bwd(g["c6"][2], a["a5"].shape), d_u3), a["a5"])
        g["c5"] = self._bwd_conv("c5", a["a4"], d)
        d = self._relu_bwd(g["c5"][2], a["a4"])
        g["c4"] = self._bwd_conv("c4", a["p2"], d)
        d = self._relu_bwd(self._add(self._pool_bwd(g["c4"][2], a["a3"].shape), d_u2), a["a3"])
        g["c3"] = self._bwd_conv("c3", a["a2"], d)
        d = self._relu_bwd(g["c3"][2], a["a2"])
        g["c2"] = self._bwd_conv("c2", a["p1"], d)
        d = self._relu_bwd(self._add(self._pool_bwd(g["c2"][2], a["a1"].shape), d_u1), a["a1"])
        g["c1"] = self._bwd_conv("c1", a["a0"], d)
        d = self._relu_bwd(g["c1"][2], a["a0"])
        g["c0"] = self._bwd_conv("c0", a["x16"], d, need_dx=False)
        return g

    # ---------------------------------------------------------------- training --
    def train_step(self, x: torch.Tensor, target: torch.Tensor, lr: float = 1e-3) -> float:
        """One Adam step on the MSE between x + net(x) and target; returns the loss."""
        out, a = self.forward(x, keep=True)
        dout = _bf16((*out.shape, 1), self.dev)
        loss = B.pyro_cnn_mse(out, target.contiguous(), dout)
        grads = self.backward(a, dout)
        self.step_count += 1
        for name, (gw, gb, _) in grads.items():
            p = self.params[name]
            B.pyro_cnn_adam(p.w, gw, p.mw, p.vw, p.w16, lr, self.step_count)
            B.pyro_cnn_adam(p.b, gb, p.mb, p.vb, None, lr, self.step_count)
        return float(loss.item())

    def state_dict(self) -> dict:
        return {n: {"w": p.w.cpu(), "b": p.b.cpu(), "mw": p.mw.cpu(), "vw": p.vw.cpu(), "mb": p.mb.cpu(),
                    "vb": p.vb.cpu()} for n, p in self.params.items()} | {"step": self.step_count}

    def load_state_dict(self, sd: dict):
        for n, p in self.params.items():
            for k in ("w", "b", "mw", "vw", "mb", "vb"):
                getattr(p, k).copy_(sd[n][k].to(self.dev))
            B.pyro_cnn_op(B.CNN_F32_TO_BF16, p.w, p.w16)
        self.step_count = int(sd["step"])
