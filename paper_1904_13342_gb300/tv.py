"""TV-regularised iterative reconstruction (Section "Iterative
Reconstruction", Eq. 7): min_x |A x - p|^2 + lambda TV(x), starting from
x = 0.

The paper trains an additive layer with TF's optimiser; the optimiser is not
specified.  Here it is gradient descent with Barzilai-Borwein steps:
  g_k = 2 A^T (A x_k - p) + lambda grad TV(x_k),
  alpha_0 = 1 / L_est (L_est from power iterations on 2 A^T A),
  alpha_k = (s.s) / (s.dy), s = x_k - x_{k-1}, dy = g_k - g_{k-1},
  clamped to [0, 10 / L_est],
  x_{k+1} = x_k - alpha_k g_k.
Every vector operation is a library kernel (FP, exact adjoint, pyro_tv,
pyro_axpby, pyro_dot); only the two scalars of each BB step come back to
the host.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import torch

from . import binding as B
from .geometry import ConeGeometry3D


@dataclass
class TVResult:
    x: torch.Tensor
    objective: List[float] = field(default_factory=list)
    steps: List[float] = field(default_factory=list)


def _ops(g):
    if isinstance(g, ConeGeometry3D):
        ws = {}

        def A(x, out=None):
            if "w" not in ws:
                ws["w"] = torch.empty(B.fp_cone3d_workspace_bytes(g, x.dtype), dtype=torch.uint8, device=x.device)
            return B.pyro_fp_cone3d_ws(x, g, workspace=ws["w"], out=out)

        def AT(y):
            if "wT" not in ws:
                ws["wT"] = torch.empty(B.fpT_cone3d_workspace_bytes(g), dtype=torch.uint8, device=y.device)
            return B.pyro_fpT_cone3d_ws(y, g, workspace=ws["wT"])

        return A, AT
    if g.fan:
        return (lambda x, out=None: B.pyro_fp_fan2d(x, g)), (lambda y: B.pyro_fpT_fan2d(y, g))
    return (lambda x, out=None: B.pyro_fp_par2d(x, g)), (lambda y: B.pyro_fpT_par2d(y, g))


def estimate_lipschitz(g, shape, device, iters: int = 20, seed: int = 0) -> float:
    """Largest eigenvalue of 2 A^T A by power iteration (FP32 kernels)."""
    A, AT = _ops(g)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    v = torch.rand(shape, generator=gen, dtype=torch.float32).to(device)
    lam = 0.0
    for _ in range(iters):
        w = AT(A(v))
        nrm = float(torch.sqrt(B.pyro_dot(w, w)).item())
        lam = nrm / max(float(torch.sqrt(B.pyro_dot(v, v)).item()), 1e-30)
        B.pyro_axpby(w, v, 1.0 / max(nrm, 1e-30), 0.0)
    return 2.0 * lam


def tv_reconstruct(p: torch.Tensor, g, n_iter: int, lam: float, eps: float, L_est: Optional[float] = None,
                   x0: Optional[torch.Tensor] = None, clamp: float = 10.0, track_objective: bool = False,
                   callback=None) -> TVResult:
    """Minimise |A x - p|^2 + lam TV(x) (Eq. 7); p is one FP32 sinogram.
    `callback(k, x)`, when given, sees the iterate after each step k."""
    A, AT = _ops(g)
    shape = tuple(g.volume_shape)
    dev = p.device
    if L_est is None:
        L_est = estimate_lipschitz(g, shape, dev)
    x = torch.zeros(shape, device=dev, dtype=torch.float32) if x0 is None else x0.clone().float()
    x_prev = torch.empty_like(x)
    g_prev = torch.empty_like(x)
    r = torch.empty_like(p)
    res = TVResult(x)
    for k in range(n_iter):
        r = A(x, out=r) if isinstance(g, ConeGeometry3D) else A(x)
        B.pyro_axpby(p, r, -1.0, 1.0)  # r = A x - p
        gd = AT(r)
        grad, tvv = B.pyro_tv(x, eps, lam, base=gd, alpha=2.0, want_value=track_objective)
        if track_objective:
            res.objective.append(float(B.pyro_dot(r, r).item()) + lam * float(tvv.item()))
        if k == 0:
            alpha = 1.0 / L_est
        else:
            B.pyro_axpby(x, x_prev, 1.0, -1.0)  # s = x_k - x_{k-1}
            B.pyro_axpby(grad, g_prev, 1.0, -1.0)  # dy = g_k - g_{k-1}
            ss = float(B.pyro_dot(x_prev, x_prev).item())
            sy = float(B.pyro_dot(x_prev, g_prev).item())
            alpha = ss / sy if sy > 0 else 1.0 / L_est
            alpha = min(max(alpha, 0.0), clamp / L_est)
        res.steps.append(alpha)
        B.pyro_axpby(x, x_prev, 1.0, 0.0)
        B.pyro_axpby(grad, g_prev, 1.0, 0.0)
        B.pyro_axpby(grad, x, -alpha, 1.0)
        if callback is not None:
            callback(k + 1, x)
    if track_objective:
        r = A(x, out=r) if isinstance(g, ConeGeometry3D) else A(x)
        B.pyro_axpby(p, r, -1.0, 1.0)
        _, tvv = B.pyro_tv(x, eps, lam, want_grad=False)
        res.objective.append(float(B.pyro_dot(r, r).item()) + lam * float(tvv.item()))
    res.x = x
    return res
