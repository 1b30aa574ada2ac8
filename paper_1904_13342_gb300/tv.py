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
pyro_axpby, and the BB step pyro_bb_dots / pyro_bb_update, which chooses
alpha on the device); an iteration reads nothing back to the host, so it can
be captured in a CUDA graph and replayed.
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


def _ops(g, storage=None):
    """A and A^T as closures with their workspaces; `storage` (cone beam
    only): the type of the projector's copy of the volume (FP16 / BF16
    storage of the FP32 iterate, FP32 accumulation), None for FP32."""
    if isinstance(g, ConeGeometry3D):
        ws = {}

        def A(x, out=None):
            st = x.dtype if storage is None else storage
            if "w" not in ws:
                ws["w"] = torch.empty(B.fp_cone3d_workspace_bytes(g, st), dtype=torch.uint8, device=x.device)
            if st == x.dtype:
                return B.pyro_fp_cone3d_ws(x, g, workspace=ws["w"], out=out)
            return B.pyro_fp_cone3d_ws_storage(x, g, st, workspace=ws["w"], out=out)

        def AT(y):
            if "wT" not in ws:
                ws["wT"] = torch.empty(B.fpT_cone3d_workspace_bytes(g), dtype=torch.uint8, device=y.device)
            return B.pyro_fpT_cone3d_ws(y, g, workspace=ws["wT"])

        return A, AT
    fp, fpT = (B.pyro_fp_fan2d_ws, B.pyro_fpT_fan2d_ws) if g.fan else (B.pyro_fp_par2d_ws, B.pyro_fpT_par2d_ws)
    ws = {}

    def work(t):  # one FP32 image: the transposed copy (FP) and accumulator (adjoint)
        if "w" not in ws:
            ws["w"] = torch.empty(B.fp2d_workspace_bytes(g, 1), dtype=torch.uint8, device=t.device)
        return ws["w"]

    return (lambda x, out=None: fp(x, g, workspace=work(x), out=out)), (lambda y: fpT(y, g, workspace=work(y)))


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
                   callback=None, graph: bool = False, storage: Optional[torch.dtype] = None) -> TVResult:
    """Minimise |A x - p|^2 + lam TV(x) (Eq. 7); p is one FP32 sinogram.

    The step size is chosen on the device (pyro_bb_dots / pyro_bb_update), so
    an iteration reads nothing back to the host unless `track_objective`
    (objective and step per iteration) or `callback(k, x)` asks for it.  With
    `graph=True` (and neither of those) one iteration is captured in a CUDA
    graph after two eager ones and replayed for the rest.  `storage`
    (cone beam): the forward projector reads an FP16 / BF16 copy of the FP32
    iterate (the half-storage pattern); the iterate, the gradients and every
    reduction stay FP32."""
    A, AT = _ops(g, storage)
    shape = tuple(g.volume_shape)
    dev = p.device
    if L_est is None:
        L_est = estimate_lipschitz(g, shape, dev)
    x = torch.zeros(shape, device=dev, dtype=torch.float32) if x0 is None else x0.clone().float()
    x_prev = torch.zeros_like(x)
    g_prev = torch.zeros_like(x)
    r = torch.empty_like(p)
    dots = torch.zeros(2, device=dev, dtype=torch.float32)
    alpha = torch.zeros(1, device=dev, dtype=torch.float32)
    alpha0, alpha_max = 1.0 / L_est, clamp / L_est
    res = TVResult(x)
    cone = isinstance(g, ConeGeometry3D)

    def step(first: bool):
        rr = A(x, out=r) if cone else A(x)
        B.pyro_axpby(p, rr, -1.0, 1.0)  # r = A x - p
        gd = AT(rr)
        grad, tvv = B.pyro_tv(x, eps, lam, base=gd, alpha=2.0, want_value=track_objective)
        if track_objective:
            res.objective.append(float(B.pyro_dot(rr, rr).item()) + lam * float(tvv.item()))
        if not first:
            B.pyro_bb_dots(x, x_prev, grad, g_prev, dots)
        B.pyro_bb_update(x, x_prev, grad, g_prev, dots, alpha0, alpha_max, first, alpha)
        if track_objective:
            res.steps.append(float(alpha.item()))

    if graph and n_iter > 2 and not track_objective and callback is None:
        step(True)
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            step(False)
        torch.cuda.current_stream(dev).wait_stream(side)
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg):
            step(False)
        for _ in range(n_iter - 2):
            cg.replay()
    else:
        for k in range(n_iter):
            step(k == 0)
            if callback is not None:
                callback(k + 1, x)
    if track_objective:
        rr = A(x, out=r) if cone else A(x)
        B.pyro_axpby(p, rr, -1.0, 1.0)
        _, tvv = B.pyro_tv(x, eps, lam, want_grad=False)
        res.objective.append(float(B.pyro_dot(rr, rr).item()) + lam * float(tvv.item()))
    res.x = x
    return res
