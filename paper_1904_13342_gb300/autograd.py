"""The operators as differentiable layers (paper, Section "The Known
Operator": the gradient of A is A^T and vice versa).

Each layer is a torch.autograd.Function whose forward and backward are calls
of the CUDA library (through ``binding``):

* ``forward_project(x, g)``: forward = ray-driven FP; backward = its exact
  adjoint A^T (``pyro_fpT_*``).  With ``grad_mode="paper"`` the backward is
  the paper's unmatched voxel-driven back-projection instead, scaled so that
  it approximates A^T (rays at depth L are spaced tau L / SDD apart, so one
  voxel of size s^d meets about s^d / spacing rays): parallel
  scale = s^2 / tau; fan omega = SID/L, scale = s^2 SDD / (tau SID);
  cone omega = (SID/L)^2, scale = s^3 SDD^2 / (tau_u tau_v SID^2).
* ``back_project(y, g, weight, scale)``: forward = voxel-driven BP; backward
  = its transpose (``pyro_bpT_*``).
* ``ramp_filter(p, tau, K)``: forward = F^H K F on each detector row (Eq. 4);
  the operator is symmetric (real even K), so d/dp is the same filter, and
  d/dK comes from ``pyro_filter_grad_K`` (Eq. 6, filter learning).
* ``fdk(p, g, K)``: the FDK network of Eq. 5 with an optional learnable K.
"""
from __future__ import annotations

import math
from typing import Optional

import torch

from . import binding as B
from .geometry import ConeGeometry3D, Geometry2D


def _is3d(g) -> bool:
    return isinstance(g, ConeGeometry3D)


def _fp(x, g):
    if _is3d(g):
        return B.pyro_fp_cone3d_ws(x, g)
    return B.pyro_fp_fan2d(x, g) if g.fan else B.pyro_fp_par2d(x, g)


def _fpT(y, g):
    if _is3d(g):
        return B.pyro_fpT_cone3d_ws(y, g)
    return B.pyro_fpT_fan2d(y, g) if g.fan else B.pyro_fpT_par2d(y, g)


def _bp(y, g, weight, scale):
    if _is3d(g):
        return B.pyro_bp_cone3d(y, g, weight, scale)
    return B.pyro_bp_fan2d(y, g, weight, scale) if g.fan else B.pyro_bp_par2d(y, g, weight, scale)


def _bpT(x, g, weight, scale):
    if _is3d(g):
        return B.pyro_bpT_cone3d(x, g, weight, scale)
    return B.pyro_bpT_fan2d(x, g, weight, scale) if g.fan else B.pyro_bpT_par2d(x, g, weight, scale)


def paper_adjoint_weighting(g):
    """(weight, scale) that make the voxel-driven BP approximate A^T."""
    if _is3d(g):
        sz, sy, sx = g.volume_spacing
        sv, su = g.detector_spacing
        return B.W_INV_L2, sx * sy * sz * g.sdd ** 2 / (su * sv * g.sid ** 2)
    sy, sx = g.volume_spacing
    if g.fan:
        return B.W_INV_L, sx * sy * g.sdd / (g.detector_spacing * g.sid)
    return B.W_NONE, sx * sy / g.detector_spacing


class _ForwardProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, g, grad_mode):
        ctx.g, ctx.mode = g, grad_mode
        return _fp(x.contiguous(), g)

    @staticmethod
    def backward(ctx, gy):
        gy = gy.contiguous()
        if ctx.mode == "paper":
            w, s = paper_adjoint_weighting(ctx.g)
            return _bp(gy, ctx.g, w, s), None, None
        return _fpT(gy, ctx.g), None, None


class _BackProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, g, weight, scale):
        ctx.g, ctx.weight, ctx.scale = g, weight, scale
        return _bp(y.contiguous(), g, weight, scale)

    @staticmethod
    def backward(ctx, gx):
        return _bpT(gx.contiguous(), ctx.g, ctx.weight, ctx.scale), None, None, None


class _RampFilter(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p, K, tau):
        p = p.contiguous()
        ctx.save_for_backward(p, K)
        ctx.tau = tau
        return B.pyro_filter_rows(p, tau, B.FILTER_CUSTOM, custom_K=K.contiguous())

    @staticmethod
    def backward(ctx, gq):
        p, K = ctx.saved_tensors
        gq = gq.contiguous()
        gp = B.pyro_filter_rows(gq, ctx.tau, B.FILTER_CUSTOM, custom_K=K.contiguous()) if ctx.needs_input_grad[0] \
            else None
        gK = None
        if ctx.needs_input_grad[1]:
            nu = p.shape[-1]
            gK = B.pyro_filter_grad_K(p.float().reshape(-1, nu), gq.float().reshape(-1, nu))
        return gp, gK, None


def forward_project(x: torch.Tensor, g, grad_mode: str = "exact") -> torch.Tensor:
    """A x; backward A^T (exact) or the paper's scaled voxel-driven BP."""
    if grad_mode not in ("exact", "paper"):
        raise ValueError("grad_mode must be 'exact' or 'paper'")
    return _ForwardProject.apply(x, g, grad_mode)


def back_project(y: torch.Tensor, g, weight: int = B.W_NONE, scale: float = 1.0) -> torch.Tensor:
    return _BackProject.apply(y, g, weight, scale)


def ramp_filter(p: torch.Tensor, tau: float, K: torch.Tensor) -> torch.Tensor:
    """F^H K F along the last axis with a (learnable) K of pad_length(nu)//2+1 taps."""
    return _RampFilter.apply(p, K, tau)


def filter_taps(kind: int, nu: int, tau: float, device) -> torch.Tensor:
    """K[0..pn/2] of a built-in filter (computed by the library) on `device`."""
    return B.pyro_filter_spectrum(kind, nu, tau).to(device)


def _weighted(p, g, redund):
    """W_red W_cos p (a weighted copy; the weights are the library's)."""
    w = p.contiguous().clone()
    if _is3d(g):
        return B.pyro_weights3d(w, g, cosine=True, redund=redund)
    return B.pyro_weights2d(w, g, cosine=True, redund=redund)


class _FDK(torch.autograd.Function):
    """x = A_bp F^H K F W p (Eq. 5).  Forward: the fused library FDK with a
    custom K.  Backward: g_q = A_bp^T g_x; g_p = W F^H K F g_q (the filter and
    W are symmetric); g_K from the spectra of W p and g_q (Eq. 6)."""

    @staticmethod
    def forward(ctx, p, K, g, redund):
        p = p.contiguous()
        ctx.save_for_backward(p, K)
        ctx.g, ctx.redund = g, redund
        return B.pyro_fdk(p, g, kind=B.FILTER_CUSTOM, redund=redund, custom_K=K.contiguous())

    @staticmethod
    def backward(ctx, gx):
        p, K = ctx.saved_tensors
        g = ctx.g
        scale = abs(g.angular_range) / g.number_of_projections
        gq = B.pyro_bpT_cone3d(gx.contiguous().float(), g, B.W_INV_L2, scale)
        tau = g.detector_spacing[1] * g.sid / g.sdd
        gp = gK = None
        if ctx.needs_input_grad[0]:
            gp = B.pyro_filter_rows(gq, tau, B.FILTER_CUSTOM, custom_K=K.contiguous())
            B.pyro_weights3d(gp, g, cosine=True, redund=ctx.redund)
            gp = gp.to(p.dtype)
        if ctx.needs_input_grad[1]:
            wp = _weighted(p.float(), g, ctx.redund)
            nu = p.shape[-1]
            gK = B.pyro_filter_grad_K(wp.reshape(-1, nu), gq.reshape(-1, nu))
        return gp, gK, None, None


class FDK(torch.nn.Module):
    """The FDK network of Eq. 5 as a layer: x = A^T F^H K F W_red W_cos p,
    with the filter K (pad_length(nu)//2+1 taps) optionally trainable."""

    def __init__(self, g: ConeGeometry3D, kind: int = B.SHEPP_LOGAN, redund: int = B.REDUND_PARKER,
                 learnable: bool = False, device="cuda"):
        super().__init__()
        self.g, self.redund = g, redund
        self.tau = g.detector_spacing[1] * g.sid / g.sdd
        self.K = torch.nn.Parameter(filter_taps(kind, g.detector_shape[1], self.tau, device),
                                    requires_grad=learnable)

    def forward(self, p: torch.Tensor) -> torch.Tensor:
        return _FDK.apply(p, self.K, self.g, self.redund)


def redundancy_table(g: ConeGeometry3D, device, redund: int = B.REDUND_PARKER) -> torch.Tensor:
    """[V, nu] redundancy weights of the geometry (computed by the library):
    Parker's for the short scan, or REDUND_SCAN's for the geometry's range."""
    from dataclasses import replace

    g1 = replace(g, detector_shape=(1, g.detector_shape[1]), _keep=[])
    ones = torch.ones((g.number_of_projections, 1, g.detector_shape[1]), device=device, dtype=torch.float32)
    return B.pyro_weights3d(ones, g1, cosine=False, redund=redund)[:, 0].contiguous()


def parker_table(g: ConeGeometry3D, device) -> torch.Tensor:
    """[V, nu] Parker weights of the geometry (computed by the library)."""
    return redundancy_table(g, device, B.REDUND_PARKER)


class _FDKTable(torch.autograd.Function):
    """x = A_bp F^H K F (W_cos * table) p, with the redundancy weights a
    learnable [V, nu] table (Section "Geometric Correction Weights").
    Backward: g_q = A_bp^T g_x; g_f = F^H K F g_q (the filter is symmetric);
    g_table = sum over rows and batch of (W_cos p) g_f; g_p = W_cos table g_f."""

    @staticmethod
    def forward(ctx, p, table, K, g):
        p = p.contiguous().float()
        ctx.save_for_backward(p, table, K)
        ctx.g = g
        tau = g.detector_spacing[1] * g.sid / g.sdd
        w = B.pyro_weights3d_table(p.clone(), g, table.detach(), cosine=True)
        q = B.pyro_filter_rows(w, tau, B.FILTER_CUSTOM, custom_K=K.detach().contiguous())
        return B.pyro_bp_cone3d(q, g, B.W_INV_L2, abs(g.angular_range) / g.number_of_projections)

    @staticmethod
    def backward(ctx, gx):
        p, table, K = ctx.saved_tensors
        g = ctx.g
        tau = g.detector_spacing[1] * g.sid / g.sdd
        gq = B.pyro_bpT_cone3d(gx.contiguous().float(), g, B.W_INV_L2,
                               abs(g.angular_range) / g.number_of_projections)
        gf = B.pyro_filter_rows(gq, tau, B.FILTER_CUSTOM, custom_K=K.detach().contiguous())
        gp = gt = gK = None
        if ctx.needs_input_grad[1]:
            wc = B.pyro_weights3d(p.clone(), g, cosine=True, redund=B.REDUND_NONE)
            gt = B.pyro_redundancy_grad(wc, gf)
        if ctx.needs_input_grad[2]:
            wp = B.pyro_weights3d_table(p.clone(), g, table.detach(), cosine=True)
            nu = p.shape[-1]
            gK = B.pyro_filter_grad_K(wp.reshape(-1, nu), gq.reshape(-1, nu))
        if ctx.needs_input_grad[0]:
            gp = B.pyro_weights3d_table(gf, g, table.detach(), cosine=True)
        return gp, gt, gK, None


class RedundancyFDK(torch.nn.Module):
    """FDK (Eq. 5) whose redundancy weights W_red are a learnable [V, nu]
    table; the filter K is fixed unless `learnable_filter`.  `init`:
    "parker", "scan" (the weighting for the geometry's own scan range, any
    range up to 2 pi), "full" (1/2 everywhere) or a [V, nu] tensor."""

    def __init__(self, g: ConeGeometry3D, kind: int = B.SHEPP_LOGAN, init="parker", learnable_filter: bool = False,
                 device="cuda"):
        super().__init__()
        self.g = g
        tau = g.detector_spacing[1] * g.sid / g.sdd
        if isinstance(init, torch.Tensor):
            t = init.to(device=device, dtype=torch.float32)
        elif init == "parker":
            t = parker_table(g, device)
        elif init == "scan":
            t = redundancy_table(g, device, B.REDUND_SCAN)
        elif init == "full":
            t = torch.full((g.number_of_projections, g.detector_shape[1]), 0.5, device=device)
        else:
            raise ValueError("init must be 'parker', 'scan', 'full' or a tensor")
        self.table = torch.nn.Parameter(t.clone())
        self.K = torch.nn.Parameter(filter_taps(kind, g.detector_shape[1], tau, device),
                                    requires_grad=learnable_filter)

    def forward(self, p: torch.Tensor) -> torch.Tensor:
        return _FDKTable.apply(p, self.table, self.K, self.g)
