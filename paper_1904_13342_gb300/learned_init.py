"""Learned initialiser for sparse-view cone-beam reconstruction.

Pipeline under test: FDK (Eq. 5) of a sparse full-scan sinogram -> residual
3D CNN (``cnn.ResidualCNN``) -> a few TV steps (Eq. 7) started from the
network's output.  Baseline: plain TV from x = 0 for many more steps.  The
network is trained on pairs the library makes itself: random ellipsoid
phantoms, ray-driven forward projection, FDK.

Quality is the PSNR over the field of view seen by every view,
10 log10(range^2 / MSE) with range = max - min of the true phantom; speed is
wall-clock seconds on the GPU (synchronised), training excluded.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import binding as B
from . import phantoms as ph
from .cnn import ResidualCNN
from .geometry import ConeGeometry3D
from .tv import estimate_lipschitz, tv_reconstruct


@dataclass
class SparseViewSetup:
    """A full-scan sparse-view cone-beam acquisition of an n^3 phantom."""
    n: int = 128
    spacing: float = 1.0
    views: int = 60
    detector: tuple = (200, 256)  # (rows, columns)
    detector_spacing: float = 1.0
    sid: float = 750.0
    sdd: float = 1200.0
    ellipsoids: int = 12

    def geometry(self) -> ConeGeometry3D:
        n, s, d = self.n, self.spacing, self.detector_spacing
        return ConeGeometry3D((n, n, n), (s, s, s), tuple(self.detector), (d, d), self.views, 2 * math.pi,
                              self.sid, self.sdd)


def fov_mask(setup: SparseViewSetup, device) -> torch.Tensor:
    """Voxels every view projects inside the detector: in-plane radius up to
    SID sin(fan half angle), and |z| up to (rows/2) s_v (SID - rho) / SDD at
    in-plane radius rho (the view that puts the voxel nearest the source)."""
    n, s = setup.n, setup.spacing
    c = (torch.arange(n, device=device, dtype=torch.float64) - (n - 1) / 2) * s
    z, y, x = torch.meshgrid(c, c, c, indexing="ij")
    rho = torch.sqrt(x * x + y * y)
    half_u = setup.detector[1] * setup.detector_spacing / 2
    half_v = setup.detector[0] * setup.detector_spacing / 2
    r_fov = setup.sid * math.sin(math.atan(half_u / setup.sdd))
    return (rho <= r_fov) & (z.abs() <= half_v * (setup.sid - rho) / setup.sdd)


def psnr(x: torch.Tensor, truth: torch.Tensor, mask: torch.Tensor) -> float:
    t = truth[mask].double()
    mse = float(((x[mask].double() - t) ** 2).mean())
    rng = float(t.max() - t.min())
    return 10.0 * math.log10(rng * rng / max(mse, 1e-300))


class PairMaker:
    """Phantom -> sinogram (ray-driven FP) -> FDK, all on the GPU."""

    def __init__(self, setup: SparseViewSetup, device="cuda", filt: int = B.SHEPP_LOGAN):
        self.setup = setup
        self.g = setup.geometry()
        self.dev = torch.device(device)
        self.filt = filt
        self._ws_fp = None
        self._ws_fdk = None

    def phantom(self, seed: int) -> torch.Tensor:
        s = self.setup
        e = ph.random_ellipsoids(s.ellipsoids, s.n * s.spacing / 2, seed)
        return ph.voxelize_ellipsoids(e, (s.n,) * 3, (s.spacing,) * 3, device=self.dev, dtype=torch.float32)

    def project(self, vol: torch.Tensor) -> torch.Tensor:
        if self._ws_fp is None:
            self._ws_fp = torch.empty(B.fp_cone3d_workspace_bytes(self.g), dtype=torch.uint8, device=self.dev)
        return B.pyro_fp_cone3d_ws(vol, self.g, workspace=self._ws_fp)

    def fdk(self, sino: torch.Tensor) -> torch.Tensor:
        return B.pyro_fdk(sino, self.g, kind=self.filt, redund=B.REDUND_FULL)

    def pairs(self, seeds: Sequence[int]):
        """(truth, sinogram, fdk) stacked over the seeds."""
        truth = torch.stack([self.phantom(s) for s in seeds])
        sino = self.project(truth)
        return truth, sino, self.fdk(sino)


def train_initializer(maker: PairMaker, seeds: Sequence[int], steps: int, batch: int = 2, lr: float = 1e-3,
                      seed: int = 0, log_every: int = 0) -> tuple:
    """Adam on the MSE between CNN(FDK) and the phantom; returns (net, losses)."""
    truth, _, fdk = maker.pairs(seeds)
    net = ResidualCNN(maker.dev, seed=seed)
    rng = np.random.default_rng(seed)
    losses = []
    for it in range(steps):
        idx = torch.as_tensor(rng.choice(len(seeds), batch, replace=False), device=maker.dev)
        step_lr = lr if it < 0.75 * steps else lr * 0.3
        losses.append(net.train_step(fdk[idx].contiguous(), truth[idx].contiguous(), lr=step_lr))
        if log_every and it % log_every == 0:
            print(f"step {it}: loss {losses[-1]:.3e}", flush=True)
    return net, losses


def _sync_time(fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def choose_lambda(maker: PairMaker, seeds: Sequence[int], lams: Sequence[float], n_iter: int, eps: float,
                  L_est: float) -> Dict[float, float]:
    """Mean PSNR of plain TV (n_iter steps from 0) per lambda on the given seeds."""
    truth, sino, _ = maker.pairs(seeds)
    mask = fov_mask(maker.setup, maker.dev)
    out = {}
    for lam in lams:
        vals = [psnr(tv_reconstruct(sino[i], maker.g, n_iter, lam, eps, L_est=L_est, graph=True).x, truth[i], mask)
                for i in range(len(seeds))]
        out[lam] = float(np.mean(vals))
    return out


@dataclass
class ABResult:
    """Per test phantom PSNRs (dB) and whole-set wall-clock seconds."""
    psnr_fdk: List[float] = field(default_factory=list)
    psnr_cnn: List[float] = field(default_factory=list)
    psnr_learned: List[float] = field(default_factory=list)  # CNN + short TV
    psnr_short_tv: List[float] = field(default_factory=list)  # the same short TV from x = 0
    psnr_plain: List[float] = field(default_factory=list)  # long TV from x = 0
    psnr_to_target: List[float] = field(default_factory=list)  # CNN + iters_to_target TV
    curve_plain: List[float] = field(default_factory=list)  # mean PSNR after k steps from x = 0
    curve_learned: List[float] = field(default_factory=list)  # mean PSNR after k steps from the CNN output
    iters_to_target: Optional[int] = None  # TV steps from the CNN output to the long TV's mean PSNR
    seconds_learned: float = 0.0
    seconds_plain: float = 0.0
    seconds_short_tv: float = 0.0
    seconds_to_target: Optional[float] = None

    def summary(self) -> dict:
        m = lambda v: float(np.mean(v)) if v else float("nan")
        return {"psnr_fdk": m(self.psnr_fdk), "psnr_cnn": m(self.psnr_cnn), "psnr_learned": m(self.psnr_learned),
                "psnr_short_tv": m(self.psnr_short_tv), "psnr_plain": m(self.psnr_plain),
                "psnr_to_target": m(self.psnr_to_target), "iters_to_target": self.iters_to_target,
                "seconds_learned": self.seconds_learned, "seconds_plain": self.seconds_plain,
                "seconds_short_tv": self.seconds_short_tv, "seconds_to_target": self.seconds_to_target,
                "n": len(self.psnr_plain)}


def _curves(maker, sino, truth, mask, x0s, lam, eps, L_est, n_iter) -> List[float]:
    """Mean PSNR over the phantoms after each of n_iter TV steps (k = 0..n_iter)."""
    n = sino.shape[0]
    acc = np.zeros((n, n_iter + 1))
    for i in range(n):
        x0 = None if x0s is None else x0s[i]
        acc[i, 0] = psnr(torch.zeros_like(truth[i]) if x0 is None else x0, truth[i], mask)

        def cb(k, x, i=i):
            acc[i, k] = psnr(x, truth[i], mask)

        tv_reconstruct(sino[i], maker.g, n_iter, lam, eps, L_est=L_est, x0=x0, callback=cb)
    return acc.mean(axis=0).tolist()


def ab_test(maker: PairMaker, net: ResidualCNN, seeds: Sequence[int], lam: float, eps: float, L_est: float,
            short_iter: int = 20, long_iter: int = 200, cnn_batch: int = 4, curves: bool = True) -> ABResult:
    """FDK -> CNN -> TV against plain TV from x = 0 on the test phantoms
    `seeds`: (a) a fixed budget, short_iter steps after the CNN against
    long_iter plain steps; (b) time to the plain path's mean PSNR, the number
    of TV steps after the CNN found on an untimed pass that records the PSNR
    after every step.  Each timed path runs from the sinograms in device
    memory to the reconstructions in device memory."""
    truth, sino, _ = maker.pairs(seeds)
    mask = fov_mask(maker.setup, maker.dev)
    res = ABResult()
    n = len(seeds)

    def learned(k):
        fdk = maker.fdk(sino)
        init = torch.cat([net.forward(fdk[i:i + cnn_batch].contiguous()) for i in range(0, n, cnn_batch)])
        xs = [tv_reconstruct(sino[i], maker.g, k, lam, eps, L_est=L_est, x0=init[i], graph=True).x for i in range(n)]
        return fdk, init, xs

    (fdk, init, xs), res.seconds_learned = _sync_time(lambda: learned(short_iter))
    plain, res.seconds_plain = _sync_time(
        lambda: [tv_reconstruct(sino[i], maker.g, long_iter, lam, eps, L_est=L_est, graph=True).x for i in range(n)])
    short, res.seconds_short_tv = _sync_time(
        lambda: [tv_reconstruct(sino[i], maker.g, short_iter, lam, eps, L_est=L_est, graph=True).x for i in range(n)])
    for i in range(n):
        res.psnr_fdk.append(psnr(fdk[i], truth[i], mask))
        res.psnr_cnn.append(psnr(init[i], truth[i], mask))
        res.psnr_learned.append(psnr(xs[i], truth[i], mask))
        res.psnr_short_tv.append(psnr(short[i], truth[i], mask))
        res.psnr_plain.append(psnr(plain[i], truth[i], mask))
    if curves:
        target = float(np.mean(res.psnr_plain))
        res.curve_plain = _curves(maker, sino, truth, mask, None, lam, eps, L_est, long_iter)
        res.curve_learned = _curves(maker, sino, truth, mask, init, lam, eps, L_est, long_iter)
        hit = [k for k, v in enumerate(res.curve_learned) if v >= target]
        if hit:
            res.iters_to_target = hit[0]
            (_, _, xt), res.seconds_to_target = _sync_time(lambda: learned(res.iters_to_target))
            res.psnr_to_target = [psnr(xt[i], truth[i], mask) for i in range(n)]
    return res


def lipschitz(maker: PairMaker) -> float:
    return estimate_lipschitz(maker.g, (maker.setup.n,) * 3, maker.dev)
