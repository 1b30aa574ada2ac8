"""The paper's two small 2D experiments, run on the library's kernels.

* Filter learning (Section "Filter Learning", Eq. 6): parallel-beam FBP as
  a network x = A_bp F^H K F p whose only trainable part is the filter
  spectrum K, initialised with the frequency-sampled ramp |m| / (Pn tau).
  Trained on (sinogram, phantom) pairs, K is fitted by least squares; the
  paper reports the result resembles the spectrum of the spatial Ram-Lak
  kernel, which removes the ramp's DC offset.  On the library's discrete
  operators the fitted K reconstructs at least as well as Ram-Lak (a
  feasible point of the same problem), its low bins need not match it.
* Sparse-view TV (Section "Iterative Reconstruction", Eq. 7): 30 parallel
  views over 180 degrees with 2 % Gaussian noise (sigma = 0.02 max p);
  TV iteration against Ram-Lak FBP.

Phantoms are random ellipses (seeded); every operator is a library call.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np
import torch

from . import binding as B
from . import phantoms as ph
from .autograd import back_project, filter_taps, forward_project, ramp_filter
from .geometry import ParallelGeometry2D
from .tv import estimate_lipschitz, tv_reconstruct


def disk_mask(n: int, device) -> torch.Tensor:
    c = torch.arange(n, device=device, dtype=torch.float64) - (n - 1) / 2
    y, x = torch.meshgrid(c, c, indexing="ij")
    return (x * x + y * y) <= (0.5 * (n - 1)) ** 2


def psnr2d(x: torch.Tensor, truth: torch.Tensor, mask: torch.Tensor) -> float:
    t = truth[mask].double()
    mse = float(((x[mask].double() - t) ** 2).mean())
    rng = float(t.max() - t.min())
    return 10.0 * math.log10(rng * rng / max(mse, 1e-300))


def phantoms2d(n: int, seeds: Sequence[int], device) -> torch.Tensor:
    return torch.stack([ph.voxelize_ellipses(ph.random_ellipses(10, n / 2, s), (n, n), (1.0, 1.0), device=device,
                                             dtype=torch.float32) for s in seeds])


@dataclass
class FilterLearning:
    K0: torch.Tensor  # ramp initialisation
    K: torch.Tensor  # learned
    K_ramlak: torch.Tensor
    losses: List[float] = field(default_factory=list)  # per loss evaluation
    loss_ramlak: float = 0.0  # the same loss with K = Ram-Lak's spectrum
    # |K - K_ramlak| / |K0 - K_ramlak| over the low band (the first `band` of the bins)
    dist_to_ramlak: List[float] = field(default_factory=list)


def learn_filter(n: int = 128, views: int = 180, iters: int = 40, seeds=range(1000, 1016), device="cuda",
                 band: float = 1.0 / 16) -> FilterLearning:
    """Fit K (ramp initialisation) by L-BFGS on the full training batch: the
    loss is quadratic in K, so its optimiser is a least-squares solve.  An
    element-wise adaptive optimiser would move the many bins whose gradient
    is near zero by its step size each iteration; L-BFGS leaves them."""
    dev = torch.device(device)
    nu = int(math.ceil(n * math.sqrt(2))) | 1
    g = ParallelGeometry2D((n, n), (1.0, 1.0), nu, 1.0, views, math.pi)
    truth = phantoms2d(n, list(seeds), dev)
    with torch.no_grad():
        sino = forward_project(truth, g)
    K0 = filter_taps(B.RAMP, nu, 1.0, dev)
    K_rl = filter_taps(B.RAMLAK, nu, 1.0, dev)
    K = torch.nn.Parameter(K0.clone())
    opt = torch.optim.LBFGS([K], lr=1.0, max_iter=iters, history_size=20, line_search_fn="strong_wolfe",
                            tolerance_grad=0.0, tolerance_change=0.0)
    mask = disk_mask(n, dev)
    scale = math.pi / views
    res = FilterLearning(K0, K.data, K_rl)
    b = max(2, int(band * K0.numel()))
    d0 = float(torch.linalg.norm(K0[:b] - K_rl[:b]))

    def closure():
        opt.zero_grad()
        x = back_project(ramp_filter(sino, 1.0, K), g, B.W_NONE, scale)
        loss = ((x - truth)[:, mask] ** 2).mean()
        loss.backward()
        res.losses.append(float(loss.item()))
        res.dist_to_ramlak.append(float(torch.linalg.norm(K.data[:b] - K_rl[:b])) / d0)
        return loss

    opt.step(closure)
    res.K = K.data.clone()
    with torch.no_grad():
        x = back_project(ramp_filter(sino, 1.0, K_rl), g, B.W_NONE, scale)
        res.loss_ramlak = float(((x - truth)[:, mask] ** 2).mean())
        x = back_project(ramp_filter(sino, 1.0, res.K), g, B.W_NONE, scale)
        res.losses.append(float(((x - truth)[:, mask] ** 2).mean()))
    return res


@dataclass
class SparseView2D:
    psnr_fbp: List[float] = field(default_factory=list)
    psnr_tv: List[float] = field(default_factory=list)
    lam: float = 0.0


def sparse_view_tv(n: int = 256, views: int = 30, noise: float = 0.02, iters: int = 200, lams=(0.3, 1.0, 3.0, 10.0),
                   tune_seeds=range(1000, 1004), test_seeds=range(0, 8), device="cuda") -> SparseView2D:
    """Ram-Lak FBP against TV (lambda from a grid on tune_seeds) on test_seeds."""
    dev = torch.device(device)
    nu = int(math.ceil(n * math.sqrt(2))) | 1
    g = ParallelGeometry2D((n, n), (1.0, 1.0), nu, 1.0, views, math.pi)
    mask = disk_mask(n, dev)
    L_est = estimate_lipschitz(g, (n, n), dev)

    def data(seeds, noise_seed):
        truth = phantoms2d(n, list(seeds), dev)
        p = B.pyro_fp_par2d(truth, g)
        gen = torch.Generator(device="cpu").manual_seed(noise_seed)
        sigma = noise * p.abs().amax(dim=(1, 2), keepdim=True)
        p = p + sigma * torch.randn(p.shape, generator=gen).to(dev)
        return truth, p.contiguous()

    def tv(p, lam, eps):
        return tv_reconstruct(p, g, iters, lam, eps, L_est=L_est).x

    t_tune, p_tune = data(tune_seeds, 7)
    eps = 1e-3
    score = {lam: float(np.mean([psnr2d(tv(p_tune[i], lam, eps), t_tune[i], mask) for i in range(len(t_tune))]))
             for lam in lams}
    lam = max(score, key=score.get)
    truth, p = data(test_seeds, 8)
    fbp = B.pyro_fbp_par2d(p, g, kind=B.RAMLAK)
    out = SparseView2D(lam=lam)
    for i in range(len(truth)):
        out.psnr_fbp.append(psnr2d(fbp[i], truth[i], mask))
        out.psnr_tv.append(psnr2d(tv(p[i], lam, eps), truth[i], mask))
    return out
