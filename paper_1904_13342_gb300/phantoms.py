"""Seeded synthetic inputs: random ellipse / ellipsoid phantoms and sinograms.

This module only draws inputs; it holds none of the projector, filter or
reconstruction arithmetic, so the CUDA path and the CPU oracle can both be
fed from it.

Phantom recipe (the workloads the paper reconstructs are Shepp-Logan-like
sums of ellipses / ellipsoids, Section "Phantoms"):
  * R = half the smallest field-of-view extent, R = min_i(N_i s_i) / 2;
  * each object has its centre uniform in [-0.8 R, 0.8 R] per axis,
    semi-axes uniform in [0.05 R, 0.4 R], an in-plane angle uniform in
    [0, pi) (2D) or a rotation uniform on SO(3) (3D, normalised Gaussian
    quaternion), and a density uniform in [-0.5, 1.0];
  * overlapping objects add;
  * a pixel / voxel holds the mean of ``supersample``^d sub-samples.
Random numbers come from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch


@dataclass
class Ellipses:
    centre: np.ndarray  # [n, 2] (x, y) mm
    axes: np.ndarray  # [n, 2] semi-axes mm
    angle: np.ndarray  # [n] rad
    density: np.ndarray  # [n]


@dataclass
class Ellipsoids:
    centre: np.ndarray  # [n, 3] (x, y, z) mm
    axes: np.ndarray  # [n, 3] semi-axes mm
    rot: np.ndarray  # [n, 3, 3]; columns are the ellipsoid's axes in world coordinates
    density: np.ndarray  # [n]


def random_ellipses(n: int, radius: float, seed: int) -> Ellipses:
    rng = np.random.default_rng(seed)
    centre = rng.uniform(-0.8, 0.8, size=(n, 2)) * radius
    axes = rng.uniform(0.05, 0.4, size=(n, 2)) * radius
    angle = rng.uniform(0.0, np.pi, size=n)
    density = rng.uniform(-0.5, 1.0, size=n)
    return Ellipses(centre, axes, angle, density)


def _quat_to_rot(q: np.ndarray) -> np.ndarray:
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def random_ellipsoids(n: int, radius: float, seed: int) -> Ellipsoids:
    rng = np.random.default_rng(seed)
    centre = rng.uniform(-0.8, 0.8, size=(n, 3)) * radius
    axes = rng.uniform(0.05, 0.4, size=(n, 3)) * radius
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    rot = np.stack([_quat_to_rot(qi) for qi in q])
    density = rng.uniform(-0.5, 1.0, size=n)
    return Ellipsoids(centre, axes, rot, density)


def _coords(n: int, s: float, ss: int, device, dtype) -> torch.Tensor:
    """Sub-sample coordinates (mm) of the n pixel centres, ss per pixel."""
    i = torch.arange(n, device=device, dtype=dtype)
    off = (torch.arange(ss, device=device, dtype=dtype) + 0.5) / ss - 0.5
    return ((i[:, None] + off[None, :]) - 0.5 * (n - 1)).reshape(-1) * s


def voxelize_ellipses(e: Ellipses, shape, spacing, supersample: int = 2, device="cpu",
                      dtype=torch.float64) -> torch.Tensor:
    """[ny, nx] image: mean of supersample^2 point samples per pixel."""
    ny, nx = shape
    sy, sx = spacing
    ss = supersample
    xs = _coords(nx, sx, ss, device, dtype)
    ys = _coords(ny, sy, ss, device, dtype)
    Y, X = torch.meshgrid(ys, xs, indexing="ij")
    img = torch.zeros_like(X)
    for c, a, ang, rho in zip(e.centre, e.axes, e.angle, e.density):
        ca, sa = float(np.cos(ang)), float(np.sin(ang))
        dx, dy = X - float(c[0]), Y - float(c[1])
        p = (ca * dx + sa * dy) / float(a[0])
        q = (-sa * dx + ca * dy) / float(a[1])
        img += float(rho) * (p * p + q * q <= 1.0).to(dtype)
    return img.reshape(ny, ss, nx, ss).mean(dim=(1, 3))


def voxelize_ellipsoids(e: Ellipsoids, shape, spacing, supersample: int = 2, device="cpu",
                        dtype=torch.float64, slab: int = 8) -> torch.Tensor:
    """[nz, ny, nx] volume: mean of supersample^3 point samples per voxel,
    evaluated ``slab`` z-slices at a time to bound memory."""
    nz, ny, nx = shape
    sz, sy, sx = spacing
    ss = supersample
    xs = _coords(nx, sx, ss, device, dtype)
    ys = _coords(ny, sy, ss, device, dtype)
    zs = _coords(nz, sz, ss, device, dtype)
    vol = torch.empty((nz, ny, nx), device=device, dtype=dtype)
    Y2, X2 = torch.meshgrid(ys, xs, indexing="ij")
    for z0 in range(0, nz, slab):
        z1 = min(nz, z0 + slab)
        zz = zs[z0 * ss:z1 * ss]
        Z = zz[:, None, None].expand(-1, Y2.shape[0], Y2.shape[1])
        acc = torch.zeros(Z.shape, device=device, dtype=dtype)
        for c, a, R, rho in zip(e.centre, e.axes, e.rot, e.density):
            dx, dy, dz = X2[None] - float(c[0]), Y2[None] - float(c[1]), Z - float(c[2])
            inside = torch.ones_like(acc, dtype=torch.bool)
            r2 = torch.zeros_like(acc)
            for ax in range(3):  # coordinate along the ellipsoid's own axis
                t = (float(R[0, ax]) * dx + float(R[1, ax]) * dy + float(R[2, ax]) * dz) / float(a[ax])
                r2 += t * t
            inside &= r2 <= 1.0
            acc += float(rho) * inside.to(dtype)
        vol[z0:z1] = acc.reshape(z1 - z0, ss, ny, ss, nx, ss).mean(dim=(1, 3, 5))
    return vol


def random_sinogram(shape, seed: int, smooth: int = 0) -> np.ndarray:
    """Seeded sinogram-shaped test data: N(0,1) noise plus a positive offset,
    optionally box-smoothed along the last axis ``smooth`` times."""
    rng = np.random.default_rng(seed)
    s = rng.standard_normal(size=shape) + 1.0
    for _ in range(smooth):
        s = (np.roll(s, 1, axis=-1) + s + np.roll(s, -1, axis=-1)) / 3.0
    return s


def random_volume(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=shape)


@dataclass
class Blobs:
    """Sum of anisotropic Gaussians rho * exp(-1/2 (X-c)^T S^-1 (X-c))."""
    centre: np.ndarray  # [n, d] mm
    cov: np.ndarray  # [n, d, d] mm^2
    density: np.ndarray  # [n]


def random_blobs(n: int, radius: float, dim: int, seed: int, sigma=(0.04, 0.12), spread: float = 0.5) -> Blobs:
    """Gaussian blobs: centres uniform in [-spread R, spread R] per axis,
    principal standard deviations uniform in sigma * R, random orientation,
    densities uniform in [0.2, 1.0]."""
    rng = np.random.default_rng(seed)
    centre = rng.uniform(-spread, spread, size=(n, dim)) * radius
    sd = rng.uniform(sigma[0], sigma[1], size=(n, dim)) * radius
    cov = np.empty((n, dim, dim))
    for i in range(n):
        q, _ = np.linalg.qr(rng.normal(size=(dim, dim)))
        cov[i] = q @ np.diag(sd[i] ** 2) @ q.T
    density = rng.uniform(0.2, 1.0, size=n)
    return Blobs(centre, cov, density)


def sample_blobs(b: Blobs, shape, spacing, device="cpu", dtype=torch.float64) -> torch.Tensor:
    """Point samples of the blob sum at the voxel centres ([ny, nx] or [nz, ny, nx])."""
    axes = [((torch.arange(n, device=device, dtype=dtype) - 0.5 * (n - 1)) * s) for n, s in zip(shape, spacing)]
    grids = torch.meshgrid(*axes, indexing="ij")  # (z,) y, x order
    X = torch.stack(list(reversed(grids)), dim=-1)  # [..., d] with x first
    out = torch.zeros(shape, device=device, dtype=dtype)
    for c, S, rho in zip(b.centre, b.cov, b.density):
        Si = torch.tensor(np.linalg.inv(S), device=device, dtype=dtype)
        r = X - torch.tensor(c, device=device, dtype=dtype)
        q = torch.einsum("...i,ij,...j->...", r, Si, r)
        out += float(rho) * torch.exp(-0.5 * q)
    return out
