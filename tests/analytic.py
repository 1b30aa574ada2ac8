"""Closed-form line integrals of ellipse / ellipsoid phantoms (test pins).

For a line X(t) = a + t d (|d| = 1) and an ellipsoid {X : |D^-1 R^T (X - c)| <= 1}
of density rho, the intersection is the interval between the roots of the
quadratic A t^2 + 2 B t + C = 0 with A = |D^-1 R^T d|^2,
B = (D^-1 R^T d).(D^-1 R^T (a - c)), C = |D^-1 R^T (a - c)|^2 - 1, so the line
integral is rho * 2 sqrt(B^2 - A C) / A (0 when B^2 < A C).  In 2D this is the
textbook ellipse projection of Kak & Slaney.  These chords are computed here
independently of the oracle's sampled line integrals.
"""
from __future__ import annotations

import numpy as np


def ellipse_line_integrals(ell, a: np.ndarray, d: np.ndarray) -> np.ndarray:
    """a, d: [R, 2] (d unit). Returns [R]."""
    out = np.zeros(a.shape[0])
    for c, ax, ang, rho in zip(ell.centre, ell.axes, ell.angle, ell.density):
        ca, sa = np.cos(ang), np.sin(ang)
        Rt = np.array([[ca, sa], [-sa, ca]])  # world -> ellipse frame
        inv = 1.0 / np.asarray(ax)
        dd = (d @ Rt.T) * inv
        aa = ((a - c) @ Rt.T) * inv
        A = np.sum(dd * dd, axis=1)
        B = np.sum(dd * aa, axis=1)
        C = np.sum(aa * aa, axis=1) - 1.0
        disc = B * B - A * C
        out += rho * np.where(disc > 0, 2.0 * np.sqrt(np.maximum(disc, 0.0)) / A, 0.0)
    return out


def ellipsoid_line_integrals(ell, a: np.ndarray, d: np.ndarray) -> np.ndarray:
    """a, d: [R, 3] (d unit). Returns [R]."""
    out = np.zeros(a.shape[0])
    for c, ax, Rm, rho in zip(ell.centre, ell.axes, ell.rot, ell.density):
        inv = 1.0 / np.asarray(ax)
        dd = (d @ Rm) * inv  # R^T d for each row
        aa = ((a - c) @ Rm) * inv
        A = np.sum(dd * dd, axis=1)
        B = np.sum(dd * aa, axis=1)
        C = np.sum(aa * aa, axis=1) - 1.0
        disc = B * B - A * C
        out += rho * np.where(disc > 0, 2.0 * np.sqrt(np.maximum(disc, 0.0)) / A, 0.0)
    return out


# ---- ray geometry written out independently from the oracle's code ----

def parallel_rays(angles, nu, su):
    """Line through u_k e_u with direction c, for every (view, bin)."""
    b = np.asarray(angles)[:, None]
    u = (np.arange(nu) - 0.5 * (nu - 1))[None, :] * su
    c = np.stack([np.cos(b) + 0 * u, np.sin(b) + 0 * u], axis=-1)
    eu = np.stack([-np.sin(b) + 0 * u, np.cos(b) + 0 * u], axis=-1)
    a = u[..., None] * eu
    return a.reshape(-1, 2), c.reshape(-1, 2)


def fan_rays(angles, nu, su, sid, sdd):
    """Line from the source -SID c to the detector bin (SDD-SID) c + u e_u."""
    b = np.asarray(angles)[:, None]
    u = (np.arange(nu) - 0.5 * (nu - 1))[None, :] * su
    c = np.stack([np.cos(b) + 0 * u, np.sin(b) + 0 * u], axis=-1)
    eu = np.stack([-np.sin(b) + 0 * u, np.cos(b) + 0 * u], axis=-1)
    src = -sid * c
    det = (sdd - sid) * c + u[..., None] * eu
    d = det - src
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    return src.reshape(-1, 2), d.reshape(-1, 2)


def cone_rays(angles, nu, nv, su, sv, sid, sdd):
    """Line from the source to detector pixel (k, l) of a flat detector."""
    b = np.asarray(angles)[:, None, None]
    u = ((np.arange(nu) - 0.5 * (nu - 1)) * su)[None, None, :]
    v = ((np.arange(nv) - 0.5 * (nv - 1)) * sv)[None, :, None]
    z = 0 * (b + u + v)
    c = np.stack([np.cos(b) + z, np.sin(b) + z, z], axis=-1)
    eu = np.stack([-np.sin(b) + z, np.cos(b) + z, z], axis=-1)
    ev = np.stack([z, z, 1 + z], axis=-1)
    src = -sid * c
    det = (sdd - sid) * c + (u + z)[..., None] * eu + (v + z)[..., None] * ev
    d = det - src
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    return src.reshape(-1, 3), d.reshape(-1, 3)


def disk_parallel_sinogram(radius, mu, centre, angles, nu, su):
    """Analytic parallel projections of a uniform disk: 2 mu sqrt(r^2 - s^2)."""
    b = np.asarray(angles)[:, None]
    u = (np.arange(nu) - 0.5 * (nu - 1))[None, :] * su
    s = u - (centre[0] * -np.sin(b) + centre[1] * np.cos(b))
    return 2.0 * mu * np.sqrt(np.maximum(radius * radius - s * s, 0.0))


def blob_line_integrals(blobs, a: np.ndarray, d: np.ndarray) -> np.ndarray:
    """Line integrals of a sum of Gaussians rho exp(-1/2 r^T S^-1 r) along
    X = a + t d: with r0 = a - c, alpha = d^T S^-1 d, beta = d^T S^-1 r0,
    gamma = r0^T S^-1 r0, the integral is
    rho sqrt(2 pi / alpha) exp(-1/2 (gamma - beta^2 / alpha))."""
    out = np.zeros(a.shape[0])
    for c, S, rho in zip(blobs.centre, blobs.cov, blobs.density):
        Si = np.linalg.inv(S)
        r0 = a - c
        al = np.einsum("ri,ij,rj->r", d, Si, d)
        be = np.einsum("ri,ij,rj->r", d, Si, r0)
        ga = np.einsum("ri,ij,rj->r", r0, Si, r0)
        out += rho * np.sqrt(2 * np.pi / al) * np.exp(-0.5 * (ga - be * be / al))
    return out


def cone_sinogram(ell, angles, det_shape, det_spacing, sid, sdd, chunk=16):
    """[V, nv, nu] analytic cone-beam projections of an ellipsoid phantom
    (torch float64 on the CPU, `chunk` views at a time)."""
    import torch

    nv, nu = det_shape
    sv, su = det_spacing
    u = (torch.arange(nu, dtype=torch.float64) - 0.5 * (nu - 1)) * su
    v = (torch.arange(nv, dtype=torch.float64) - 0.5 * (nv - 1)) * sv
    V, U = torch.meshgrid(v, u, indexing="ij")
    out = np.empty((len(angles), nv, nu))
    for j0 in range(0, len(angles), chunk):
        b = torch.as_tensor(np.asarray(angles[j0:j0 + chunk], dtype=np.float64))[:, None, None]
        cb, sb = torch.cos(b), torch.sin(b)
        # source -SID c and direction to the pixel (SDD-SID) c + u e_u + v e_v
        src = torch.stack([-sid * cb, -sid * sb, torch.zeros_like(b)], -1).expand(-1, nv, nu, 3)
        d = torch.stack([sdd * cb - U * sb, sdd * sb + U * cb, V.expand_as(U * cb)], -1)
        d = d / torch.linalg.norm(d, dim=-1, keepdim=True)
        acc = torch.zeros(d.shape[:-1], dtype=torch.float64)
        for c, ax, Rm, rho in zip(ell.centre, ell.axes, ell.rot, ell.density):
            R = torch.as_tensor(Rm) / torch.as_tensor(ax)[None, :]
            dd = d @ R
            aa = (src - torch.as_tensor(c)) @ R
            A = (dd * dd).sum(-1)
            Bq = (dd * aa).sum(-1)
            C = (aa * aa).sum(-1) - 1.0
            disc = Bq * Bq - A * C
            acc += rho * torch.where(disc > 0, 2.0 * torch.sqrt(disc.clamp_min(0.0)) / A, torch.zeros_like(A))
        out[j0:j0 + chunk] = acc.numpy()
    return out


def fan_sinogram(ell, angles, nu, su, sid, sdd):
    a, d = fan_rays(angles, nu, su, sid, sdd)
    return ellipse_line_integrals(ell, a, d).reshape(len(angles), nu)


def parallel_sinogram(ell, angles, nu, su):
    a, d = parallel_rays(angles, nu, su)
    return ellipse_line_integrals(ell, a, d).reshape(len(angles), nu)
