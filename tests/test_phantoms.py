"""Pins of the seeded phantom voxelisers (CPU): the voxelised mass, centroid
and second moments of random ellipses / ellipsoids against their closed
forms.  A solid ellipsoid with semi-axes a, rotation R (columns = its axes in
world coordinates) and centre c has volume V = 4/3 pi a0 a1 a2, first moment
V c and second moment V/5 R diag(a^2) R^T + V c c^T (an ellipse: V = pi a0
a1, V/4 R diag(a^2) R^T + V c c^T).  The second moment fixes the rotation
convention (the transposed rotation misses the gate by about 3-7x), the
mass the axis and spacing scales.  Only objects wholly inside the field of
view are kept, so that the closed forms apply."""
import numpy as np
import pytest

from paper_1904_13342_gb300 import phantoms as ph


def _moments(img, spacing):
    """mass, first and second moments of a [.., y, x] or [z, y, x] array
    about the centred grid (coordinates in mm, x first)."""
    axes = [(np.arange(n) - 0.5 * (n - 1)) * s for n, s in zip(img.shape, spacing)]
    grids = np.meshgrid(*axes, indexing="ij")[::-1]  # x, y[, z]
    P = np.stack(grids, -1).reshape(-1, img.ndim)
    f = img.reshape(-1)
    dV = float(np.prod(spacing))
    return f.sum() * dV, P.T @ f * dV, (P * f[:, None]).T @ P * dV


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ellipsoid_voxeliser_mass_and_moments(seed):
    n, s = 96, 0.5
    half = n * s / 2
    e = ph.random_ellipsoids(12, half, seed)
    ext = np.sqrt(np.einsum("nik,nk->ni", e.rot ** 2, e.axes ** 2))  # half-extent along each world axis
    keep = np.all(np.abs(e.centre) + ext <= half, axis=1)
    assert keep.sum() >= 6
    sub = ph.Ellipsoids(e.centre[keep], e.axes[keep], e.rot[keep], e.density[keep])
    vol = ph.voxelize_ellipsoids(sub, (n, n, n), (s, s, s)).numpy()
    m0, m1, m2 = _moments(vol, (s, s, s))
    V = 4.0 / 3.0 * np.pi * np.prod(sub.axes, axis=1)
    e0 = np.sum(sub.density * V)
    e1 = np.sum((sub.density * V)[:, None] * sub.centre, axis=0)
    e2 = sum(r * (v / 5 * R @ np.diag(a ** 2) @ R.T + v * np.outer(c, c))
             for r, v, R, a, c in zip(sub.density, V, sub.rot, sub.axes, sub.centre))
    w = np.abs(sub.density) * V  # scales of the signed sums
    assert abs(m0 - e0) < 5e-3 * np.sum(w)
    assert np.abs(m1 - e1).max() < 5e-3 * np.sum(w * np.linalg.norm(sub.centre, axis=1))
    scale2 = np.sum(w * (np.sum(sub.axes ** 2, axis=1) / 5 + np.sum(sub.centre ** 2, axis=1)))
    assert np.abs(m2 - e2).max() < 1.5e-3 * scale2


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ellipse_voxeliser_mass_and_moments(seed):
    n, s = 256, 0.25
    half = n * s / 2
    e = ph.random_ellipses(10, half, seed)
    c_, s_ = np.cos(e.angle), np.sin(e.angle)
    R = np.stack([np.stack([c_, -s_], -1), np.stack([s_, c_], -1)], -2)  # columns: the ellipse's axes
    ext = np.sqrt(np.einsum("nik,nk->ni", R ** 2, e.axes ** 2))
    keep = np.all(np.abs(e.centre) + ext <= half, axis=1)
    assert keep.sum() >= 4
    sub = ph.Ellipses(e.centre[keep], e.axes[keep], e.angle[keep], e.density[keep])
    img = ph.voxelize_ellipses(sub, (n, n), (s, s)).numpy()
    m0, m1, m2 = _moments(img, (s, s))
    V = np.pi * np.prod(sub.axes, axis=1)
    e0 = np.sum(sub.density * V)
    e1 = np.sum((sub.density * V)[:, None] * sub.centre, axis=0)
    e2 = sum(r * (v / 4 * Ri @ np.diag(a ** 2) @ Ri.T + v * np.outer(c, c))
             for r, v, Ri, a, c in zip(sub.density, V, R[keep], sub.axes, sub.centre))
    w = np.abs(sub.density) * V
    assert abs(m0 - e0) < 5e-3 * np.sum(w)
    assert np.abs(m1 - e1).max() < 5e-3 * np.sum(w * np.linalg.norm(sub.centre, axis=1))
    scale2 = np.sum(w * (np.sum(sub.axes ** 2, axis=1) / 4 + np.sum(sub.centre ** 2, axis=1)))
    assert np.abs(m2 - e2).max() < 1.5e-3 * scale2
