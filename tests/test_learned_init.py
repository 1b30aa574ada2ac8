"""Host-side pieces of the learned-initialiser study: the field-of-view mask
and the PSNR, checked against projections through the oracle's projection
matrices (an independent construction of the same geometry)."""
import math

import numpy as np
import torch

import oracle
from paper_1904_13342_gb300 import learned_init as LI


def project(P, X):
    """detector (k, l) of the world points X [n, 3] in every view: [V, n, 2]"""
    h = np.concatenate([X, np.ones((len(X), 1))], axis=1)
    q = np.einsum("vij,nj->vni", P, h)
    return q[..., :2] / q[..., 2:3]


def test_fov_mask_is_the_set_every_view_sees():
    setup = LI.SparseViewSetup(n=32, spacing=4.0, views=360, detector=(50, 64), detector_spacing=4.0)
    mask = LI.fov_mask(setup, "cpu").numpy()
    n, s = setup.n, setup.spacing
    c = (np.arange(n) - (n - 1) / 2) * s
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    X = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    P = oracle.circular_pmats(oracle.uniform_angles(setup.views, 2 * math.pi), setup.sid, setup.sdd,
                              setup.detector, (setup.detector_spacing,) * 2)
    kl = project(P, X)
    nv, nu = setup.detector
    # detector edges in pixel-index units are -0.5 and n - 0.5
    seen = ((kl[..., 0] >= -0.5) & (kl[..., 0] <= nu - 0.5) & (kl[..., 1] >= -0.5) & (kl[..., 1] <= nv - 0.5)).all(0)
    seen = seen.reshape(mask.shape)
    assert mask.any() and not mask.all()
    # inside the mask every view sees the voxel
    assert seen[mask].all()
    # and the mask misses only voxels within a whisker of its boundary (the
    # views are discrete, so a few voxels just outside are still seen)
    assert (seen & ~mask).sum() <= 0.01 * mask.sum()


def test_psnr_definition():
    t = torch.zeros(8, 8, 8, dtype=torch.float64)
    t[2:6, 2:6, 2:6] = 2.0
    m = torch.ones_like(t, dtype=torch.bool)
    x = t + 0.1
    # range 2, MSE 0.01 -> 10 log10(4 / 0.01)
    assert abs(LI.psnr(x, t, m) - 10 * math.log10(400.0)) < 1e-9
    m2 = torch.zeros_like(m)
    m2[3:5, 3:5, 3:5] = True
    m2[0, 0, 0] = True
    assert abs(LI.psnr(x, t, m2) - 10 * math.log10(400.0)) < 1e-9
