"""Shards through the library on one GPU: the forward projection of view
subsets, and the back-projection and FDK of z-slabs, against the matching
parts of the unsharded calls (the full-size cone workload's geometry)."""
import numpy as np
import pytest
import torch

from paper_1904_13342_gb300 import binding as B
from paper_1904_13342_gb300 import phantoms as ph
from paper_1904_13342_gb300 import shard
from paper_1904_13342_gb300.geometry import ConeGeometry3D, short_scan_range

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def rel(a, b):
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


@pytest.mark.parametrize("world", [2, 3])
def test_view_and_slab_shards_reassemble(world):
    g = ConeGeometry3D((96, 128, 112), (0.5, 0.5, 0.5), (240, 310), (0.616, 0.616), 62,
                       short_scan_range(310 * 0.616, 1200.0), 750.0, 1200.0)
    e = ph.random_ellipsoids(8, 28.0, seed=3)
    vol = ph.voxelize_ellipsoids(e, g.volume_shape, g.volume_spacing, device=DEV, dtype=torch.float32)
    full = B.pyro_fp_cone3d_ws(vol, g)
    parts = [B.pyro_fp_cone3d_ws(vol, shard.view_shard(g, world, r)[0]) for r in range(world)]
    assert rel(torch.cat(parts), full) < 1e-6
    bp = B.pyro_bp_cone3d(full, g, weight=B.W_INV_L2, scale=0.01)
    fdk = B.pyro_fdk(full, g)
    bps, fdks = [], []
    for r in range(world):
        gz, _ = shard.z_slab(g, world, r)
        bps.append(B.pyro_bp_cone3d(full, gz, weight=B.W_INV_L2, scale=0.01))
        fdks.append(B.pyro_fdk(full, gz))
    assert rel(torch.cat(bps), bp) < 1e-5
    assert rel(torch.cat(fdks), fdk) < 1e-5
