"""Partitions of the cone-beam path over independent workers (one process
per GPU), none of which needs a data exchange:

* forward projection by view subsets: every view's rays depend on the
  volume and that view's projection matrix only, so a worker holding the
  whole volume projects its share of the views;
* back-projection and FDK by z-slabs: a voxel's value depends on the
  (filtered) sinogram and its own position only, so a worker holding the
  whole sinogram reconstructs its slab.  The slab's geometry is the full
  geometry with the projection matrices shifted to the slab's centre,
  P' = P T(dz) (column 3 += dz column 2), and the full angle list (the
  short-scan weights depend on the view angles).

Each shard is an ordinary geometry, so a worker runs the ordinary calls on
it; concatenating the shards' outputs (views, or z-slabs) gives the
unsharded result.  The matrices come from the library
(pyro_cone_projection_matrices), so a shard uses exactly the matrices the
unsharded call would.
"""
from __future__ import annotations

import ctypes
from dataclasses import replace
from typing import Tuple

import numpy as np

from .geometry import ConeGeometry3D


def split(n: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous balanced share [begin, end) of n items for `rank` of `world`."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    q, r = divmod(n, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def projection_matrices(g: ConeGeometry3D) -> np.ndarray:
    """[V, 3, 4] normalised projection matrices the library uses for g (host)."""
    from . import binding as B

    out = np.empty((g.number_of_projections, 3, 4), dtype=np.float64)
    cg = g.to_c()
    B._check(B.lib().pyro_cone_projection_matrices(ctypes.byref(cg), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def view_shard(g: ConeGeometry3D, world: int, rank: int) -> Tuple[ConeGeometry3D, Tuple[int, int]]:
    """Geometry of views [v0, v1) of g, for the forward projection."""
    v0, v1 = split(g.number_of_projections, world, rank)
    P = projection_matrices(g)[v0:v1]
    ang = g.view_angles()[v0:v1]
    # a shard's range is its share of the scan, so that uniform-angle users
    # of range see consistent numbers; the matrices and angles are explicit
    rng = g.angular_range * (v1 - v0) / g.number_of_projections
    return replace(g, number_of_projections=v1 - v0, angular_range=rng, projection_matrices=P.copy(),
                   angles=ang.copy(), _keep=[]), (v0, v1)


def z_slab(g: ConeGeometry3D, world: int, rank: int) -> Tuple[ConeGeometry3D, Tuple[int, int]]:
    """Geometry of volume slices [z0, z1) of g, for back-projection and FDK
    (all views, the full angle list, matrices shifted to the slab)."""
    nz, ny, nx = g.volume_shape
    z0, z1 = split(nz, world, rank)
    sz = g.volume_spacing[0]
    # slab voxel iz' sits at world z = (z0 + iz' - (nz - 1) / 2) sz; its slab-centred
    # coordinate is (iz' - (nz' - 1) / 2) sz, so the slab's origin is at dz
    dz = (z0 + 0.5 * (z1 - z0 - 1) - 0.5 * (nz - 1)) * sz
    P = projection_matrices(g).copy()
    P[:, :, 3] += P[:, :, 2] * dz
    return replace(g, volume_shape=(z1 - z0, ny, nx), projection_matrices=P, angles=g.view_angles().copy(),
                   _keep=[]), (z0, z1)
