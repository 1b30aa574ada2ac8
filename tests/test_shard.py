"""Sharding of the cone-beam path over two ranks (gloo, CPU): forward
projection by view subsets and back-projection / FDK by z-slabs, each rank
computing its share with the FP64 oracle on the shard geometry, gathered
over the process group and compared with the unsharded result."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1904_13342_gb300 import shard
from paper_1904_13342_gb300.geometry import ConeGeometry3D, short_scan_range


def geometry():
    nv, nu, sv, su, sdd = 14, 22, 1.6, 1.5, 320.0
    return ConeGeometry3D((13, 16, 18), (1.1, 1.0, 0.9), (nv, nu), (sv, su), 11, short_scan_range(nu * su, sdd),
                          200.0, sdd)


def test_split_covers_every_item_once():
    for n in (0, 1, 7, 10, 33):
        for world in (1, 2, 3, 8):
            parts = [shard.split(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            assert max(e - b for b, e in parts) - min(e - b for b, e in parts) <= 1
    with pytest.raises(ValueError):
        shard.split(4, 2, 2)


def test_library_matrices_are_the_circular_trajectory():
    g = geometry()
    P = shard.projection_matrices(g)
    ref = oracle.circular_pmats(g.view_angles(), g.sid, g.sdd, g.detector_shape, g.detector_spacing)
    assert np.max(np.abs(P - ref)) < 1e-9 * np.max(np.abs(ref))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = geometry()
        rng = np.random.default_rng(5)
        vol = rng.random(g.volume_shape)
        sino = rng.random(g.sinogram_shape)
        spacing = g.volume_spacing
        gv, (v0, v1) = shard.view_shard(g, world, rank)
        fp = oracle.fp_cone3d(vol, spacing, g.detector_shape, gv.projection_matrices)
        gz, (z0, z1) = shard.z_slab(g, world, rank)
        bp = oracle.bp_cone3d(sino, gz.volume_shape, spacing, gz.projection_matrices, g.sid, 2, 0.7)
        dbeta = g.angular_range / g.number_of_projections
        fdk = oracle.fdk(sino, gz.volume_shape, spacing, g.detector_spacing, gz.angles, gz.projection_matrices,
                         g.sid, g.sdd, dbeta)
        parts = [None] * world
        dist.all_gather_object(parts, {"v": (v0, v1), "z": (z0, z1), "fp": fp, "bp": bp, "fdk": fdk})
        if rank == 0:
            P = shard.projection_matrices(g)
            full_fp = oracle.fp_cone3d(vol, spacing, g.detector_shape, P)
            full_bp = oracle.bp_cone3d(sino, g.volume_shape, spacing, P, g.sid, 2, 0.7)
            full_fdk = oracle.fdk(sino, g.volume_shape, spacing, g.detector_spacing, g.view_angles(), P, g.sid,
                                  g.sdd, dbeta)
            assert [p["v"] for p in parts] == [shard.split(g.number_of_projections, world, r) for r in range(world)]
            fp_cat = np.concatenate([p["fp"] for p in parts])
            bp_cat = np.concatenate([p["bp"] for p in parts])
            fdk_cat = np.concatenate([p["fdk"] for p in parts])
            # each view is the same computation: equal to the bit
            assert np.array_equal(fp_cat, full_fp)
            # slab voxel positions come from the shifted matrices: rounding only
            assert np.max(np.abs(bp_cat - full_bp)) <= 1e-11 * np.max(np.abs(full_bp))
            assert np.max(np.abs(fdk_cat - full_fdk)) <= 1e-11 * np.max(np.abs(full_fdk))
            np.save(os.path.join(out_dir, "ok.npy"), np.array([1]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_fp_bp_fdk_over_gloo_ranks(world, tmp_path):
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    assert (tmp_path / "ok.npy").exists()


def test_geometry_trajectory_helpers():
    """Central-ray vectors (2D) round-trip through the angles; trajectory()
    (3D) is the library's matrices, the circular ones when none are given."""
    from paper_1904_13342_gb300.geometry import FanGeometry2D

    g2 = FanGeometry2D((16, 16), (1.0, 1.0), 24, 1.2, 10, 2 * math.pi, 300.0, 500.0)
    v = g2.central_ray_vectors()
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    g2b = g2.with_central_ray_vectors(3.0 * v[::-1])
    assert g2b.number_of_projections == 10
    assert np.allclose(g2b.central_ray_vectors(), v[::-1])
    g = geometry()
    assert np.array_equal(g.trajectory(), shard.projection_matrices(g))
