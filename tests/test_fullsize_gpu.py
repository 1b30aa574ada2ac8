"""Parity at the full sizes of the headline workloads, in the launch
configuration the benchmark times, on outputs the oracle computes one by one
(sampled rays, sampled voxels) or on whole small problems.

  * 3D cone-beam short-scan FDK: 256^3 volume (0.5 mm) of 12 random
    ellipsoids, 248 views over pi + 2 delta, 620 x 480 detector (0.616 mm),
    SID 750 mm, SDD 1200 mm, Parker weights, Shepp-Logan filter;
  * 2D fan-beam batch: 16 random-ellipse phantoms 512^2 (0.5 mm), 360 views
    over 2 pi, 1024 bins (1.0 mm), SID 750 mm, SDD 1200 mm;
  * 2D parallel beam: 128^2 (1.0 mm), 180 views over pi, 183 bins, whole;
  * the 512^3 iterative workload's FP, BP and exact adjoint;
  * the learned initialiser's batch of 32 FDKs at 128^3.
"""
import math

import numpy as np
import pytest
import torch

import analytic as an
import oracle
from paper_1904_13342_gb300 import binding as B
from paper_1904_13342_gb300 import phantoms as ph
from paper_1904_13342_gb300.geometry import ConeGeometry3D, FanGeometry2D, ParallelGeometry2D, short_scan_range

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def cone_workload():
    n, s = 256, 0.5
    nv, nu, sv, su, sid, sdd = 480, 620, 0.616, 0.616, 750.0, 1200.0
    rng_ = short_scan_range(nu * su, sdd)
    g = ConeGeometry3D((n, n, n), (s, s, s), (nv, nu), (sv, su), 248, rng_, sid, sdd)
    return g


@pytest.fixture(scope="module")
def cone():
    g = cone_workload()
    n = g.volume_shape[0]
    e = ph.random_ellipsoids(12, n * 0.5 / 2, seed=0)
    vol = ph.voxelize_ellipsoids(e, g.volume_shape, g.volume_spacing, device=DEV, dtype=torch.float32)
    ang = g.view_angles()
    P = oracle.circular_pmats(ang, g.sid, g.sdd, g.detector_shape, g.detector_spacing)
    return g, vol, ang, P


@pytest.mark.parametrize("mode", ["direct", "staged"])
def test_cone_fp_full_size_sampled_rays(cone, mode):
    g, vol, ang, P = cone
    sino = B.pyro_fp_cone3d(vol, g) if mode == "direct" else B.pyro_fp_cone3d_ws(vol, g)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    nvw, (nv, nu) = g.number_of_projections, g.detector_shape
    views = rng.integers(0, nvw, 300)
    ks, ls = rng.integers(0, nu, 300), rng.integers(0, nv, 300)
    # include the detector corners and the central pixel
    views = np.r_[views, 0, nvw - 1, 17, 100]
    ks = np.r_[ks, 0, nu - 1, nu // 2, 0]
    ls = np.r_[ls, 0, nv - 1, nv // 2, nv - 1]
    v64 = vol.double().cpu().numpy()
    ref = oracle.fp_cone3d_rays(v64, g.volume_spacing, P, views, ks, ls)
    got = sino[views, ls, ks].double().cpu().numpy()
    assert rel(got, ref) < 1e-5
    assert np.max(np.abs(got - ref)) < 1e-4 * np.max(np.abs(ref))


def test_cone_bp_full_size_sampled_voxels(cone):
    g, _, ang, P = cone
    y = ph.random_sinogram((g.number_of_projections, *g.detector_shape), 2)
    yt = torch.from_numpy(y).float().to(DEV)
    vol = B.pyro_bp_cone3d(yt, g, weight=B.W_INV_L2, scale=0.01)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    n = g.volume_shape[0]
    ii, jj, kk = rng.integers(0, n, 200), rng.integers(0, n, 200), rng.integers(0, n, 200)
    ii, jj, kk = np.r_[ii, 0, n - 1, 0], np.r_[jj, 0, n - 1, n - 1], np.r_[kk, 0, n - 1, n // 2]
    ref = oracle.bp_cone3d_voxels(yt.double().cpu().numpy(), g.volume_shape, g.volume_spacing, P, g.sid, ii, jj, kk,
                                  weight=2, scale=0.01)
    got = vol[kk, jj, ii].double().cpu().numpy()
    assert rel(got, ref) < 1e-5


def _fdk_check(g, ang, P, y, tol):
    yt = torch.from_numpy(y).float().to(DEV)
    rec = B.pyro_fdk(yt, g, kind=B.SHEPP_LOGAN, redund=B.REDUND_PARKER)
    torch.cuda.synchronize()
    n = g.volume_shape[0]
    rng = np.random.default_rng(5)
    kk = np.repeat([n // 2, 37, n - 1], 12)
    ii, jj = rng.integers(0, n, kk.size), rng.integers(0, n, kk.size)
    ref = oracle.fdk_voxels(yt.double().cpu().numpy(), g.volume_shape, g.volume_spacing, g.detector_spacing, ang, P,
                            g.sid, g.sdd, g.angular_range / g.number_of_projections, ii, jj, kk,
                            kind=oracle.SHEPP_LOGAN, redund=oracle.REDUND_PARKER)
    got = rec[kk, jj, ii].double().cpu().numpy()
    assert rel(got, ref) < tol


def test_fdk_full_size_sampled_voxels(cone):
    """FDK of the analytic projections of the workload's ellipsoid phantom."""
    g, _, ang, P = cone
    e = ph.random_ellipsoids(12, g.volume_shape[0] * 0.5 / 2, seed=0)
    y = an.cone_sinogram(e, ang, g.detector_shape, g.detector_spacing, g.sid, g.sdd)
    _fdk_check(g, ang, P, y, 1e-5)


def test_fdk_full_size_noise_input(cone):
    """Back-projected noise is the input that exposes detector-coordinate
    rounding (an absolute FP32 coordinate near pixel 300 carries ~2e-5 pixel,
    which gave ~2.6e-5 relative); the anchored coordinates keep it at ~1e-6."""
    g, _, ang, P = cone
    y = ph.random_sinogram((g.number_of_projections, *g.detector_shape), 4, smooth=4)
    _fdk_check(g, ang, P, y, 1e-5)


@pytest.mark.parametrize("mode", ["direct", "staged"])
def test_cone_fp_full_size_noise_volume(cone, mode):
    """A white-noise volume is the input that shows sample-position rounding:
    absolute FP32 voxel coordinates gave 2.4e-5 on these rays, the anchored
    positions 6e-7..1e-6."""
    g, _, ang, P = cone
    vol = ph.random_volume(g.volume_shape, 7).astype(np.float32)
    v = torch.from_numpy(vol).to(DEV)
    sino = B.pyro_fp_cone3d(v, g) if mode == "direct" else B.pyro_fp_cone3d_ws(v, g)
    rng = np.random.default_rng(1)
    views, ks, ls = rng.integers(0, 248, 300), rng.integers(0, 620, 300), rng.integers(0, 480, 300)
    ref = oracle.fp_cone3d_rays(vol.astype(np.float64), g.volume_spacing, P, views, ks, ls)
    assert rel(sino[views, ls, ks].double().cpu().numpy(), ref) < 1e-5


def test_fan_full_size_noise_fp_and_adjoint():
    """One image of the 16-phantom fan workload (512^2 at 0.5 mm, 360 views,
    1024 bins): FP of a noise image and the exact adjoint of a noise sinogram,
    plain and staged, against the oracle on the whole problem (absolute FP32
    pixel coordinates gave 1.9e-5 on the FP)."""
    n, s = 512, 0.5
    g = FanGeometry2D((n, n), (s, s), 1024, 1.0, 360, 2 * math.pi, 750.0, 1200.0)
    ang = g.view_angles()
    img = ph.random_volume((n, n), 3).astype(np.float32)
    ref = oracle.fp_fan2d(img.astype(np.float64), (s, s), 1024, 1.0, ang, 750.0, 1200.0)
    x = torch.from_numpy(img[None]).to(DEV)
    assert rel(B.pyro_fp_fan2d(x, g)[0].double().cpu().numpy(), ref) < 1e-5
    assert rel(B.pyro_fp_fan2d_ws(x, g)[0].double().cpu().numpy(), ref) < 1e-5
    y = ph.random_sinogram((360, 1024), 5).astype(np.float32)
    ref = oracle.fpT_fan2d(y.astype(np.float64), (n, n), (s, s), 1.0, ang, 750.0, 1200.0)
    yd = torch.from_numpy(y[None]).to(DEV)
    assert rel(B.pyro_fpT_fan2d(yd, g)[0].double().cpu().numpy(), ref) < 1e-5
    assert rel(B.pyro_fpT_fan2d_ws(yd, g)[0].double().cpu().numpy(), ref) < 1e-5


def test_fan_batch_full_size_sampled_views():
    n, s = 512, 0.5
    g = FanGeometry2D((n, n), (s, s), 1024, 1.0, 360, 2 * math.pi, 750.0, 1200.0)
    imgs = torch.stack([ph.voxelize_ellipses(ph.random_ellipses(10, n * s / 2, seed=k), (n, n), (s, s), device=DEV,
                                             dtype=torch.float32) for k in range(16)])
    sino = B.pyro_fp_fan2d(imgs, g)
    torch.cuda.synchronize()
    ang = g.view_angles()
    sel = np.array([0, 45, 179, 359])
    for b in (0, 15):
        ref = oracle.fp_fan2d(imgs[b].double().cpu().numpy(), (s, s), 1024, 1.0, ang[sel], 750.0, 1200.0)
        assert rel(sino[b, sel].double().cpu().numpy(), ref) < 1e-5
    # exact adjoint on the same batch, checked through <Ax, y> = <x, A^T y>
    y = torch.from_numpy(ph.random_sinogram((16, 360, 1024), 6)).float().to(DEV)
    aty = B.pyro_fpT_fan2d(y, g)
    lhs = torch.sum(sino.double() * y.double()).item()
    rhs = torch.sum(imgs.double() * aty.double()).item()
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)


def test_parallel_full_problem():
    n = 128
    g = ParallelGeometry2D((n, n), (1.0, 1.0), 183, 1.0, 180, math.pi)
    img = ph.voxelize_ellipses(ph.random_ellipses(10, 64.0, seed=0), (n, n), (1.0, 1.0)).float()
    ang = g.view_angles()
    sino = B.pyro_fp_par2d(img.to(DEV), g)
    ref = oracle.fp_par2d(img.double().numpy(), (1.0, 1.0), 183, 1.0, ang)
    assert rel(sino.double().cpu().numpy(), ref) < 1e-5
    y = torch.from_numpy(ref).float()
    rec = B.pyro_fbp_par2d(y.to(DEV), g, kind=B.RAMLAK)
    rref = oracle.fbp_par2d(y.double().numpy(), (n, n), (1.0, 1.0), 1.0, ang, oracle.RAMLAK)
    assert rel(rec.double().cpu().numpy(), rref) < 1e-5


def test_tv512_geometry_full_size():
    """The 512^3 iterative workload's operators at full size (0.5 mm, 496
    views over 2 pi, 1240 x 960 detector at 0.308 mm): staged FP on sampled
    rays and BP on sampled voxels against the oracle; the staged exact
    adjoint through <A x, y> = <x, A^T y> on the whole problem."""
    n = 512
    g = ConeGeometry3D((n, n, n), (0.5,) * 3, (960, 1240), (0.308, 0.308), 496, 2 * math.pi, 750.0, 1200.0)
    vol = ph.voxelize_ellipsoids(ph.random_ellipsoids(20, n * 0.5 / 2, seed=0), g.volume_shape, g.volume_spacing,
                                 device=DEV, dtype=torch.float32)
    sino = B.pyro_fp_cone3d_ws(vol, g)
    torch.cuda.synchronize()
    P = oracle.circular_pmats(g.view_angles(), g.sid, g.sdd, g.detector_shape, g.detector_spacing)
    rng = np.random.default_rng(11)
    views, ks, ls = rng.integers(0, 496, 150), rng.integers(0, 1240, 150), rng.integers(0, 960, 150)
    views, ks, ls = np.r_[views, 0, 495], np.r_[ks, 0, 1239], np.r_[ls, 0, 959]
    ref = oracle.fp_cone3d_rays(vol.double().cpu().numpy(), g.volume_spacing, P, views, ks, ls)
    assert rel(sino[views, ls, ks].double().cpu().numpy(), ref) < 1e-5
    y = sino.contiguous()
    bp = B.pyro_bp_cone3d(y, g, weight=B.W_INV_L2, scale=0.01)
    torch.cuda.synchronize()
    ii, jj, kk = rng.integers(0, n, 60), rng.integers(0, n, 60), rng.integers(0, n, 60)
    refv = oracle.bp_cone3d_voxels(y.double().cpu().numpy(), g.volume_shape, g.volume_spacing, P, g.sid, ii, jj, kk,
                                   weight=2, scale=0.01)
    assert rel(bp[kk, jj, ii].double().cpu().numpy(), refv) < 1e-5
    w = torch.from_numpy(ph.random_sinogram((496, 960, 1240), 12)).float().to(DEV)
    atw = B.pyro_fpT_cone3d_ws(w, g)
    lhs = torch.sum(sino.double() * w.double()).item()
    rhs = torch.sum(vol.double() * atw.double()).item()
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)


def test_tv512_adjoint_elementwise_on_a_view_subset():
    """The gathered exact adjoint in the 512^3 iterative workload's geometry
    (0.5 mm voxels, 1240 x 960 detector at 0.308 mm: a row step of 0.27 to
    0.5 voxel, so 12-row windows), on 8 views and a noise sinogram, element
    by element on sampled voxels against the oracle's voxel-wise adjoint;
    sampled voxels include the volume's faces and corners."""
    n = 512
    g = ConeGeometry3D((n, n, n), (0.5,) * 3, (960, 1240), (0.308, 0.308), 8, 2 * math.pi, 750.0, 1200.0)
    P = oracle.circular_pmats(g.view_angles(), g.sid, g.sdd, g.detector_shape, g.detector_spacing)
    y = ph.random_sinogram((8, 960, 1240), 14).astype(np.float32)
    at = B.pyro_fpT_cone3d_ws(torch.from_numpy(y).to(DEV), g)
    torch.cuda.synchronize()
    rng = np.random.default_rng(15)
    ii, jj, kk = rng.integers(0, n, 200), rng.integers(0, n, 200), rng.integers(0, n, 200)
    ii, jj, kk = np.r_[ii, 0, n - 1, 0, n - 1], np.r_[jj, 0, n - 1, n - 1, 0], np.r_[kk, 0, n - 1, 0, n // 2]
    ref = oracle.fpT_cone3d_voxels(y.astype(np.float64), g.volume_shape, g.volume_spacing, P, ii, jj, kk)
    assert rel(at[kk, jj, ii].double().cpu().numpy(), ref) < 1e-5


def test_learned_init_batch_full_size():
    """The learned-initialiser workload's FDK on its batch of 32 128^3
    phantoms (60 views over 2 pi, 256 x 200 at 1 mm): sampled voxels of the
    first and last volume against the oracle."""
    g = ConeGeometry3D((128,) * 3, (1.0,) * 3, (200, 256), (1.0, 1.0), 60, 2 * math.pi, 750.0, 1200.0)
    vols = torch.stack([ph.voxelize_ellipsoids(ph.random_ellipsoids(12, 64.0, seed=s), g.volume_shape,
                                               g.volume_spacing, device=DEV, dtype=torch.float32) for s in range(32)])
    sino = B.pyro_fp_cone3d_ws(vols, g)
    rec = B.pyro_fdk(sino, g, kind=B.SHEPP_LOGAN, redund=B.REDUND_FULL)
    torch.cuda.synchronize()
    P = oracle.circular_pmats(g.view_angles(), g.sid, g.sdd, g.detector_shape, g.detector_spacing)
    rng = np.random.default_rng(13)
    ii, jj, kk = rng.integers(0, 128, 300), rng.integers(0, 128, 300), rng.integers(0, 128, 300)
    for b in (0, 31):
        ref = oracle.fdk_voxels(sino[b].double().cpu().numpy(), g.volume_shape, g.volume_spacing, g.detector_spacing,
                                g.view_angles(), P, g.sid, g.sdd, 2 * math.pi / 60, ii, jj, kk,
                                kind=oracle.SHEPP_LOGAN, redund=oracle.REDUND_FULL)
        assert rel(rec[b][kk, jj, ii].double().cpu().numpy(), ref) < 1e-5
