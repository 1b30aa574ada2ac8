"""GPU parity: every C-ABI call against the FP64 oracle on the same inputs.

Inputs are seeded (paper_1904_13342_gb300.phantoms).  The CUDA side gets
FP32 (or FP16/BF16) tensors; the oracle gets the same values as float64.
Gate (element-wise comparison, relative L2): <= 1e-5 for FP32 storage,
<= 2e-3 for FP16 storage against the oracle fed the original FP32 input
(end to end, storage rounding included); BF16 is reported with 1e-2.
Small cases span several thread-block tiles with ragged tails; the full
sizes of the headline workloads are checked on sampled outputs.
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
TOL = {torch.float32: 1e-5, torch.float16: 2e-3, torch.bfloat16: 1e-2}


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.float32).to(dtype).to(DEV)


def host(t):
    return t.double().cpu().numpy()


def f32(a):
    """the FP32 values the device sees, as float64"""
    return np.asarray(a, np.float32).astype(np.float64)


# ----------------------------------------------------------------- cases --
PAR = dict(shape=(53, 70), spacing=(0.9, 1.1), nu=77, su=1.2, views=23, range=math.pi)
FAN = dict(shape=(53, 70), spacing=(0.9, 1.1), nu=77, su=1.6, views=23, range=2 * math.pi, sid=300.0, sdd=520.0)
CONE = dict(shape=(19, 37, 45), spacing=(1.0, 0.9, 1.1), det=(29, 41), dspacing=(1.5, 1.4), views=17,
            range=2 * math.pi, sid=250.0, sdd=420.0)


def par_geom(c, angles=None):
    return ParallelGeometry2D(c["shape"], c["spacing"], c["nu"], c["su"], c["views"], c["range"], angles=angles)


def fan_geom(c, angles=None):
    return FanGeometry2D(c["shape"], c["spacing"], c["nu"], c["su"], c["views"], c["range"], c["sid"], c["sdd"],
                         angles=angles)


def cone_geom(c, P=None):
    return ConeGeometry3D(c["shape"], c["spacing"], c["det"], c["dspacing"], c["views"], c["range"], c["sid"], c["sdd"],
                          projection_matrices=P)


def cone_pmats(c, ang):
    return oracle.circular_pmats(ang, c["sid"], c["sdd"], c["det"], c["dspacing"])


def tilted_pmats(c, ang, tilt=0.12, du=2.3, dv=-1.7):
    """A non-circular trajectory written out here: the circular matrices of
    the oracle, rotated about the x axis by `tilt` and with a shifted
    principal point."""
    P = cone_pmats(c, ang)
    ct, st = math.cos(tilt), math.sin(tilt)
    Rx = np.array([[1, 0, 0, 0], [0, ct, -st, 0], [0, st, ct, 0], [0, 0, 0, 1.0]])
    T = np.array([[1, 0, du], [0, 1, dv], [0, 0, 1.0]])
    return np.einsum("ij,vjk,kl->vil", T, P, Rx)


# ------------------------------------------------------------------ 2D ----
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("geom", ["par", "fan"])
def test_fp_2d(geom, dtype):
    c = PAR if geom == "par" else FAN
    img = ph.voxelize_ellipses(ph.random_ellipses(6, 30.0, seed=1), c["shape"], c["spacing"]).numpy()
    img = np.stack([img, ph.random_volume(c["shape"], 2)])  # batch of 2
    ang = oracle.uniform_angles(c["views"], c["range"])
    if geom == "par":
        got = B.pyro_fp_par2d(to_dev(img, dtype), par_geom(c))
        ref = [oracle.fp_par2d(f32(x), c["spacing"], c["nu"], c["su"], ang) for x in img]
    else:
        got = B.pyro_fp_fan2d(to_dev(img, dtype), fan_geom(c))
        ref = [oracle.fp_fan2d(f32(x), c["spacing"], c["nu"], c["su"], ang, c["sid"], c["sdd"]) for x in img]
    assert got.shape == (2, c["views"], c["nu"]) and got.dtype == dtype
    assert rel(host(got), np.stack(ref)) < TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("geom", ["par", "fan"])
def test_fp_2d_staged(geom, dtype):
    """The staged 2D projector (a transposed copy for the views whose rays run
    closer to x) against the oracle and the plain call; views all round."""
    c = dict(PAR if geom == "par" else FAN, views=37, range=2 * math.pi)
    ang = oracle.uniform_angles(c["views"], c["range"])
    vol = np.stack([ph.voxelize_ellipses(ph.random_ellipses(6, 25.0, seed=60 + k), c["shape"], c["spacing"]).numpy()
                    for k in range(3)])
    if geom == "par":
        g = par_geom(c)
        ref = np.stack([oracle.fp_par2d(f32(v), c["spacing"], c["nu"], c["su"], ang) for v in vol])
        got = B.pyro_fp_par2d_ws(to_dev(vol, dtype), g)
        plain = B.pyro_fp_par2d(to_dev(vol, dtype), g)
    else:
        g = fan_geom(c)
        ref = np.stack([oracle.fp_fan2d(f32(v), c["spacing"], c["nu"], c["su"], ang, c["sid"], c["sdd"]) for v in vol])
        got = B.pyro_fp_fan2d_ws(to_dev(vol, dtype), g)
        plain = B.pyro_fp_fan2d(to_dev(vol, dtype), g)
    assert rel(host(got), ref) < TOL[dtype]
    assert rel(host(got), host(plain)) < TOL[dtype]
    small = torch.empty(16, dtype=torch.uint8, device=DEV)
    with pytest.raises(B.PyroError) as e:
        B.pyro_fp_par2d_ws(to_dev(vol), par_geom(c), workspace=small) if geom == "par" else \
            B.pyro_fp_fan2d_ws(to_dev(vol), fan_geom(c), workspace=small)
    assert e.value.status == 5


@pytest.mark.parametrize("geom", ["par", "fan"])
def test_fp_adjoint_2d(geom):
    c = PAR if geom == "par" else FAN
    y = ph.random_sinogram((2, c["views"], c["nu"]), 3)
    ang = np.random.default_rng(4).uniform(0, 2 * np.pi, c["views"])  # explicit, unordered angles
    if geom == "par":
        got = B.pyro_fpT_par2d(to_dev(y), par_geom(c, angles=ang))
        staged = B.pyro_fpT_par2d_ws(to_dev(y), par_geom(c, angles=ang))
        ref = [oracle.fpT_par2d(f32(s), c["shape"], c["spacing"], c["su"], ang) for s in y]
    else:
        got = B.pyro_fpT_fan2d(to_dev(y), fan_geom(c, angles=ang))
        staged = B.pyro_fpT_fan2d_ws(to_dev(y), fan_geom(c, angles=ang))
        ref = [oracle.fpT_fan2d(f32(s), c["shape"], c["spacing"], c["su"], ang, c["sid"], c["sdd"]) for s in y]
    assert rel(host(got), np.stack(ref)) < 1e-5
    # the transposed accumulator: views of both kinds (the angles cover the circle)
    assert rel(host(staged), np.stack(ref)) < 1e-5
    assert rel(host(staged), host(got)) < 1e-5
    small = torch.empty(16, dtype=torch.uint8, device=DEV)
    with pytest.raises(B.PyroError) as e:
        B.pyro_fpT_par2d_ws(to_dev(y), par_geom(c, angles=ang), workspace=small) if geom == "par" else \
            B.pyro_fpT_fan2d_ws(to_dev(y), fan_geom(c, angles=ang), workspace=small)
    assert e.value.status == 5


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("geom,weight", [("par", 0), ("fan", 0), ("fan", 1), ("fan", 2)])
def test_bp_2d(geom, weight, dtype):
    c = PAR if geom == "par" else FAN
    y = ph.random_sinogram((2, c["views"], c["nu"]), 5, smooth=2)
    ang = oracle.uniform_angles(c["views"], c["range"])
    if geom == "par":
        got = B.pyro_bp_par2d(to_dev(y, dtype), par_geom(c), scale=0.37)
        ref = [oracle.bp_par2d(f32(s), c["shape"], c["spacing"], c["su"], ang, scale=0.37) for s in y]
    else:
        got = B.pyro_bp_fan2d(to_dev(y, dtype), fan_geom(c), weight=weight, scale=0.37)
        ref = [oracle.bp_fan2d(f32(s), c["shape"], c["spacing"], c["su"], ang, c["sid"], c["sdd"], weight, 0.37)
               for s in y]
    assert rel(host(got), np.stack(ref)) < TOL[dtype]


@pytest.mark.parametrize("geom", ["par", "fan"])
def test_bp_transpose_2d(geom):
    c = PAR if geom == "par" else FAN
    x = ph.random_volume((2, *c["shape"]), 6)
    ang = oracle.uniform_angles(c["views"], c["range"])
    if geom == "par":
        got = B.pyro_bpT_par2d(to_dev(x), par_geom(c), scale=0.5)
        ref = [oracle.bpT_par2d(f32(v), c["nu"], c["su"], ang, c["spacing"], 0.5) for v in x]
    else:
        got = B.pyro_bpT_fan2d(to_dev(x), fan_geom(c), weight=2, scale=0.5)
        ref = [oracle.bpT_fan2d(f32(v), c["nu"], c["su"], ang, c["spacing"], c["sid"], c["sdd"], 2, 0.5) for v in x]
    assert rel(host(got), np.stack(ref)) < 1e-5


# ------------------------------------------------------------------ 3D ----
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("traj", ["circular", "tilted"])
def test_fp_cone(traj, dtype):
    c = CONE
    ang = oracle.uniform_angles(c["views"], c["range"])
    P = cone_pmats(c, ang) if traj == "circular" else tilted_pmats(c, ang)
    vol = ph.voxelize_ellipsoids(ph.random_ellipsoids(5, 18.0, seed=7), c["shape"], c["spacing"]).numpy()
    vol = np.stack([vol, ph.random_volume(c["shape"], 8)])
    g = cone_geom(c, None if traj == "circular" else P)
    got = B.pyro_fp_cone3d(to_dev(vol, dtype), g)
    ref = np.stack([oracle.fp_cone3d(f32(v), c["spacing"], c["det"], P) for v in vol])
    assert got.shape == (2, c["views"], *c["det"])
    assert rel(host(got), ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("traj", ["circular", "tilted"])
def test_fp_cone_staged(traj, dtype):
    """z-major staged projector: same values as the oracle (and the direct path)."""
    c = CONE
    ang = oracle.uniform_angles(c["views"], c["range"])
    P = cone_pmats(c, ang) if traj == "circular" else tilted_pmats(c, ang)
    vol = ph.voxelize_ellipsoids(ph.random_ellipsoids(5, 18.0, seed=27), c["shape"], c["spacing"]).numpy()
    vol = np.stack([vol, ph.random_volume(c["shape"], 28), vol[::-1].copy()])
    g = cone_geom(c, None if traj == "circular" else P)
    got = B.pyro_fp_cone3d_ws(to_dev(vol, dtype), g)
    ref = np.stack([oracle.fp_cone3d(f32(v), c["spacing"], c["det"], P) for v in vol])
    assert got.shape == (3, c["views"], *c["det"])
    assert rel(host(got), ref) < TOL[dtype]
    direct = B.pyro_fp_cone3d(to_dev(vol, dtype), g)
    assert rel(host(got), host(direct)) < TOL[dtype]


# Circular cases that take the column-shared staged kernel (rows of a detector
# column share (x, y); 31 row steps stay below 29.5 voxels in z): one to four
# 32-row windows per warp with ragged tails, and a row step of 0.94 voxel that
# puts the last taps at the end of a window's 32-voxel run.  CONE itself
# (a row step just above one voxel) and every tilted trajectory take the
# general z-major kernel.
# "near_limit": a row step of 0.949 voxel, 31 steps = 29.43 voxels, just
# inside the kernel's 29.5-voxel bound.  Row steps below about 0.76 voxel
# take the two-rays-per-lane kernels: "three_windows" and "four_windows"
# (windows of 64 rows) and "pair_rows_50" (a row step of 0.598 voxel:
# windows of 50 rows, so lanes 18..31 carry one ray).
COLUMN_CASES = {
    "one_window": dict(CONE, det=(20, 41), dspacing=(1.2, 1.4)),
    "three_windows": dict(CONE, shape=(23, 37, 45), det=(70, 41), dspacing=(0.45, 1.4)),
    "four_windows": dict(CONE, shape=(23, 37, 45), det=(150, 43), dspacing=(0.2, 1.3)),
    "wide_rows": dict(CONE, det=(64, 41), dspacing=(1.4, 1.4)),
    "near_limit": dict(CONE, det=(64, 41), dspacing=(1.412, 1.4)),
    "pair_rows_50": dict(CONE, det=(110, 41), dspacing=(0.89, 1.4)),
}


@pytest.mark.parametrize("case", sorted(COLUMN_CASES))
def test_fp_cone_staged_column_kernel(case):
    c = COLUMN_CASES[case]
    ang = oracle.uniform_angles(c["views"], c["range"])
    P = cone_pmats(c, ang)
    vol = ph.voxelize_ellipsoids(ph.random_ellipsoids(5, 18.0, seed=31), c["shape"], c["spacing"]).numpy()
    vol = np.stack([vol, ph.random_volume(c["shape"], 32)])
    g = cone_geom(c)
    got = B.pyro_fp_cone3d_ws(to_dev(vol), g)
    ref = np.stack([oracle.fp_cone3d(f32(v), c["spacing"], c["det"], P) for v in vol])
    assert rel(host(got), ref) < 1e-5
    # every ray, including the first and last rows and columns
    assert np.max(np.abs(host(got) - ref)) < 1e-4 * np.max(np.abs(ref))
    for dtype in (torch.float16, torch.bfloat16):
        assert rel(host(B.pyro_fp_cone3d_ws(to_dev(vol, dtype), g)), ref) < TOL[dtype]


@pytest.mark.parametrize("case", sorted(COLUMN_CASES) + ["general", "tilted"])
def test_fp_adjoint_cone_staged(case):
    """Exact adjoint through the gathered (circular) or per-sample scatter
    (tilted) path: the oracle's A^T, the scatter, and <A x, y> = <x, A^T y>
    against the staged FP."""
    c = COLUMN_CASES.get(case, CONE)
    ang = oracle.uniform_angles(c["views"], c["range"])
    P = tilted_pmats(c, ang) if case == "tilted" else cone_pmats(c, ang)
    g = cone_geom(c, P if case == "tilted" else None)
    y = ph.random_sinogram((2, c["views"], *c["det"]), 41)
    got = B.pyro_fpT_cone3d_ws(to_dev(y), g)
    ref = np.stack([oracle.fpT_cone3d(f32(s), c["shape"], c["spacing"], P) for s in y])
    assert rel(host(got), ref) < 1e-5
    assert rel(host(got), host(B.pyro_fpT_cone3d(to_dev(y), g))) < 1e-5
    x = ph.random_volume(c["shape"], 42)
    ax = host(B.pyro_fp_cone3d_ws(to_dev(x), g))
    lhs = float(np.sum(ax * f32(y[0])))
    rhs = float(np.sum(f32(x) * host(got[0])))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("case", ["one_window", "four_windows", "near_limit"])
def test_fp_adjoint_cone_gathered_is_deterministic(case):
    """The gathered adjoint sums every voxel in a fixed order: two calls
    (and a call into a reused workspace) give the same bits, over several
    view chunks (250 views: two launches, the second adding)."""
    c = dict(COLUMN_CASES[case], views=250)
    g = cone_geom(c)
    y = to_dev(ph.random_sinogram((1, c["views"], *c["det"]), 43))
    ws = torch.empty(B.fpT_cone3d_workspace_bytes(g), dtype=torch.uint8, device=DEV)
    a = B.pyro_fpT_cone3d_ws(y, g, workspace=ws).clone()
    b = B.pyro_fpT_cone3d_ws(y, g, workspace=ws)
    c2 = B.pyro_fpT_cone3d_ws(y, g)
    assert torch.equal(a, b) and torch.equal(a, c2)
    # and the scatter (atomics, any order) agrees to rounding
    assert rel(host(a), host(B.pyro_fpT_cone3d(y, g))) < 1e-5


def test_fp_adjoint_cone_staged_large_footprint():
    """A 512 x 512 footprint (100 slices, 1 mm detector columns): the staged
    adjoint against the oracle, and against the per-sample scatter on the
    GPU (same FP32 coordinates: agreement to summation order)."""
    shape, spacing = (100, 512, 512), (0.5, 0.5, 0.5)
    det, dsp, views = (60, 420), (0.5, 1.0), 6
    g = ConeGeometry3D(shape, spacing, det, dsp, views, 2 * math.pi, 750.0, 1200.0)
    P = oracle.circular_pmats(oracle.uniform_angles(views, 2 * math.pi), 750.0, 1200.0, det, dsp)
    # a smooth sinogram (white noise would bring in the FP32 coordinate
    # rounding that the noise gate allows for)
    v, l, k = np.meshgrid(np.arange(views), np.arange(det[0]), np.arange(det[1]), indexing="ij")
    y = 1.0 + 0.5 * np.sin(2 * np.pi * k / det[1] + v) * np.cos(2 * np.pi * l / det[0])
    got = host(B.pyro_fpT_cone3d_ws(to_dev(y), g))
    ref = oracle.fpT_cone3d(f32(y), shape, spacing, P)
    assert rel(got, ref) < 1e-5
    assert rel(got, host(B.pyro_fpT_cone3d(to_dev(y), g))) < 1e-6
    # noise data, the input that shows sample-position rounding (absolute FP32
    # coordinates near index 500 gave 7e-6 here; anchored ones 3e-7)
    noise = ph.random_sinogram((views, *det), 43)
    assert rel(host(B.pyro_fpT_cone3d_ws(to_dev(noise), g)),
               oracle.fpT_cone3d(f32(noise), shape, spacing, P)) < 1e-5


@pytest.mark.parametrize("storage", [torch.float16, torch.bfloat16])
def test_fp_cone_staged_half_storage_copy(storage):
    """An FP32 volume projected from an FP16 / BF16 workspace copy into an
    FP32 sinogram: against the oracle fed the FP32 volume (end to end, the
    storage rounding included), on a geometry the column kernels serve (a
    row step of 0.7 voxel)."""
    c = dict(CONE, det=(40, 41), dspacing=(1.0, 1.4))
    ang = oracle.uniform_angles(c["views"], c["range"])
    P = cone_pmats(c, ang)
    vol = ph.voxelize_ellipsoids(ph.random_ellipsoids(5, 18.0, seed=57), c["shape"], c["spacing"]).numpy()
    got = B.pyro_fp_cone3d_ws_storage(to_dev(vol), cone_geom(c), storage)
    assert got.dtype == torch.float32
    ref = oracle.fp_cone3d(f32(vol), c["spacing"], c["det"], P)
    assert rel(host(got), ref) < TOL[storage]
    other = torch.bfloat16 if storage == torch.float16 else torch.float16
    with pytest.raises(B.PyroError):  # a storage type of its own needs an FP32 volume
        B.pyro_fp_cone3d_ws_storage(to_dev(vol, other), cone_geom(c), storage)


def test_fp_cone_staged_workspace_checks():
    c = CONE
    g = cone_geom(c)
    vol = to_dev(ph.random_volume(c["shape"], 29))
    small = torch.empty(vol.numel() * 4 - 16, dtype=torch.uint8, device=DEV)
    with pytest.raises(B.PyroError) as e:
        B.pyro_fp_cone3d_ws(vol, g, workspace=small)
    assert e.value.status == 5
    sino = B.pyro_fp_cone3d(vol, g)
    small_t = torch.empty(B.fpT_cone3d_workspace_bytes(g) - 4, dtype=torch.uint8, device=DEV)
    with pytest.raises(B.PyroError) as e:
        B.pyro_fpT_cone3d_ws(sino, g, workspace=small_t)
    assert e.value.status == 5
    with pytest.raises(B.PyroError) as e:  # the adjoint is FP32 only
        B.pyro_fpT_cone3d_ws(sino.half(), g)
    assert e.value.status == 4


@pytest.mark.parametrize("traj", ["circular", "tilted"])
def test_fp_adjoint_cone(traj):
    c = CONE
    ang = oracle.uniform_angles(c["views"], c["range"])
    P = cone_pmats(c, ang) if traj == "circular" else tilted_pmats(c, ang)
    y = ph.random_sinogram((2, c["views"], *c["det"]), 9)
    got = B.pyro_fpT_cone3d(to_dev(y), cone_geom(c, None if traj == "circular" else P))
    ref = np.stack([oracle.fpT_cone3d(f32(s), c["shape"], c["spacing"], P) for s in y])
    assert rel(host(got), ref) < 1e-5


@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("traj,weight", [("circular", 0), ("circular", 2), ("tilted", 1), ("tilted", 2)])
def test_bp_cone(traj, weight, dtype):
    c = CONE
    ang = oracle.uniform_angles(c["views"], c["range"])
    P = cone_pmats(c, ang) if traj == "circular" else tilted_pmats(c, ang)
    y = ph.random_sinogram((2, c["views"], *c["det"]), 10, smooth=2)
    got = B.pyro_bp_cone3d(to_dev(y, dtype), cone_geom(c, None if traj == "circular" else P), weight=weight,
                           scale=0.25)
    ref = np.stack([oracle.bp_cone3d(f32(s), c["shape"], c["spacing"], P, c["sid"], weight, 0.25) for s in y])
    assert rel(host(got), ref) < TOL[dtype]


def test_bp_transpose_cone():
    c = CONE
    ang = oracle.uniform_angles(c["views"], c["range"])
    P = cone_pmats(c, ang)
    x = ph.random_volume((2, *c["shape"]), 11)
    got = B.pyro_bpT_cone3d(to_dev(x), cone_geom(c), weight=2, scale=0.5)
    ref = np.stack([oracle.bpT_cone3d(f32(v), c["det"], c["spacing"], P, c["sid"], 2, 0.5) for v in x])
    assert rel(host(got), ref) < 1e-5


# ---------------------------------------------------- weights / filters ---
# scan ranges for REDUND_SCAN: super-short (pi + 2 x 2 deg, the detector's half
# fan angle is 3.9 deg), below pi (every ray measured once) and an over-scan
SCAN_RANGES = [math.pi + math.radians(4.0), 0.9 * math.pi, 1.4 * math.pi]


@pytest.mark.parametrize("redund,scan", [(B.REDUND_FULL, None), (B.REDUND_PARKER, None), (B.REDUND_NONE, None)] +
                         [(B.REDUND_SCAN, r) for r in SCAN_RANGES])
def test_weights_cone(redund, scan):
    c = dict(CONE)
    c["range"] = short_scan_range(c["det"][1] * c["dspacing"][1], c["sdd"]) if redund == B.REDUND_PARKER else 2 * math.pi
    if scan:
        c["range"] = scan
    y = ph.random_sinogram((2, c["views"], *c["det"]), 12)
    ang = oracle.uniform_angles(c["views"], c["range"])
    got = B.pyro_weights3d(to_dev(y), cone_geom(c), cosine=True, redund=redund)
    ref = np.stack([oracle.weights(f32(s), c["dspacing"], ang, c["sdd"], True, redund, scan_range=c["range"])
                    for s in y])
    assert rel(host(got), ref) < 1e-6


@pytest.mark.parametrize("scan", SCAN_RANGES)
def test_weights_fan_scan(scan):
    c = dict(FAN, range=scan)
    y = ph.random_sinogram((2, c["views"], c["nu"]), 12)
    ang = oracle.uniform_angles(c["views"], c["range"])
    got = B.pyro_weights2d(to_dev(y), fan_geom(c), cosine=True, redund=B.REDUND_SCAN)
    ref = np.stack([oracle.weights(f32(s), c["su"], ang, c["sdd"], True, B.REDUND_SCAN, scan_range=scan) for s in y])
    assert rel(host(got), ref) < 1e-6
    with pytest.raises(B.PyroError):  # outside (0, 2 pi]
        B.pyro_weights2d(to_dev(y), fan_geom(dict(c, range=7.0)), cosine=True, redund=B.REDUND_SCAN)


@pytest.mark.parametrize("nu", [1, 37, 183, 620, 1240])
@pytest.mark.parametrize("kind", [B.RAMLAK, B.RAMP, B.SHEPP_LOGAN, B.FILTER_CUSTOM])
def test_filter_rows(kind, nu):
    n_rows = 7 if nu > 600 else 13  # odd: the last FFT pair is half empty
    rows = ph.random_sinogram((n_rows, nu), 13)
    pn = B.pyro_filter_pad_length(nu)
    K = np.random.default_rng(14).uniform(0, 1, pn // 2 + 1) if kind == B.FILTER_CUSTOM else None
    got = B.pyro_filter_rows(to_dev(rows), 0.616, kind, custom_K=None if K is None else to_dev(K))
    ref = oracle.filter_rows(f32(rows), 0.616, kind, K=None if K is None else f32(K))
    assert rel(host(got), ref) < 1e-5


def test_filter_rows_in_place_and_half():
    rows = ph.random_sinogram((9, 300), 15, smooth=1)
    t = to_dev(rows)
    ref = oracle.filter_rows(f32(rows), 0.5, B.SHEPP_LOGAN)
    B.pyro_filter_rows(t, 0.5, B.SHEPP_LOGAN, out=t)
    assert rel(host(t), ref) < 1e-5
    h = B.pyro_filter_rows(to_dev(rows, torch.float16), 0.5, B.SHEPP_LOGAN)
    assert rel(host(h), ref) < 2e-3


def test_filter_grad_K():
    nu = 183
    p = ph.random_sinogram((11, nu), 16)
    g = ph.random_sinogram((11, nu), 17)
    got = B.pyro_filter_grad_K(to_dev(p), to_dev(g))
    ref = oracle.filter_grad_K(f32(p), f32(g))
    assert rel(host(got), ref) < 1e-5


# ------------------------------------------------------------- FBP/FDK ----


@pytest.mark.parametrize("data", ["phantom", "noise"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16])
@pytest.mark.parametrize("redund,kind", [(B.REDUND_PARKER, B.SHEPP_LOGAN), (B.REDUND_FULL, B.RAMLAK),
                                         (B.REDUND_SCAN, B.SHEPP_LOGAN)])
def test_fdk(redund, kind, dtype, data):
    c = dict(CONE)
    c["range"] = short_scan_range(c["det"][1] * c["dspacing"][1], c["sdd"]) if redund == B.REDUND_PARKER else 2 * math.pi
    if redund == B.REDUND_SCAN:
        c["range"] = SCAN_RANGES[0]
    ang = oracle.uniform_angles(c["views"], c["range"])
    P = cone_pmats(c, ang)
    if data == "phantom":
        y = np.stack([an.cone_sinogram(ph.random_ellipsoids(5, 18.0, seed=s), ang, c["det"], c["dspacing"], c["sid"],
                                       c["sdd"]) for s in (30, 31)])
    else:
        y = ph.random_sinogram((2, c["views"], *c["det"]), 18, smooth=3)
    got = B.pyro_fdk(to_dev(y, dtype), cone_geom(c), kind=kind, redund=redund)
    ref = np.stack([oracle.fdk(f32(s), c["shape"], c["spacing"], c["dspacing"], ang, P, c["sid"], c["sdd"],
                               c["range"] / c["views"], kind, redund, scan_range=c["range"]) for s in y])
    assert rel(host(got), ref) < TOL[dtype]


@pytest.mark.parametrize("data", ["phantom", "noise"])
@pytest.mark.parametrize("geom", ["par", "fan_full", "fan_parker", "fan_scan"])
def test_fbp_2d(geom, data):
    c = dict(PAR if geom == "par" else FAN)
    if geom == "fan_parker":
        c["range"] = short_scan_range(c["nu"] * c["su"], c["sdd"])
    if geom == "fan_scan":  # super-short: pi + 2 x 6 deg, the detector's half fan angle is 6.8 deg
        c["range"] = math.pi + math.radians(12.0)
    ang = oracle.uniform_angles(c["views"], c["range"])
    if data == "phantom":
        es = [ph.random_ellipses(6, 30.0, seed=s) for s in (40, 41)]
        if geom == "par":
            y = np.stack([an.parallel_sinogram(e, ang, c["nu"], c["su"]) for e in es])
        else:
            y = np.stack([an.fan_sinogram(e, ang, c["nu"], c["su"], c["sid"], c["sdd"]) for e in es])
    else:
        y = ph.random_sinogram((2, c["views"], c["nu"]), 19, smooth=3)
    if geom == "par":
        got = B.pyro_fbp_par2d(to_dev(y), par_geom(c), kind=B.RAMLAK)
        ref = [oracle.fbp_par2d(f32(s), c["shape"], c["spacing"], c["su"], ang, B.RAMLAK) for s in y]
    else:
        red = {"fan_full": B.REDUND_FULL, "fan_parker": B.REDUND_PARKER, "fan_scan": B.REDUND_SCAN}[geom]
        got = B.pyro_fbp_fan2d(to_dev(y), fan_geom(c), kind=B.SHEPP_LOGAN, redund=red)
        ref = [oracle.fbp_fan2d(f32(s), c["shape"], c["spacing"], c["su"], ang, c["sid"], c["sdd"],
                                c["range"] / c["views"], B.SHEPP_LOGAN, red, scan_range=c["range"]) for s in y]
    assert rel(host(got), np.stack(ref)) < 1e-5


# ------------------------------------------------------- edge cases -------
def test_empty_batch_and_single_pixel():
    g = ParallelGeometry2D((1, 1), (1.0, 1.0), 1, 1.0, 1)
    x = torch.ones((0, 1, 1), device=DEV)
    assert B.pyro_fp_par2d(x, g).shape == (0, 1, 1)
    one = torch.full((1, 1), 2.0, device=DEV)
    got = host(B.pyro_fp_par2d(one, g))
    ref = oracle.fp_par2d(np.full((1, 1), 2.0), (1.0, 1.0), 1, 1.0, np.zeros(1))
    assert rel(got, ref) < 1e-6


def test_many_views_are_chunked():
    """More views than one kernel-parameter pack holds (cone BP 600, FP 400,
    2D 1024): chunking must not change the result."""
    c = dict(CONE, shape=(9, 12, 11), det=(10, 14), views=1100)
    ang = oracle.uniform_angles(c["views"], c["range"])
    P = cone_pmats(c, ang)
    vol = ph.random_volume(c["shape"], 20)
    y = ph.random_sinogram((c["views"], *c["det"]), 21)
    g = cone_geom(c)
    assert rel(host(B.pyro_fp_cone3d(to_dev(vol), g)), oracle.fp_cone3d(f32(vol), c["spacing"], c["det"], P)) < 1e-5
    assert rel(host(B.pyro_bp_cone3d(to_dev(y), g, weight=2)),
               oracle.bp_cone3d(f32(y), c["shape"], c["spacing"], P, c["sid"], 2, 1.0)) < 1e-5
    # the staged projector and its adjoint through the column-shared kernels
    c3 = dict(c, dspacing=(0.6, 1.4))
    P3 = cone_pmats(c3, ang)
    g3 = cone_geom(c3)
    assert rel(host(B.pyro_fp_cone3d_ws(to_dev(vol), g3)),
               oracle.fp_cone3d(f32(vol), c3["spacing"], c3["det"], P3)) < 1e-5
    assert rel(host(B.pyro_fpT_cone3d_ws(to_dev(y), g3)),
               oracle.fpT_cone3d(f32(y), c3["shape"], c3["spacing"], P3)) < 1e-5
    c2 = dict(PAR, views=2100)
    ang2 = oracle.uniform_angles(c2["views"], c2["range"])
    y2 = ph.random_sinogram((c2["views"], c2["nu"]), 22)
    assert rel(host(B.pyro_bp_par2d(to_dev(y2), par_geom(c2))),
               oracle.bp_par2d(f32(y2), c2["shape"], c2["spacing"], c2["su"], ang2)) < 1e-5


@pytest.mark.parametrize("weight", [0, 1, 2])
def test_bp_cone_tma_staged(weight):
    """A detector whose width is a multiple of 4 and an FP32 sinogram: the cone
    BP of a circular trajectory stages its detector boxes with tensor copies.
    Against the oracle, with more views than one parameter pack (chunks) and
    voxels whose rays leave the detector (zero-filled boxes)."""
    c = dict(CONE, det=(30, 44), dspacing=(1.2, 1.0), views=700)
    ang = oracle.uniform_angles(c["views"], c["range"])
    P = cone_pmats(c, ang)
    y = ph.random_sinogram((2, c["views"], *c["det"]), 51, smooth=2)
    got = B.pyro_bp_cone3d(to_dev(y), cone_geom(c), weight=weight, scale=0.3)
    ref = np.stack([oracle.bp_cone3d(f32(s), c["shape"], c["spacing"], P, c["sid"], weight, 0.3) for s in y])
    assert rel(host(got), ref) < 1e-5
    vol = ph.voxelize_ellipsoids(ph.random_ellipsoids(5, 18.0, seed=52), c["shape"], c["spacing"]).numpy()
    p = f32(oracle.fp_cone3d(vol, c["spacing"], c["det"], P))
    fdk = B.pyro_fdk(to_dev(p), cone_geom(c), kind=B.SHEPP_LOGAN, redund=B.REDUND_FULL)
    ref = oracle.fdk(p, c["shape"], c["spacing"], c["dspacing"], ang, P, c["sid"], c["sdd"], c["range"] / c["views"],
                     kind=oracle.SHEPP_LOGAN, redund=oracle.REDUND_FULL)
    assert rel(host(fdk), ref) < 1e-5
    B.pyro_sync_status()


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_bp_cone_tma_staged_half(dtype):
    """A 16-bit sinogram whose rows are a multiple of 16 bytes (48 columns)
    is staged by tensor copies of 16-bit boxes; the volume is written in the
    same type.  Against the oracle fed the FP32 input (end to end)."""
    c = dict(CONE, det=(30, 48), dspacing=(1.2, 1.0), views=90)
    ang = oracle.uniform_angles(c["views"], c["range"])
    P = cone_pmats(c, ang)
    y = ph.random_sinogram((2, c["views"], *c["det"]), 53, smooth=2)
    got = B.pyro_bp_cone3d(to_dev(y, dtype), cone_geom(c), weight=2, scale=0.3)
    assert got.dtype == dtype
    ref = np.stack([oracle.bp_cone3d(f32(s), c["shape"], c["spacing"], P, c["sid"], 2, 0.3) for s in y])
    assert rel(host(got), ref) < TOL[dtype]
    B.pyro_sync_status()


def test_bp_cone_tma_staged_fine_rows():
    """Fine detector rows (0.25 mm, about 7 rows per 1 mm voxel): a 16-deep
    tile needs 129-row boxes (a 128 KB ring), an 8-deep one 68-row boxes
    (69 KB); no plan fits four blocks per SM, so the host takes the smaller,
    the 8-deep tile with one view per stage."""
    c = dict(CONE, det=(130, 44), dspacing=(0.25, 1.0), views=60)
    ang = oracle.uniform_angles(c["views"], c["range"])
    P = cone_pmats(c, ang)
    y = ph.random_sinogram((1, c["views"], *c["det"]), 54, smooth=2)
    got = B.pyro_bp_cone3d(to_dev(y), cone_geom(c), weight=2, scale=0.3)
    ref = oracle.bp_cone3d(f32(y[0]), c["shape"], c["spacing"], P, c["sid"], 2, 0.3)
    assert rel(host(got[0]), ref) < 1e-5
    B.pyro_sync_status()


def test_sync_status_reports_a_clean_stream():
    B.pyro_fp_cone3d(to_dev(ph.random_volume(CONE["shape"], 50)), cone_geom(CONE))
    B.pyro_sync_status()  # raises PyroError if the stream faulted


def test_a_wait_that_runs_out_is_reported_and_the_context_survives():
    """A bounded device-side wait on a barrier nothing completes gives up
    after 20 ms and sets the status word: pyro_sync_status reports
    PYRO_ETIMEOUT once, clears it, and the context keeps working."""
    B.pyro_selftest_wait_timeout(20)
    with pytest.raises(B.PyroError) as e:
        B.pyro_sync_status()
    assert e.value.status == 3
    B.pyro_sync_status()  # cleared
    c = CONE
    vol = ph.random_volume(c["shape"], 53)
    P = cone_pmats(c, oracle.uniform_angles(c["views"], c["range"]))
    got = B.pyro_fp_cone3d(to_dev(vol), cone_geom(c))
    assert rel(host(got), oracle.fp_cone3d(f32(vol), c["spacing"], c["det"], P)) < 1e-5


def test_invalid_call_enqueues_nothing():
    g = ParallelGeometry2D((8, 8), (1.0, 1.0), 9, 1.0, 4)
    with pytest.raises(ValueError):
        B.pyro_fp_par2d(torch.zeros((8, 9), device=DEV), g)  # wrong shape caught in the binding
    bad = ParallelGeometry2D((8, 8), (1.0, -1.0), 9, 1.0, 4)
    with pytest.raises(B.PyroError) as e:
        B.pyro_fp_par2d(torch.zeros((8, 8), device=DEV), bad)
    assert e.value.status == 1
