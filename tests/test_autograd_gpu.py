"""Differentiable layers: GPU gradients against the FP64 oracle's gradient
and against FP64 finite differences of the oracle's loss.

For the quadratic loss L = 1/2 |A x - y|^2 the gradient is A^T (A x - y)
(Section "The Known Operator": the gradient of A is A^T); central
differences in FP64 are exact up to rounding for a quadratic, so they pin
the direction of every gradient independently of the adjoint code.
"""
import math

import numpy as np
import pytest
import torch

import analytic as an
import oracle
from paper_1904_13342_gb300 import autograd as AG
from paper_1904_13342_gb300 import binding as B
from paper_1904_13342_gb300 import phantoms as ph
from paper_1904_13342_gb300.geometry import ConeGeometry3D, FanGeometry2D, ParallelGeometry2D, short_scan_range

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).float().to(DEV)


FAN = dict(shape=(32, 32), spacing=(0.5, 0.5), nu=64, su=1.0, views=60, sid=750.0, sdd=1200.0)


def fan_case():
    c = FAN
    g = FanGeometry2D(c["shape"], c["spacing"], c["nu"], c["su"], c["views"], 2 * math.pi, c["sid"], c["sdd"])
    return c, g, oracle.uniform_angles(c["views"], 2 * math.pi)


def oracle_fan_loss(x, y, c, ang):
    r = oracle.fp_fan2d(x, c["spacing"], c["nu"], c["su"], ang, c["sid"], c["sdd"]) - y
    return 0.5 * float(np.sum(r * r))


@pytest.mark.parametrize("geom", ["par", "fan", "cone"])
def test_fp_gradient_equals_oracle_adjoint(geom):
    rng = np.random.default_rng(1)
    if geom == "cone":
        shape, sp = (12, 14, 16), (1.0, 1.0, 1.0)
        g = ConeGeometry3D(shape, sp, (18, 22), (1.5, 1.5), 15, 2 * math.pi, 200.0, 350.0)
        ang = g.view_angles()
        P = oracle.circular_pmats(ang, 200.0, 350.0, (18, 22), (1.5, 1.5))
        fwd = lambda v: oracle.fp_cone3d(v, sp, (18, 22), P)
        adj = lambda s: oracle.fpT_cone3d(s, shape, sp, P)
    else:
        shape, sp = (20, 24), (1.0, 1.0)
        if geom == "par":
            g = ParallelGeometry2D(shape, sp, 35, 1.0, 30, math.pi)
            ang = g.view_angles()
            fwd = lambda v: oracle.fp_par2d(v, sp, 35, 1.0, ang)
            adj = lambda s: oracle.fpT_par2d(s, shape, sp, 1.0, ang)
        else:
            g = FanGeometry2D(shape, sp, 35, 1.4, 30, 2 * math.pi, 100.0, 180.0)
            ang = g.view_angles()
            fwd = lambda v: oracle.fp_fan2d(v, sp, 35, 1.4, ang, 100.0, 180.0)
            adj = lambda s: oracle.fpT_fan2d(s, shape, sp, 1.4, ang, 100.0, 180.0)
    x = rng.standard_normal(shape)
    y = rng.standard_normal((g.number_of_projections,) + tuple(np.atleast_1d(g.detector_shape)))
    xt = dev(x).requires_grad_(True)
    loss = 0.5 * ((AG.forward_project(xt, g) - dev(y)) ** 2).sum()
    loss.backward()
    ref = adj(fwd(f32(x)) - f32(y))
    assert rel(xt.grad.double().cpu().numpy(), ref) < 1e-5


def test_fp_gradient_matches_finite_differences():
    """16 single-pixel and 8 random directions: <grad, e> vs the FP64 central
    difference of the oracle's loss."""
    c, g, ang = fan_case()
    rng = np.random.default_rng(2)
    x = f32(ph.voxelize_ellipses(ph.random_ellipses(4, 8.0, seed=3), c["shape"], c["spacing"]).numpy())
    y = f32(rng.standard_normal((c["views"], c["nu"])))
    xt = dev(x).requires_grad_(True)
    loss = 0.5 * ((AG.forward_project(xt, g) - dev(y)) ** 2).sum()
    loss.backward()
    grad = xt.grad.double().cpu().numpy()
    dirs = []
    for _ in range(16):
        e = np.zeros(c["shape"])
        e[tuple(rng.integers(0, 32, 2))] = 1.0
        dirs.append(e)
    dirs += [rng.standard_normal(c["shape"]) for _ in range(8)]
    h = 1e-3
    for e in dirs:
        fd = (oracle_fan_loss(x + h * e, y, c, ang) - oracle_fan_loss(x - h * e, y, c, ang)) / (2 * h)
        assert abs(np.sum(grad * e) - fd) < 1e-5 * max(abs(fd), np.linalg.norm(grad) * np.linalg.norm(e) * 1e-2)


@pytest.mark.parametrize("crop", [(240, 240), (20, 460)])
def test_fp_gradient_finite_differences_on_crops_of_the_full_fan_geometry(crop):
    """The 16-phantom fan workload's geometry in full (512^2 at 0.5 mm, 360
    views over 2 pi, 1024 bins at 1 mm, SID 750, SDD 1200, dt 0.25 mm): the
    loss 1/2 |S (A x - y)|^2 over the rays S that cross a 32 x 32 crop (a
    central one and one near the edge); the gradient on the whole image
    through autograd, then 16 single-pixel and 8 random directions inside the
    crop against FP64 central differences of the oracle's loss."""
    n, sp = 512, (0.5, 0.5)
    g = FanGeometry2D((n, n), sp, 1024, 1.0, 360, 2 * math.pi, 750.0, 1200.0)
    ang = g.view_angles()
    fwd = lambda v: oracle.fp_fan2d(v, sp, 1024, 1.0, ang, 750.0, 1200.0)
    j0, i0 = crop
    box = np.zeros((n, n))
    box[j0:j0 + 32, i0:i0 + 32] = 1.0
    S = fwd(box) > 0.0  # the crop's shadow
    rng = np.random.default_rng(21)
    x = f32(ph.voxelize_ellipses(ph.random_ellipses(10, n * 0.5 / 2, seed=22), (n, n), sp).numpy())
    # data independent of A x, so that the residual does not cancel A x (a
    # residual far below |A x| would amplify the FP32 projection's rounding)
    y = f32(rng.standard_normal(S.shape))
    mask = S.astype(np.float64)
    xt = dev(x).requires_grad_(True)
    loss = 0.5 * (((AG.forward_project(xt, g) - dev(y)) * dev(mask)) ** 2).sum()
    loss.backward()
    grad = xt.grad.double().cpu().numpy()
    r0 = (fwd(x) - y) * mask
    def oracle_loss(v):
        r = (fwd(v) - y) * mask
        return 0.5 * float(np.sum(r * r))
    dirs = []
    for _ in range(16):
        e = np.zeros((n, n))
        e[j0 + rng.integers(0, 32), i0 + rng.integers(0, 32)] = 1.0
        dirs.append(e)
    for _ in range(8):
        e = np.zeros((n, n))
        e[j0:j0 + 32, i0:i0 + 32] = rng.standard_normal((32, 32))
        dirs.append(e)
    h = 1e-3
    for e in dirs:
        fd = (oracle_loss(x + h * e) - oracle_loss(x - h * e)) / (2 * h)
        assert abs(np.sum(grad * e) - fd) < 1e-5 * max(abs(fd), np.linalg.norm(grad * box) * np.linalg.norm(e) * 1e-2)
    assert float(np.sum(r0 * r0)) > 0.0


def test_bp_gradient_is_its_transpose():
    c, g, ang = fan_case()
    rng = np.random.default_rng(4)
    y = rng.standard_normal((c["views"], c["nu"]))
    t = rng.standard_normal(c["shape"])
    yt = dev(y).requires_grad_(True)
    loss = 0.5 * ((AG.back_project(yt, g, B.W_INV_L2, 0.3) - dev(t)) ** 2).sum()
    loss.backward()
    bp = lambda s: oracle.bp_fan2d(s, c["shape"], c["spacing"], c["su"], ang, c["sid"], c["sdd"], 2, 0.3)
    ref = oracle.bpT_fan2d(bp(f32(y)) - f32(t), c["nu"], c["su"], ang, c["spacing"], c["sid"], c["sdd"], 2, 0.3)
    assert rel(yt.grad.double().cpu().numpy(), ref) < 1e-5


def test_ramp_filter_gradients():
    rng = np.random.default_rng(5)
    nu = 50
    pn = B.pyro_filter_pad_length(nu)
    p = rng.standard_normal((6, nu))
    K = rng.uniform(0, 1, pn // 2 + 1)
    t = rng.standard_normal((6, nu))
    pt, Kt = dev(p).requires_grad_(True), dev(K).requires_grad_(True)
    loss = 0.5 * ((AG.ramp_filter(pt, 0.5, Kt) - dev(t)) ** 2).sum()
    loss.backward()
    r = oracle.filter_rows(f32(p), 0.5, oracle.CUSTOM, K=f32(K)) - f32(t)
    assert rel(pt.grad.double().cpu().numpy(), oracle.filter_rows(r, 0.5, oracle.CUSTOM, K=f32(K))) < 1e-5
    assert rel(Kt.grad.double().cpu().numpy(), oracle.filter_grad_K(f32(p), r)) < 1e-5


def test_fdk_module_gradients_match_the_oracle():
    """The learnable-K FDK layer (Eq. 5, 6): dL/dK and dL/dp for
    L = <x, t> against the oracle's chain W, F^H K F, A_bp transposed, and dL/dK
    against FP64 finite differences of the oracle's FDK."""
    nv, nu, s, views = 12, 20, 1.5, 16
    sid, sdd = 150.0, 260.0
    rng_ = short_scan_range(nu * s, sdd)
    g = ConeGeometry3D((8, 10, 12), (1.0, 1.0, 1.0), (nv, nu), (s, s), views, rng_, sid, sdd)
    ang = g.view_angles()
    P = oracle.circular_pmats(ang, sid, sdd, (nv, nu), (s, s))
    # smooth data (phantom projections, a phantom volume as the loss weight)
    e = ph.random_ellipsoids(3, 4.0, seed=7)
    p = f32(an.cone_sinogram(e, ang, (nv, nu), (s, s), sid, sdd))
    t = f32(ph.voxelize_ellipsoids(ph.random_ellipsoids(3, 4.0, seed=9), g.volume_shape, g.volume_spacing).numpy())
    layer = AG.FDK(g, kind=B.RAMLAK, redund=B.REDUND_PARKER, learnable=True, device=DEV)
    K = layer.K.detach().double().cpu().numpy()
    pt = dev(p).requires_grad_(True)
    x = layer(pt)
    (x * dev(t)).sum().backward()
    dbeta = rng_ / views
    ref_x = oracle.fdk(p, g.volume_shape, g.volume_spacing, (s, s), ang, P, sid, sdd, dbeta, oracle.CUSTOM,
                       oracle.REDUND_PARKER, K=K)
    assert rel(x.detach().double().cpu().numpy(), ref_x) < 1e-5
    gq = oracle.bpT_cone3d(t, (nv, nu), g.volume_spacing, P, sid, 2, dbeta)
    tau = s * sid / sdd
    wp = oracle.weights(p, (s, s), ang, sdd, True, oracle.REDUND_PARKER)
    ref_gK = oracle.filter_grad_K(wp, gq)
    ref_gp = oracle.weights(oracle.filter_rows(gq, tau, oracle.CUSTOM, K=K), (s, s), ang, sdd, True,
                            oracle.REDUND_PARKER)
    assert rel(layer.K.grad.double().cpu().numpy(), ref_gK) < 1e-5
    assert rel(pt.grad.double().cpu().numpy(), ref_gp) < 1e-5
    # finite differences of the oracle's FDK in K (linear in K: exact up to rounding)
    for m in (0, 3, 10, len(K) - 1):
        e = np.zeros_like(K)
        e[m] = 1e-2
        lp = np.sum(t * oracle.fdk(p, g.volume_shape, g.volume_spacing, (s, s), ang, P, sid, sdd, dbeta, oracle.CUSTOM,
                                   oracle.REDUND_PARKER, K=K + e))
        lm = np.sum(t * oracle.fdk(p, g.volume_shape, g.volume_spacing, (s, s), ang, P, sid, sdd, dbeta, oracle.CUSTOM,
                                   oracle.REDUND_PARKER, K=K - e))
        fd = (lp - lm) / 2e-2
        assert abs(layer.K.grad[m].item() - fd) < 1e-4 * np.abs(ref_gK).max()


def test_paper_mode_gradient_is_close_to_the_adjoint():
    """The paper's unmatched pair: the scaled voxel-driven BP points nearly
    along A^T r; the defect is reported, not required to vanish."""
    c, g, ang = fan_case()
    rng = np.random.default_rng(8)
    x = rng.standard_normal(c["shape"])
    y = rng.standard_normal((c["views"], c["nu"]))
    grads = []
    for mode in ("exact", "paper"):
        xt = dev(x).requires_grad_(True)
        (0.5 * ((AG.forward_project(xt, g, grad_mode=mode) - dev(y)) ** 2).sum()).backward()
        grads.append(xt.grad.double().cpu().numpy().ravel())
    ge, gp = grads
    cos = ge @ gp / (np.linalg.norm(ge) * np.linalg.norm(gp))
    defect = np.linalg.norm(gp - ge) / np.linalg.norm(ge)
    print(f"paper-mode gradient: cosine {cos:.4f}, relative defect {defect:.3f}")
    assert cos > 0.9
