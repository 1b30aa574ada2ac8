"""Learnable redundancy weights (Section "Geometric Correction Weights"):
the table weighting and its gradient kernel against the oracle and their
definitions, the FDK with a [V, nu] weight table against the oracle's
composition of the same steps, its table gradient against the oracle's
central differences, and a learning run on a short scan."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1904_13342_gb300 import autograd as AG
from paper_1904_13342_gb300 import binding as B
from paper_1904_13342_gb300 import phantoms as ph
from paper_1904_13342_gb300.geometry import ConeGeometry3D, short_scan_range

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def short_scan(shape=(12, 20, 22), views=24):
    nv, nu, sv, su, sid, sdd = 14, 36, 1.4, 1.3, 250.0, 420.0
    return ConeGeometry3D(shape, (1.0, 1.0, 1.0), (nv, nu), (sv, su), views, short_scan_range(nu * su, sdd), sid, sdd)


def oracle_fdk_table(p, g, table):
    """W_cos * table, Shepp-Logan rows, FDK back-projection: the oracle's steps."""
    P = oracle.circular_pmats(g.view_angles(), g.sid, g.sdd, g.detector_shape, g.detector_spacing)
    w = oracle.weights(p, g.detector_spacing, g.view_angles(), g.sdd, cosine=True, redund=oracle.REDUND_NONE)
    w = w * np.asarray(table, np.float64)[:, None, :]
    tau = g.detector_spacing[1] * g.sid / g.sdd
    q = oracle.filter_rows(w, tau, oracle.SHEPP_LOGAN)
    return oracle.bp_cone3d(q, g.volume_shape, g.volume_spacing, P, g.sid, 2, g.angular_range / g.number_of_projections)


def test_weights_table_and_its_gradient_kernel():
    g = short_scan()
    rng = np.random.default_rng(1)
    p = rng.standard_normal((2, *g.sinogram_shape)).astype(np.float32)
    table = rng.uniform(0.0, 1.0, (g.number_of_projections, g.detector_shape[1])).astype(np.float32)
    td = torch.from_numpy(table).to(DEV)
    for cosine in (True, False):
        got = B.pyro_weights3d_table(torch.from_numpy(p).to(DEV), g, td, cosine=cosine).cpu().numpy()
        ref = np.stack([oracle.weights(f32(s), g.detector_spacing, g.view_angles(), g.sdd, cosine=cosine,
                                       redund=oracle.REDUND_NONE) for s in p]) * f32(table)[None, :, None, :]
        assert rel(got, ref) < 1e-6
    a = rng.standard_normal((2, *g.sinogram_shape)).astype(np.float32)
    b = rng.standard_normal((2, *g.sinogram_shape)).astype(np.float32)
    got = B.pyro_redundancy_grad(torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)).cpu().numpy()
    assert rel(got, np.einsum("bvlk,bvlk->vk", f32(a), f32(b))) < 1e-5


def test_table_fdk_matches_the_oracle_and_the_parker_fdk():
    g = short_scan()
    vol = ph.voxelize_ellipsoids(ph.random_ellipsoids(4, 8.0, seed=2), g.volume_shape, g.volume_spacing).numpy()
    P = oracle.circular_pmats(g.view_angles(), g.sid, g.sdd, g.detector_shape, g.detector_spacing)
    p = f32(oracle.fp_cone3d(vol, g.volume_spacing, g.detector_shape, P))
    m = AG.RedundancyFDK(g, init="parker", device=DEV)
    x = m(torch.from_numpy(p).float().to(DEV)).detach()
    ref = oracle_fdk_table(p, g, f32(m.table.detach().cpu().numpy()))
    assert rel(x.cpu().numpy(), ref) < 1e-5
    fused = B.pyro_fdk(torch.from_numpy(p).float().to(DEV), g, kind=B.SHEPP_LOGAN, redund=B.REDUND_PARKER)
    assert rel(x.cpu().numpy(), fused.cpu().numpy()) < 1e-5


def test_table_gradient_matches_oracle_central_differences():
    g = short_scan()
    rng = np.random.default_rng(3)
    vol = ph.voxelize_ellipsoids(ph.random_ellipsoids(4, 8.0, seed=4), g.volume_shape, g.volume_spacing).numpy()
    P = oracle.circular_pmats(g.view_angles(), g.sid, g.sdd, g.detector_shape, g.detector_spacing)
    p = f32(oracle.fp_cone3d(vol, g.volume_spacing, g.detector_shape, P))
    target = f32(vol)
    m = AG.RedundancyFDK(g, init="full", device=DEV)
    x = m(torch.from_numpy(p).float().to(DEV))
    loss = 0.5 * ((x - torch.from_numpy(target).float().to(DEV)) ** 2).sum()
    loss.backward()
    grad = m.table.grad.cpu().numpy().astype(np.float64)
    t0 = f32(m.table.detach().cpu().numpy())
    L = lambda t: 0.5 * float(np.sum((oracle_fdk_table(p, g, t) - target) ** 2))
    h = 1e-2  # the loss is quadratic in the table: central differences are exact up to rounding
    idx = [(0, 5), (3, 17), (11, 30), (23, 2), (17, 18), (9, 35)]
    fd = []
    for v, k in idx:
        tp, tm = t0.copy(), t0.copy()
        tp[v, k] += h
        tm[v, k] -= h
        fd.append((L(tp) - L(tm)) / (2 * h))
    got = np.array([grad[v, k] for v, k in idx])
    assert rel(got, np.array(fd)) < 1e-3, (got, fd)


def test_learned_table_from_the_full_scan_start():
    """Short scan, FDK with W_red = 1/2 everywhere (wrong for a short scan):
    fitting the table by L-BFGS on training phantoms lowers the error well
    below the start, to at most the Parker table's, and moves the table
    toward Parker's."""
    g = ConeGeometry3D((16, 32, 32), (1.0, 1.0, 1.0), (20, 48), (1.4, 1.3), 40, short_scan_range(48 * 1.3, 420.0),
                       250.0, 420.0)
    truth = torch.stack([ph.voxelize_ellipsoids(ph.random_ellipsoids(6, 14.0, seed=s), g.volume_shape,
                                                g.volume_spacing, device=DEV, dtype=torch.float32)
                         for s in range(1000, 1008)])
    p = B.pyro_fp_cone3d(truth, g)
    m = AG.RedundancyFDK(g, init="full", device=DEV)
    opt = torch.optim.LBFGS([m.table], lr=1.0, max_iter=40, history_size=20, line_search_fn="strong_wolfe")
    losses = []

    def closure():
        opt.zero_grad()
        loss = ((m(p) - truth) ** 2).mean()
        loss.backward()
        losses.append(float(loss.item()))
        return loss

    opt.step(closure)
    with torch.no_grad():
        start = losses[0]
        learned = float(((m(p) - truth) ** 2).mean())
        parker = float(((B.pyro_fdk(p, g, kind=B.SHEPP_LOGAN, redund=B.REDUND_PARKER) - truth) ** 2).mean())
        pk = AG.parker_table(g, DEV)
        dist0 = float(torch.linalg.norm(0.5 - pk))
        dist1 = float(torch.linalg.norm(m.table - pk))
    print(f"\nMSE start {start:.4e} learned {learned:.4e} parker {parker:.4e}; |table - parker| {dist0:.3f} -> {dist1:.3f}")
    assert learned < 0.5 * start
    # a least-squares fit on these phantoms: the Parker table is one feasible point
    assert learned <= parker
    assert dist1 < 0.8 * dist0


def test_learned_table_on_a_super_short_scan():
    """A super-short scan (pi + 2 x 3.5 deg; the detector's half fan angle is
    4.25 deg): the table initialised with REDUND_SCAN's weights reproduces the
    fused FDK with those weights, and a table fitted from 1/2 everywhere
    (the paper's 'weights learned for arbitrary short-scan angles') ends at
    most at the scan weights' error."""
    rng_ = math.pi + math.radians(7.0)
    g = ConeGeometry3D((16, 32, 32), (1.0, 1.0, 1.0), (20, 48), (1.4, 1.3), 40, rng_, 250.0, 420.0)
    truth = torch.stack([ph.voxelize_ellipsoids(ph.random_ellipsoids(6, 12.0, seed=s), g.volume_shape,
                                                g.volume_spacing, device=DEV, dtype=torch.float32)
                         for s in range(1000, 1008)])
    p = B.pyro_fp_cone3d(truth, g)
    scan = AG.RedundancyFDK(g, init="scan", device=DEV)
    fused = B.pyro_fdk(p, g, kind=B.SHEPP_LOGAN, redund=B.REDUND_SCAN)
    with torch.no_grad():
        assert rel(scan(p).cpu().numpy(), fused.cpu().numpy()) < 1e-5
    m = AG.RedundancyFDK(g, init="full", device=DEV)
    opt = torch.optim.LBFGS([m.table], lr=1.0, max_iter=40, history_size=20, line_search_fn="strong_wolfe")
    losses = []

    def closure():
        opt.zero_grad()
        loss = ((m(p) - truth) ** 2).mean()
        loss.backward()
        losses.append(float(loss.item()))
        return loss

    opt.step(closure)
    with torch.no_grad():
        learned = float(((m(p) - truth) ** 2).mean())
        ref = float(((fused - truth) ** 2).mean())
        parker = float(((B.pyro_fdk(p, g, kind=B.SHEPP_LOGAN, redund=B.REDUND_PARKER) - truth) ** 2).mean())
    print(f"\nsuper-short MSE start {losses[0]:.4e} learned {learned:.4e} scan weights {ref:.4e} "
          f"parker (detector fan) {parker:.4e}")
    assert learned < 0.5 * losses[0]
    assert learned <= ref
    assert ref < parker  # Parker's weights assume the longer scan pi + 2 delta
