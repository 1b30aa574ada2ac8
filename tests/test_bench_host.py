"""Host-side pieces of bench.py (no GPU): the sample count behind the FP
roofline's achieved FLOP/s.

bench.fp_sample_count estimates, per ray, the chord through the support box
divided by the sample spacing along the ray.  Here the samples are counted
one by one instead: the depth planes w = SID + m dt of the workload, the
point S + w g of each ray on them, and the open support box
(-(N+1)/2 s, (N+1)/2 s)^3 in which the projector's interpolant can be
nonzero."""
import math

import numpy as np
import pytest

import bench


def exact_counts(beta, U, Vv):
    N, s = bench.N, bench.SPACING
    half = 0.5 * (N + 1) * s
    dt = 0.5 * s
    T = 0.5 * math.sqrt(3.0) * (N + 1) * s
    M = math.ceil(T / dt)
    c = np.array([math.cos(beta), math.sin(beta), 0.0])
    eu = np.array([-math.sin(beta), math.cos(beta), 0.0])
    S = -bench.SID * c
    # direction of unit depth along c through detector point (u, v)
    g = c[None, :] + (U.ravel()[:, None] / bench.SDD) * eu[None, :] + (Vv.ravel()[:, None] / bench.SDD) * np.array(
        [0.0, 0.0, 1.0])[None, :]
    w = bench.SID + np.arange(-M, M + 1) * dt
    X = S[None, None, :] + w[None, :, None] * g[:, None, :]
    inside = np.all(np.abs(X) < half, axis=2)
    return inside.sum(axis=1).reshape(U.shape)


@pytest.mark.parametrize("beta", [0.0, 0.7, 2.1, 3.3])
def test_sample_estimate_matches_the_exact_count(beta):
    g = bench.geometry()
    nv, nu = g.detector_shape
    sv, su = g.detector_spacing
    u = (np.arange(0, nu, 29) - 0.5 * (nu - 1)) * su
    v = (np.arange(0, nv, 23) - 0.5 * (nv - 1)) * sv
    U, Vv = np.meshgrid(u, v)
    est = bench.ray_sample_estimate(beta, U, Vv)
    exact = exact_counts(beta, U, Vv)
    # each ray's estimate is within one sample of its count
    assert np.max(np.abs(est - exact)) <= 1.0 + 1e-9
    assert abs(est.sum() - exact.sum()) <= 5e-3 * exact.sum()
    assert exact.sum() > 0


def test_view_subsampling_of_the_count():
    """Every 15th view, scaled, against all views (coarse ray grid)."""
    g = bench.geometry()
    nv, nu = g.detector_shape
    sv, su = g.detector_spacing
    u = (np.arange(0, nu, 31) - 0.5 * (nu - 1)) * su
    v = (np.arange(0, nv, 31) - 0.5 * (nv - 1)) * sv
    U, Vv = np.meshgrid(u, v)
    ang = g.view_angles()
    full = sum(bench.ray_sample_estimate(b, U, Vv).sum() for b in ang)
    sub = ang[:: max(1, len(ang) // 16)]
    scaled = sum(bench.ray_sample_estimate(b, U, Vv).sum() for b in sub) * len(ang) / len(sub)
    assert abs(scaled - full) <= 5e-3 * full
