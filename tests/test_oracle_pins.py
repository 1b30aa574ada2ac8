"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test compares the oracle with something computed independently of it:
closed-form line integrals of Gaussian blobs and ellipses, brute-force
evaluation of the same discrete operators through the tent-basis form of
linear interpolation and ray/detector-plane intersections written out here,
exact identities (adjointness, the Parker conjugate-ray sum), analytic
reconstructions (uniform disk / sphere), and library routines (numpy FFT).
"""
import copy

import numpy as np
import pytest

import analytic as an
import oracle
from paper_1904_13342_gb300 import phantoms as ph

pytestmark = pytest.mark.filterwarnings("ignore")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def smoothed(b, h, dim):
    """Blobs seen through linear interpolation of their point samples: the
    interpolant of a smooth f carries on average the extra variance h^2/6 per
    axis (tent kernel), at equal total mass."""
    b2 = copy.deepcopy(b)
    b2.cov = b.cov + np.eye(dim)[None] * h * h / 6.0
    b2.density = b.density * np.sqrt(np.linalg.det(b.cov) / np.linalg.det(b2.cov))
    return b2


# ------------------------------------------------------------------ FP ---

def test_fp_par2d_matches_blob_line_integrals():
    N, s = 128, 1.0
    b = ph.random_blobs(6, N * s / 2, 2, seed=0)
    img = ph.sample_blobs(b, (N, N), (s, s)).numpy()
    ang = oracle.uniform_angles(180, np.pi)
    sino = oracle.fp_par2d(img, (s, s), 183, 1.0, ang)
    a, d = an.parallel_rays(ang, 183, 1.0)
    ref = an.blob_line_integrals(smoothed(b, s, 2), a, d).reshape(180, 183)
    assert rel(sino, ref) < 1e-3
    # the pin is sharp: a 0.05-pixel detector shift is already visible
    eu = np.stack([-np.sin(np.repeat(ang, 183)), np.cos(np.repeat(ang, 183))], 1)
    shifted = an.blob_line_integrals(smoothed(b, s, 2), a + 0.05 * eu, d).reshape(180, 183)
    assert rel(sino, shifted) > 2e-3


def test_fp_fan2d_matches_blob_line_integrals():
    N, s = 256, 0.5
    b = ph.random_blobs(6, N * s / 2, 2, seed=1)
    img = ph.sample_blobs(b, (N, N), (s, s)).numpy()
    ang = oracle.uniform_angles(90, 2 * np.pi)
    sino = oracle.fp_fan2d(img, (s, s), 512, 1.0, ang, 750.0, 1200.0)
    a, d = an.fan_rays(ang, 512, 1.0, 750.0, 1200.0)
    ref = an.blob_line_integrals(smoothed(b, s, 2), a, d).reshape(90, 512)
    assert rel(sino, ref) < 2e-4


def test_fp_cone3d_matches_blob_line_integrals():
    N, s = 64, 1.0
    b = ph.random_blobs(5, N * s / 2, 3, seed=2, sigma=(0.08, 0.14), spread=0.3)
    vol = ph.sample_blobs(b, (N, N, N), (s, s, s)).numpy()
    ang = 0.37 + oracle.uniform_angles(8, 2 * np.pi)
    P = oracle.circular_pmats(ang, 750.0, 1200.0, (70, 80), (1.6, 1.6))
    sino = oracle.fp_cone3d(vol, (s, s, s), (70, 80), P)
    a, d = an.cone_rays(ang, 80, 70, 1.6, 1.6, 750.0, 1200.0)
    ref = an.blob_line_integrals(smoothed(b, s, 3), a, d).reshape(8, 70, 80)
    assert rel(sino, ref) < 3e-3
    up = an.blob_line_integrals(smoothed(b, s, 3), a + np.array([0, 0, 0.05]), d).reshape(8, 70, 80)
    assert rel(sino, up) > 5e-3


def test_fp_par2d_matches_ellipse_line_integrals():
    """128^2 phantom of 10 random ellipses (4x4 supersampled): the sampled
    projector follows the analytic projections to discretisation error,
    while a mirrored detector axis is far off."""
    N, s = 128, 1.0
    e = ph.random_ellipses(10, N * s / 2, seed=0)
    img = ph.voxelize_ellipses(e, (N, N), (s, s), supersample=4).numpy()
    ang = oracle.uniform_angles(180, np.pi)
    sino = oracle.fp_par2d(img, (s, s), 183, 1.0, ang)
    a, d = an.parallel_rays(ang, 183, 1.0)
    ref = an.ellipse_line_integrals(e, a, d).reshape(180, 183)
    assert rel(sino, ref) < 3.5e-2
    assert rel(sino, ref[:, ::-1]) > 0.5


def _tent(f, n):
    """[M, n] tent-basis weights max(0, 1 - |f - i|) of positions f [M]."""
    return np.maximum(0.0, 1.0 - np.abs(f[:, None] - np.arange(n)[None, :]))


def _depth_param(a, d, parallel):
    """Ray written as X(w) = a + w g with unit depth along the view's
    principal axis c: parallel beam c = d, w0 = 0; fan / cone c points from
    the source a to the iso-centre, w0 = |a| (the iso-centre's depth)."""
    if parallel:
        return d, 0.0
    c = -a / np.linalg.norm(a)
    return d / (d @ c), float(np.linalg.norm(a))


def _brute_line2(img, s, dt, a, d, parallel):
    ny, nx = img.shape
    T = 0.5 * np.hypot((nx + 1) * s[1], (ny + 1) * s[0])
    M = int(np.ceil(T / dt))
    g, w0 = _depth_param(a, d, parallel)
    w = w0 + np.arange(-M, M + 1) * dt
    X = a[None, :] + w[:, None] * g[None, :]
    hx = _tent(X[:, 0] / s[1] + 0.5 * (nx - 1), nx)
    hy = _tent(X[:, 1] / s[0] + 0.5 * (ny - 1), ny)
    return dt * np.linalg.norm(g) * np.einsum("mj,ji,mi->", hy, img, hx)


def _brute_line3(vol, s, dt, a, d):
    nz, ny, nx = vol.shape
    T = 0.5 * np.sqrt(((nx + 1) * s[2]) ** 2 + ((ny + 1) * s[1]) ** 2 + ((nz + 1) * s[0]) ** 2)
    M = int(np.ceil(T / dt))
    g, w0 = _depth_param(a, d, False)
    w = w0 + np.arange(-M, M + 1) * dt
    X = a[None, :] + w[:, None] * g[None, :]
    hx = _tent(X[:, 0] / s[2] + 0.5 * (nx - 1), nx)
    hy = _tent(X[:, 1] / s[1] + 0.5 * (ny - 1), ny)
    hz = _tent(X[:, 2] / s[0] + 0.5 * (nz - 1), nz)
    return dt * np.linalg.norm(g) * np.einsum("mk,mj,mi,kji->", hz, hy, hx, vol)


def test_fp_bruteforce_tent_basis_2d():
    rng = np.random.default_rng(5)
    img = rng.standard_normal((8, 7))
    s = (0.9, 1.1)
    ang = rng.uniform(0, 2 * np.pi, 5)
    dt = 0.3
    par = oracle.fp_par2d(img, s, 9, 1.3, ang, step=dt)
    fan = oracle.fp_fan2d(img, s, 9, 1.3, ang, 40.0, 70.0, step=dt)
    a, d = an.parallel_rays(ang, 9, 1.3)
    ref = np.array([_brute_line2(img, s, dt, a[r], d[r], True) for r in range(a.shape[0])]).reshape(5, 9)
    assert np.max(np.abs(par - ref)) < 1e-12 * np.max(np.abs(ref))
    a, d = an.fan_rays(ang, 9, 1.3, 40.0, 70.0)
    ref = np.array([_brute_line2(img, s, dt, a[r], d[r], False) for r in range(a.shape[0])]).reshape(5, 9)
    assert np.max(np.abs(fan - ref)) < 1e-12 * np.max(np.abs(ref))


def test_fp_bruteforce_tent_basis_3d():
    rng = np.random.default_rng(6)
    vol = rng.standard_normal((5, 7, 6))
    s = (1.2, 0.8, 1.0)
    ang = rng.uniform(0, 2 * np.pi, 3)
    dt = 0.35
    P = oracle.circular_pmats(ang, 40.0, 70.0, (6, 8), (1.5, 1.7))
    sino = oracle.fp_cone3d(vol, s, (6, 8), P, step=dt)
    a, d = an.cone_rays(ang, 8, 6, 1.7, 1.5, 40.0, 70.0)
    ref = np.array([_brute_line3(vol, s, dt, a[r], d[r]) for r in range(a.shape[0])]).reshape(3, 6, 8)
    assert np.max(np.abs(sino - ref)) < 1e-12 * np.max(np.abs(ref))


def test_fp_cone_central_row_equals_fan_of_slice():
    """A volume constant along z, seen by the central row of an odd-height
    detector, projects exactly like its slice in the fan-beam geometry."""
    rng = np.random.default_rng(7)
    sl = rng.standard_normal((16, 16))
    vol = np.repeat(sl[None], 9, axis=0)
    ang = oracle.uniform_angles(7, 2 * np.pi)
    P = oracle.circular_pmats(ang, 60.0, 100.0, (5, 21), (1.0, 1.4))
    cone = oracle.fp_cone3d(vol, (1.0, 1.0, 1.0), (5, 21), P, step=0.5)
    fan = oracle.fp_fan2d(sl, (1.0, 1.0), 21, 1.4, ang, 60.0, 100.0, step=0.5)
    assert np.max(np.abs(cone[:, 2, :] - fan)) < 1e-12 * np.max(np.abs(fan))


def test_pmats_project_points_onto_flat_detector():
    """P (X,1) agrees with the intersection of the source ray through X
    with the detector plane, computed here from the geometry."""
    rng = np.random.default_rng(8)
    ang = rng.uniform(0, 2 * np.pi, 6)
    sid, sdd, nu, nv, su, sv = 750.0, 1200.0, 620, 480, 0.616, 0.616
    P = oracle.circular_pmats(ang, sid, sdd, (nv, nu), (sv, su))
    for j, b in enumerate(ang):
        c = np.array([np.cos(b), np.sin(b), 0.0])
        eu = np.array([-np.sin(b), np.cos(b), 0.0])
        ev = np.array([0.0, 0.0, 1.0])
        S = -sid * c
        for X in rng.uniform(-60, 60, (5, 3)):
            t = sdd / (c @ (X - S))  # line S + t (X - S) meets the plane c.Y = sdd - sid
            Y = S + t * (X - S)
            k = (Y @ eu) / su + 0.5 * (nu - 1)
            l = (Y @ ev) / sv + 0.5 * (nv - 1)
            x, y, w = P[j] @ np.append(X, 1.0)
            assert abs(x / w - k) < 1e-9 and abs(y / w - l) < 1e-9
            assert abs(w - c @ (X - S)) < 1e-9  # w is the depth along the central ray
        assert np.allclose(np.cross(eu, ev), c)  # right-handed detector frame


def test_fp_cone_rays_equals_full_projection():
    rng = np.random.default_rng(9)
    vol = rng.standard_normal((6, 7, 8))
    ang = oracle.uniform_angles(4, 2 * np.pi)
    P = oracle.circular_pmats(ang, 50.0, 90.0, (5, 9), (1.5, 1.5))
    full = oracle.fp_cone3d(vol, (1, 1, 1), (5, 9), P)
    v, l, k = np.meshgrid(np.arange(4), np.arange(5), np.arange(9), indexing="ij")
    part = oracle.fp_cone3d_rays(vol, (1, 1, 1), P, v.ravel(), k.ravel(), l.ravel())
    assert np.array_equal(part.reshape(full.shape), full)


# ------------------------------------------------------ adjoint pairs ---

@pytest.mark.parametrize("geom", ["par", "fan", "cone"])
def test_fp_adjointness(geom):
    rng = np.random.default_rng(10)
    if geom == "cone":
        x = rng.standard_normal((7, 8, 9))
        ang = rng.uniform(0, 2 * np.pi, 5)
        P = oracle.circular_pmats(ang, 40.0, 70.0, (6, 10), (1.6, 1.5))
        Ax = oracle.fp_cone3d(x, (1, 1.1, 0.9), (6, 10), P)
        y = rng.standard_normal(Ax.shape)
        ATy = oracle.fpT_cone3d(y, x.shape, (1, 1.1, 0.9), P)
    else:
        x = rng.standard_normal((11, 9))
        ang = rng.uniform(0, 2 * np.pi, 6)
        if geom == "par":
            Ax = oracle.fp_par2d(x, (1.0, 1.2), 13, 1.1, ang)
            y = rng.standard_normal(Ax.shape)
            ATy = oracle.fpT_par2d(y, x.shape, (1.0, 1.2), 1.1, ang)
        else:
            Ax = oracle.fp_fan2d(x, (1.0, 1.2), 13, 1.1, ang, 30.0, 55.0)
            y = rng.standard_normal(Ax.shape)
            ATy = oracle.fpT_fan2d(y, x.shape, (1.0, 1.2), 1.1, ang, 30.0, 55.0)
    lhs, rhs = np.sum(Ax * y), np.sum(x * ATy)
    assert abs(lhs - rhs) < 1e-12 * np.sqrt(np.sum(Ax * Ax) * np.sum(y * y))


def test_fpT_cone3d_voxels_equals_the_full_adjoint():
    """The adjoint evaluated voxel by voxel (gathering the rays and planes
    whose samples fall in a voxel's support) equals the ray-by-ray scatter at
    every voxel, on a circular and on a tilted trajectory with anisotropic
    spacing."""
    rng = np.random.default_rng(12)
    shape, sp = (7, 8, 9), (1.0, 1.1, 0.9)
    ang = rng.uniform(0, 2 * np.pi, 5)
    P = oracle.circular_pmats(ang, 40.0, 70.0, (6, 10), (1.6, 1.5))
    ct, st = np.cos(0.2), np.sin(0.2)
    tilt = np.array([[1, 0, 0, 0], [0, ct, -st, 0], [0, st, ct, 0], [0, 0, 0, 1.0]])
    for pm in (P, P @ tilt):
        y = rng.standard_normal((5, 6, 10))
        full = oracle.fpT_cone3d(y, shape, sp, pm)
        kk, jj, ii = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
        vox = oracle.fpT_cone3d_voxels(y, shape, sp, pm, ii.ravel(), jj.ravel(), kk.ravel())
        assert np.max(np.abs(vox - full.ravel())) < 1e-12 * np.max(np.abs(full))


@pytest.mark.parametrize("geom", ["par", "fan", "cone"])
def test_bp_transpose_identity(geom):
    rng = np.random.default_rng(11)
    if geom == "cone":
        shape, sp = (6, 7, 8), (1.0, 1.1, 0.9)
        ang = rng.uniform(0, 2 * np.pi, 5)
        P = oracle.circular_pmats(ang, 40.0, 70.0, (6, 10), (1.6, 1.5))
        y = rng.standard_normal((5, 6, 10))
        Bx = oracle.bp_cone3d(y, shape, sp, P, 40.0, weight=2, scale=0.7)
        g = rng.standard_normal(shape)
        BTg = oracle.bpT_cone3d(g, (6, 10), sp, P, 40.0, weight=2, scale=0.7)
    else:
        shape, sp = (10, 9), (1.0, 1.2)
        ang = rng.uniform(0, 2 * np.pi, 6)
        y = rng.standard_normal((6, 13))
        g = rng.standard_normal(shape)
        if geom == "par":
            Bx = oracle.bp_par2d(y, shape, sp, 1.1, ang, scale=0.3)
            BTg = oracle.bpT_par2d(g, 13, 1.1, ang, sp, scale=0.3)
        else:
            Bx = oracle.bp_fan2d(y, shape, sp, 1.1, ang, 30.0, 55.0, weight=1, scale=0.3)
            BTg = oracle.bpT_fan2d(g, 13, 1.1, ang, sp, 30.0, 55.0, weight=1, scale=0.3)
    lhs, rhs = np.sum(Bx * g), np.sum(y * BTg)
    assert abs(lhs - rhs) < 1e-12 * np.sqrt(np.sum(Bx * Bx) * np.sum(g * g))


# ---------------------------------------------------------------- BP ----

def _tent_bp_2d(y, shape, sp, su, ang, fan, sid, sdd, wexp, scale):
    """Voxel-driven BP through line/plane intersection and tent weights."""
    ny, nx = shape
    nu = y.shape[1]
    out = np.zeros(shape)
    for j in range(ny):
        for i in range(nx):
            X = np.array([(i - 0.5 * (nx - 1)) * sp[1], (j - 0.5 * (ny - 1)) * sp[0]])
            acc = 0.0
            for v, b in enumerate(ang):
                c = np.array([np.cos(b), np.sin(b)])
                eu = np.array([-np.sin(b), np.cos(b)])
                if fan:
                    S = -sid * c
                    t = sdd / (c @ (X - S))
                    u = eu @ (S + t * (X - S))
                    w = (sid / (c @ (X - S))) ** wexp
                else:
                    u, w = X @ eu, 1.0
                kk = u / su + 0.5 * (nu - 1)
                acc += w * np.sum(y[v] * np.maximum(0.0, 1.0 - np.abs(kk - np.arange(nu))))
            out[j, i] = scale * acc
    return out


def test_bp_2d_bruteforce():
    rng = np.random.default_rng(12)
    y = rng.standard_normal((5, 11))
    ang = rng.uniform(0, 2 * np.pi, 5)
    shape, sp = (7, 6), (1.1, 0.9)
    ref = _tent_bp_2d(y, shape, sp, 1.2, ang, False, 0, 0, 0, 0.4)
    assert np.allclose(oracle.bp_par2d(y, shape, sp, 1.2, ang, scale=0.4), ref, rtol=0, atol=1e-12)
    for wexp in (0, 1, 2):
        ref = _tent_bp_2d(y, shape, sp, 1.2, ang, True, 30.0, 50.0, wexp, 0.4)
        got = oracle.bp_fan2d(y, shape, sp, 1.2, ang, 30.0, 50.0, weight=wexp, scale=0.4)
        assert np.allclose(got, ref, rtol=0, atol=1e-12)


def test_bp_cone_bruteforce_and_voxel_list():
    rng = np.random.default_rng(13)
    ang = rng.uniform(0, 2 * np.pi, 4)
    sid, sdd, nu, nv, su, sv = 40.0, 65.0, 10, 8, 1.4, 1.6
    P = oracle.circular_pmats(ang, sid, sdd, (nv, nu), (sv, su))
    y = rng.standard_normal((4, nv, nu))
    shape, sp = (5, 6, 7), (1.0, 0.9, 1.1)
    got = oracle.bp_cone3d(y, shape, sp, P, sid, weight=2, scale=0.5)
    nz, ny, nx = shape
    ref = np.zeros(shape)
    for kz in range(nz):
        for j in range(ny):
            for i in range(nx):
                X = np.array([(i - 0.5 * (nx - 1)) * sp[2], (j - 0.5 * (ny - 1)) * sp[1], (kz - 0.5 * (nz - 1)) * sp[0]])
                acc = 0.0
                for v, b in enumerate(ang):
                    c = np.array([np.cos(b), np.sin(b), 0.0])
                    eu = np.array([-np.sin(b), np.cos(b), 0.0])
                    S = -sid * c
                    L = c @ (X - S)
                    Y = S + (sdd / L) * (X - S)
                    kk = (Y @ eu) / su + 0.5 * (nu - 1)
                    ll = Y[2] / sv + 0.5 * (nv - 1)
                    tk = np.maximum(0.0, 1.0 - np.abs(kk - np.arange(nu)))
                    tl = np.maximum(0.0, 1.0 - np.abs(ll - np.arange(nv)))
                    acc += (sid / L) ** 2 * (tl @ y[v] @ tk)
                ref[kz, j, i] = 0.5 * acc
    assert np.allclose(got, ref, rtol=0, atol=1e-12)
    ii, jj, kk = rng.integers(0, nx, 9), rng.integers(0, ny, 9), rng.integers(0, nz, 9)
    part = oracle.bp_cone3d_voxels(y, shape, sp, P, sid, ii, jj, kk, weight=2, scale=0.5)
    assert np.array_equal(part, got[kk, jj, ii])


def test_bp_parallel_constant_sinogram():
    """BP of a constant sinogram is N_views * scale wherever every view's
    projection falls inside the detector."""
    ang = oracle.uniform_angles(30, np.pi)
    y = np.full((30, 41), 2.0)
    img = oracle.bp_par2d(y, (16, 16), (1.0, 1.0), 1.0, ang, scale=0.25)
    assert np.allclose(img, 30 * 0.25 * 2.0, rtol=0, atol=1e-12)


# ------------------------------------------------ weights and filters ---

def test_parker_conjugate_rays_sum_to_one():
    """w(b, g) + w(b + pi + 2 g, -g) = 1 on the short scan pi + 2 delta."""
    delta = np.arctan(0.5 * 620 * 0.616 / 1200.0)
    rng = np.random.default_rng(14)
    for _ in range(4000):
        g = rng.uniform(-delta, delta)
        b = rng.uniform(0, np.pi + 2 * delta)
        w = oracle.parker_weight(b, g, delta)
        assert 0.0 <= w <= 1.0
        b2 = b + np.pi + 2 * g
        if b2 > 2 * np.pi:
            b2 -= 2 * np.pi
        if 0 <= b2 <= np.pi + 2 * delta:
            assert abs(w + oracle.parker_weight(b2, -g, delta) - 1.0) < 1e-12
    # continuity across the region borders
    for g in (-0.1, 0.0, 0.12):
        for edge in (2 * (delta - g), np.pi - 2 * g):
            a, b = oracle.parker_weight(edge - 1e-9, g, delta), oracle.parker_weight(edge + 1e-9, g, delta)
            assert abs(a - b) < 1e-7


def _same_line(a1, d1, a2, d2, tol=1e-9):
    """two 2D rays (origin, unit direction) lie on one line"""
    cross = d1[0] * d2[1] - d1[1] * d2[0]
    off = (a2[0] - a1[0]) * d1[1] - (a2[1] - a1[1]) * d1[0]
    return abs(cross) < tol and abs(off) < tol * 1e3


def test_conjugate_ray_convention_matches_the_fan_geometry():
    """The partner (beta + pi + 2 gamma, -gamma) the scan weights assume is
    the same line as (beta, gamma), built from the source and detector
    positions of the geometry (a symmetric detector: bin nu-1-k has -gamma)."""
    nu, su, sid, sdd = 65, 1.3, 400.0, 700.0
    rng = np.random.default_rng(41)
    for _ in range(50):
        b, k = rng.uniform(0, 2 * np.pi), int(rng.integers(nu))
        g = np.arctan((k - 0.5 * (nu - 1)) * su / sdd)
        a1, d1 = an.fan_rays([b], nu, su, sid, sdd)
        a2, d2 = an.fan_rays([b + np.pi + 2 * g], nu, su, sid, sdd)
        assert _same_line(a1[k], d1[k], a2[nu - 1 - k], d2[nu - 1 - k])
        # and not the other sign
        a3, d3 = an.fan_rays([b + np.pi - 2 * g], nu, su, sid, sdd)
        if abs(g) > 1e-3:
            assert not _same_line(a1[k], d1[k], a3[nu - 1 - k], d3[nu - 1 - k])


@pytest.mark.parametrize("frac", [-0.6, 0.0, 0.4, 1.0, 1.7, None])
def test_scan_weights_partition_every_line(frac):
    """Scan over [0, R] for R from below pi to 2 pi: every ray's line, summed
    over all its measurements inside the scan (brute-force enumeration of
    the partners at beta +- pi + 2 gamma, with their 2 pi images), has total
    weight 1; 0 <= w <= 1; and R = pi + 2 delta gives Parker's weights."""
    delta = np.arctan(0.5 * 620 * 0.616 / 1200.0)
    R = 2 * np.pi if frac is None else np.pi + 2 * frac * delta
    rng = np.random.default_rng(42)
    for _ in range(3000):
        g = rng.uniform(-delta, delta)
        b = rng.uniform(0, R)
        w = oracle.scan_weight(b, g, R)
        assert 0.0 <= w <= 1.0
        total, seen = w, []
        for b2 in [b + np.pi + 2 * g + 2 * np.pi * m for m in (-2, -1, 0, 1)]:
            if 0.0 <= b2 <= R and all(abs(b2 - x) > 1e-9 for x in seen):
                seen.append(b2)
                total += oracle.scan_weight(b2, -g, R)
        assert abs(total - 1.0) < 1e-12, (b, g, R, w, total)
        if frac == 1.0:
            assert abs(w - oracle.parker_weight(b, g, delta)) < 1e-12
    # outside the scan: 0; inside, continuous across the overlap borders
    assert oracle.scan_weight(-1e-9, 0.01, R) == 0.0 and oracle.scan_weight(R + 1e-9, 0.01, R) == 0.0
    for g in (-0.1, 0.0, 0.07):
        for edge in (R - np.pi - 2 * g, np.pi - 2 * g):
            if 1e-6 < edge < R - 1e-6:
                lo, hi = oracle.scan_weight(edge - 1e-9, g, R), oracle.scan_weight(edge + 1e-9, g, R)
                assert abs(lo - hi) < 1e-6


def test_filter_rows_equals_fft_circular_convolution():
    """Linear convolution with the Ram-Lak / Shepp-Logan taps equals F^H K F
    on the zero-padded row (numpy FFT), K the DFT of the truncated taps."""
    rng = np.random.default_rng(15)
    nu, tau = 37, 0.7
    rows = rng.standard_normal((4, nu))
    pn = oracle.pad_length(nu)
    assert pn == 128
    n = np.arange(pn)
    n = np.where(n < pn // 2, n, n - pn)
    nf = n.astype(float)
    odd = np.abs(n) % 2 == 1
    h_rl = np.zeros(pn)
    h_rl[n == 0] = 1.0 / (4 * tau * tau)
    h_rl[odd] = -1.0 / (np.pi ** 2 * tau * tau * nf[odd] ** 2)
    h_sl = -2.0 / (np.pi ** 2 * tau * tau * (4.0 * nf ** 2 - 1))
    for kind, h in ((oracle.RAMLAK, h_rl), (oracle.SHEPP_LOGAN, h_sl)):
        h = h.copy()
        h[pn // 2] = 0.0
        K = np.fft.fft(tau * h)
        ref = np.real(np.fft.ifft(np.fft.fft(rows, pn) * K))[:, :nu]
        got = oracle.filter_rows(rows, tau, kind)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    # ramp and a custom K go through the naive DFT: compare with numpy FFT
    Kr = np.abs(n) / (pn * tau)
    ref = np.real(np.fft.ifft(np.fft.fft(rows, pn) * Kr))[:, :nu]
    assert np.max(np.abs(oracle.filter_rows(rows, tau, oracle.RAMP) - ref)) < 1e-12 * np.max(np.abs(ref))
    Kc = rng.uniform(0, 1, pn // 2 + 1)
    Kfull = Kc[np.abs(n)]
    ref = np.real(np.fft.ifft(np.fft.fft(rows, pn) * Kfull))[:, :nu]
    got = oracle.filter_rows(rows, tau, oracle.CUSTOM, K=Kc)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_ramlak_frequency_response_is_the_ramp():
    """Kak & Slaney: the Ram-Lak taps are the band-limited ramp |f|, so the
    response to a pure cosine of frequency m/pn is |m|/(pn tau) (mid band),
    and the DC response is ~0."""
    nu, tau = 256, 0.5
    pn = oracle.pad_length(nu)
    k = np.arange(nu)
    for m in (16, 40, 100):
        row = np.cos(2 * np.pi * m * k / pn)
        q = oracle.filter_rows(row[None], tau, oracle.RAMLAK)[0]
        mid = slice(nu // 4, 3 * nu // 4)
        gain = np.sum(q[mid] * row[mid]) / np.sum(row[mid] * row[mid])
        assert abs(gain - m / (pn * tau)) < 0.02 * m / (pn * tau)
    q = oracle.filter_rows(np.ones((1, nu)), tau, oracle.RAMLAK)[0]
    assert abs(q[nu // 2]) < 0.01 / tau


def test_filter_grad_K_matches_finite_differences():
    rng = np.random.default_rng(16)
    nu = 13
    p = rng.standard_normal((3, nu))
    g = rng.standard_normal((3, nu))
    pn = oracle.pad_length(nu)
    K = rng.uniform(0, 1, pn // 2 + 1)
    dK = oracle.filter_grad_K(p, g)
    for m in range(pn // 2 + 1):
        e = np.zeros_like(K)
        e[m] = 1e-3
        lp = np.sum(g * oracle.filter_rows(p, 1.0, oracle.CUSTOM, K=K + e))
        lm = np.sum(g * oracle.filter_rows(p, 1.0, oracle.CUSTOM, K=K - e))
        assert abs((lp - lm) / 2e-3 - dK[m]) < 1e-9 * max(1.0, abs(dK[m]))


# ------------------------------------------------------------ FBP/FDK ---

def test_fbp_par2d_uniform_disk():
    """Ram-Lak FBP of the analytic projections of an off-centre uniform disk
    returns its density inside 0.8 r (1 %); the frequency-sampled ramp shows
    the DC offset / cupping the paper describes for an undiscretised ramp."""
    N, s, nu, su = 128, 1.0, 183, 1.0
    r, mu, c = 30.0, 1.0, (12.0, -9.0)
    ang = oracle.uniform_angles(360, np.pi)
    sino = an.disk_parallel_sinogram(r, mu, c, ang, nu, su)
    img = oracle.fbp_par2d(sino, (N, N), (s, s), su, ang, kind=oracle.RAMLAK)
    x = (np.arange(N) - 0.5 * (N - 1)) * s
    X, Y = np.meshgrid(x, x)
    dist = np.hypot(X - c[0], Y - c[1])
    inside, outside = dist < 0.8 * r, dist > 1.2 * r
    assert np.max(np.abs(img[inside] - mu)) < 0.01 * mu
    assert abs(np.mean(img[outside])) < 0.01 * mu
    ramp = oracle.fbp_par2d(sino, (N, N), (s, s), su, ang, kind=oracle.RAMP)
    assert abs(np.mean(ramp[inside]) - mu) > 0.005 * mu


@pytest.mark.parametrize("redund", [oracle.REDUND_FULL, oracle.REDUND_PARKER, oracle.REDUND_SCAN])
def test_fbp_fan2d_uniform_disk(redund):
    """REDUND_SCAN runs a super-short scan: pi plus twice the disk's own half
    fan angle (6.1 deg) and a margin, shorter than pi + 2 delta (delta 12.4 deg)."""
    N, s, nu, su, sid, sdd = 128, 1.0, 256, 1.2, 400.0, 700.0
    r, mu, c = 25.0, 1.0, (-14.0, 10.0)
    delta = np.arctan(0.5 * nu * su / sdd)
    rng_ = {oracle.REDUND_FULL: 2 * np.pi, oracle.REDUND_PARKER: np.pi + 2 * delta,
            oracle.REDUND_SCAN: np.pi + 2 * np.radians(7.5)}[redund]
    nviews = 360 if redund == oracle.REDUND_FULL else 220
    ang = oracle.uniform_angles(nviews, rng_)
    a, d = an.fan_rays(ang, nu, su, sid, sdd)
    disk = ph.Ellipses(np.array([c]), np.array([[r, r]]), np.array([0.0]), np.array([mu]))
    sino = an.ellipse_line_integrals(disk, a, d).reshape(nviews, nu)
    img = oracle.fbp_fan2d(sino, (N, N), (s, s), su, ang, sid, sdd, rng_ / nviews, kind=oracle.RAMLAK, redund=redund,
                           scan_range=rng_)
    if redund == oracle.REDUND_SCAN:
        # control: Parker's weights for the full detector fan on this shorter scan miss the lines' late halves
        bad = oracle.fbp_fan2d(sino, (N, N), (s, s), su, ang, sid, sdd, rng_ / nviews, kind=oracle.RAMLAK,
                               redund=oracle.REDUND_PARKER)
    x = (np.arange(N) - 0.5 * (N - 1)) * s
    X, Y = np.meshgrid(x, x)
    dist = np.hypot(X - c[0], Y - c[1])
    assert np.max(np.abs(img[dist < 0.8 * r] - mu)) < 0.015 * mu
    assert abs(np.mean(img[dist > 1.2 * r])) < 0.01 * mu
    if redund == oracle.REDUND_SCAN:
        assert np.max(np.abs(bad[dist < 0.8 * r] - mu)) > 0.015 * mu  # fails the gate the scan weights pass


@pytest.mark.parametrize("redund", [oracle.REDUND_FULL, oracle.REDUND_PARKER, oracle.REDUND_SCAN])
def test_fdk_uniform_sphere(redund):
    """FDK (Eq. 5) of the analytic cone projections of an off-centre sphere:
    the mid-plane through the sphere reconstructs its density within 2 %.
    REDUND_SCAN: a super-short scan of pi + 2 x 5.5 deg (the sphere's half fan
    angle is 4.2 deg, the detector's 7.3 deg)."""
    n, s = 64, 1.0
    nu, nv, su, sv, sid, sdd = 128, 96, 1.0, 1.0, 300.0, 500.0
    r, mu, c = 12.0, 1.0, np.array([8.0, -6.0, 2.0])
    delta = np.arctan(0.5 * nu * su / sdd)
    rng_ = {oracle.REDUND_FULL: 2 * np.pi, oracle.REDUND_PARKER: np.pi + 2 * delta,
            oracle.REDUND_SCAN: np.pi + 2 * np.radians(5.5)}[redund]
    nviews = 180 if redund == oracle.REDUND_FULL else 120
    ang = oracle.uniform_angles(nviews, rng_)
    P = oracle.circular_pmats(ang, sid, sdd, (nv, nu), (sv, su))
    a, d = an.cone_rays(ang, nu, nv, su, sv, sid, sdd)
    sph = ph.Ellipsoids(c[None], np.array([[r, r, r]]), np.eye(3)[None], np.array([mu]))
    sino = an.ellipsoid_line_integrals(sph, a, d).reshape(nviews, nv, nu)
    kz = int(round(c[2] / s + 0.5 * (n - 1)))
    # reconstruct the slice through the sphere centre only, via the voxel list
    x = (np.arange(n) - 0.5 * (n - 1)) * s
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    vals = oracle.fdk_voxels(sino, (n, n, n), (s, s, s), (sv, su), ang, P, sid, sdd, rng_ / nviews,
                             ii.ravel(), jj.ravel(), np.full(ii.size, kz), kind=oracle.RAMLAK, redund=redund,
                             scan_range=rng_)
    img = vals.reshape(n, n)
    X, Y = np.meshgrid(x, x)
    zc = (kz - 0.5 * (n - 1)) * s - c[2]
    rr = np.sqrt(r * r - zc * zc)
    dist = np.hypot(X - c[0], Y - c[1])
    assert np.max(np.abs(img[dist < 0.8 * rr] - mu)) < 0.02 * mu
    assert abs(np.mean(img[dist > 1.3 * rr])) < 0.02 * mu


def test_fdk_voxels_equals_full_fdk():
    rng = np.random.default_rng(17)
    ang = oracle.uniform_angles(10, 2 * np.pi)
    P = oracle.circular_pmats(ang, 60.0, 100.0, (8, 12), (1.5, 1.5))
    y = rng.standard_normal((10, 8, 12))
    full = oracle.fdk(y, (6, 7, 8), (1, 1, 1), (1.5, 1.5), ang, P, 60.0, 100.0, 2 * np.pi / 10,
                      kind=oracle.SHEPP_LOGAN, redund=oracle.REDUND_FULL)
    ii, jj, kk = rng.integers(0, 8, 7), rng.integers(0, 7, 7), rng.integers(0, 6, 7)
    part = oracle.fdk_voxels(y, (6, 7, 8), (1, 1, 1), (1.5, 1.5), ang, P, 60.0, 100.0, 2 * np.pi / 10, ii, jj, kk,
                             kind=oracle.SHEPP_LOGAN, redund=oracle.REDUND_FULL)
    assert np.allclose(part, full[kk, jj, ii], rtol=1e-13, atol=1e-13)


# ----------------------------------------------------------------- TV ---

def test_tv_closed_form_and_gradient():
    eps = 1e-2
    n = 6
    ramp = np.broadcast_to(0.3 * np.arange(n)[None, None, :], (n, n, n)).copy()
    expected = (n - 1) * n * n * (np.sqrt(0.09 + eps * eps) - eps)
    assert abs(oracle.tv_value(ramp, eps) - expected) < 1e-12
    rng = np.random.default_rng(18)
    x = rng.standard_normal((4, 5, 6))
    g = oracle.tv_grad(x, eps)
    h = 1e-6
    for _ in range(20):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (oracle.tv_value(xp, eps) - oracle.tv_value(xm, eps)) / (2 * h)
        assert abs(fd - g[idx]) < 1e-6


def test_tv_solver_zero_lambda_reaches_least_squares():
    """With lambda = 0 the iteration of Eq. 7 minimises |A x - p|^2: on an
    8x8 parallel problem it reaches the least-squares optimum of the explicit
    system matrix (numpy lstsq)."""
    n, nu = 8, 13
    ang = oracle.uniform_angles(12, np.pi)
    fwd = lambda v: oracle.fp_par2d(v, (1.0, 1.0), nu, 1.0, ang)
    adj = lambda s: oracle.fpT_par2d(s, (n, n), (1.0, 1.0), 1.0, ang)
    A = np.stack([fwd(np.eye(n * n)[i].reshape(n, n)).ravel() for i in range(n * n)], axis=1)
    rng = np.random.default_rng(19)
    p = fwd(rng.uniform(0, 1, (n, n))) + 0.01 * rng.standard_normal((12, nu))
    x_ls = np.linalg.lstsq(A, p.ravel(), rcond=None)[0]
    j_ls = float(np.sum((A @ x_ls - p.ravel()) ** 2))
    L = oracle.lipschitz(fwd, adj, (n, n))
    assert abs(L - 2 * np.linalg.eigvalsh(A.T @ A).max()) < 1e-6 * L
    x, obj = oracle.tv_solve(p, fwd, adj, 0.0, 1e-3, 400, L)
    assert obj[-1] <= obj[0]
    assert abs(obj[-1] - j_ls) < 1e-6 * obj[0]


def test_tv_solver_is_first_order_optimal_with_lambda():
    n, nu = 8, 13
    ang = oracle.uniform_angles(12, np.pi)
    fwd = lambda v: oracle.fp_par2d(v, (1.0, 1.0), nu, 1.0, ang)
    adj = lambda s: oracle.fpT_par2d(s, (n, n), (1.0, 1.0), 1.0, ang)
    rng = np.random.default_rng(20)
    truth = np.zeros((n, n))
    truth[2:6, 3:7] = 1.0
    p = fwd(truth) + 0.05 * rng.standard_normal((12, nu))
    L = oracle.lipschitz(fwd, adj, (n, n))
    lam, eps = 0.5, 1e-2
    x, obj = oracle.tv_solve(p, fwd, adj, lam, eps, 600, L)
    g = 2 * adj(fwd(x) - p) + lam * oracle.tv_grad(x, eps)
    g0 = 2 * adj(-p)
    assert np.linalg.norm(g) < 1e-4 * np.linalg.norm(g0)
    # the TV term lowers the error against the piecewise-constant truth vs plain least squares
    x0, _ = oracle.tv_solve(p, fwd, adj, 0.0, eps, 600, L)
    assert np.linalg.norm(x - truth) < np.linalg.norm(x0 - truth)


# --------------------------------------------------------- CNN reference ---

def test_cnn_reference_conv_pins():
    """The reference convolution against closed forms: a centre-tap identity
    kernel copies the input; a kernel of ones sums the 3x3x3 neighbourhood
    (zero padding); wgrad is the adjoint of the map w -> conv(x, w)."""
    import torch
    from oracle import cnn as R
    rng = np.random.default_rng(21)
    x = torch.from_numpy(rng.standard_normal((1, 4, 5, 6, 2)))
    w = torch.zeros(27, 2, 2, dtype=torch.float64)
    w[13, 0, 0] = w[13, 1, 1] = 1.0  # tap (1,1,1) is the centre
    assert torch.allclose(R.conv3d(x, w), x)
    ones = torch.ones(27, 1, 1, dtype=torch.float64)
    s = torch.from_numpy(rng.standard_normal((1, 4, 5, 6, 1)))
    box = R.conv3d(s, ones)[0, 1, 2, 3, 0]
    assert abs(float(box) - float(s[0, 0:3, 1:4, 2:5, 0].sum())) < 1e-12
    corner = R.conv3d(s, ones)[0, 0, 0, 0, 0]
    assert abs(float(corner) - float(s[0, 0:2, 0:2, 0:2, 0].sum())) < 1e-12
    # tap convention: a kernel with only tap (dz,dy,dx) = (2,1,1) reads x[z+1]
    w1 = torch.zeros(27, 1, 1, dtype=torch.float64)
    w1[(2 * 3 + 1) * 3 + 1] = 1.0
    y = R.conv3d(s, w1)
    assert torch.allclose(y[:, :-1], s[:, 1:]) and torch.all(y[:, -1] == 0)
    dy = torch.from_numpy(rng.standard_normal((1, 4, 5, 6, 3)))
    wr = torch.from_numpy(rng.standard_normal((27, 3, 2)))
    lhs = float((R.conv3d(x, wr) * dy).sum())
    rhs = float((R.conv3d_wgrad(x, dy) * wr).sum())
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_cnn_reference_network_pins():
    """Zero last layer: the residual network returns its input exactly;
    pooling / upsampling are the mean / copy they are defined to be."""
    import torch
    from oracle import cnn as R
    rng = np.random.default_rng(22)
    params = {n: (torch.from_numpy(rng.standard_normal((27, co, ci)) * 0.1), torch.zeros(co, dtype=torch.float64))
              for n, ci, co in R.LAYERS}
    params["c11"] = (torch.zeros(27, 1, 16, dtype=torch.float64), torch.zeros(1, dtype=torch.float64))
    x = torch.from_numpy(rng.standard_normal((1, 16, 16, 16)))
    assert torch.equal(R.network(x, params), x)
    v = torch.from_numpy(rng.standard_normal((1, 4, 4, 4, 3)))
    assert torch.allclose(R.avgpool2(v)[0, 1, 0, 1], v[0, 2:4, 0:2, 2:4].mean(dim=(0, 1, 2)))
    assert torch.equal(R.upsample2(v)[0, 5, 2, 7], v[0, 2, 1, 3])
