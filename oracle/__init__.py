"""FP64 CPU oracle for the PYRO-NN known-operator CT layers.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the product library
never imports, links or runs it.  It shares no code with the CUDA path.

The arithmetic lives in ``pyro_oracle.c`` (plain double-precision loops that
restate the paper's operators); this module only compiles it with gcc and
marshals numpy arrays in and out.  Every function takes the same plain
geometry description as the product API (shapes, spacings in mm, angle list
in radians, SID/SDD in mm, ray sampling step in mm) and returns float64
arrays.

Parity unpinned: none of the paper's own numerical outputs (its figures are
placeholders and it ships no data), so every pin below comes from closed
forms, invariants and brute force (see ``tests/test_oracle_pins.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pyro_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_I = ctypes.c_int
_L = ctypes.c_long
_PD = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, OpenMP, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "oracle_circular_pmats": [_I, _PD, _D, _D, _I, _I, _D, _D, _PD],
                "oracle_fp_par2d": [_PD, _I, _I, _D, _D, _I, _D, _I, _PD, _D, _PD],
                "oracle_fp_fan2d": [_PD, _I, _I, _D, _D, _I, _D, _I, _PD, _D, _D, _D, _PD],
                "oracle_fpT_par2d": [_PD, _I, _I, _D, _D, _I, _D, _I, _PD, _D, _PD],
                "oracle_fpT_fan2d": [_PD, _I, _I, _D, _D, _I, _D, _I, _PD, _D, _D, _D, _PD],
                "oracle_fp_cone3d": [_PD, _I, _I, _I, _D, _D, _D, _I, _I, _I, _PD, _D, _PD],
                "oracle_fp_cone3d_rays": [_PD, _I, _I, _I, _D, _D, _D, _PD, _D, _I, _PI, _PI, _PI, _PD],
                "oracle_fpT_cone3d": [_PD, _I, _I, _I, _D, _D, _D, _I, _I, _I, _PD, _D, _PD],
                "oracle_fpT_cone3d_voxels": [_PD, _I, _I, _I, _D, _D, _D, _I, _I, _I, _PD, _D, _I, _PI, _PI, _PI,
                                             _PD],
                "oracle_bp_par2d": [_PD, _I, _I, _D, _D, _I, _D, _I, _PD, _D, _PD],
                "oracle_bp_fan2d": [_PD, _I, _I, _D, _D, _I, _D, _I, _PD, _D, _D, _I, _D, _PD],
                "oracle_bpT_par2d": [_PD, _I, _I, _D, _D, _I, _D, _I, _PD, _D, _PD],
                "oracle_bpT_fan2d": [_PD, _I, _I, _D, _D, _I, _D, _I, _PD, _D, _D, _I, _D, _PD],
                "oracle_bp_cone3d": [_PD, _I, _I, _I, _D, _D, _D, _I, _I, _I, _PD, _D, _I, _D, _PD],
                "oracle_bp_cone3d_voxels": [_PD, _I, _I, _I, _D, _D, _D, _I, _I, _I, _PD, _D, _I, _D, _I,
                                            _PI, _PI, _PI, _PD],
                "oracle_bpT_cone3d": [_PD, _I, _I, _I, _D, _D, _D, _I, _I, _I, _PD, _D, _I, _D, _PD],
                "oracle_parker_weight": [_D, _D, _D],
                "oracle_scan_weight": [_D, _D, _D],
                "oracle_weights": [_PD, _I, _I, _I, _D, _D, _PD, _D, _I, _I, _D],
                "oracle_pad_length": [_I],
                "oracle_filter_rows": [_PD, _PD, _L, _I, _D, _I, _PD],
                "oracle_filter_grad_K": [_PD, _PD, _L, _I, _PD],
                "oracle_fbp_par2d": [_PD, _I, _I, _D, _D, _I, _D, _I, _PD, _I, _PD, _PD],
                "oracle_fbp_fan2d": [_PD, _I, _I, _D, _D, _I, _D, _I, _PD, _D, _D, _D, _I, _PD, _I, _D, _PD],
                "oracle_fdk": [_PD, _I, _I, _I, _D, _D, _D, _I, _I, _D, _D, _I, _PD, _PD, _D, _D, _D, _I, _PD,
                               _I, _D, _PD],
                "oracle_fdk_voxels": [_PD, _I, _I, _I, _D, _D, _D, _I, _I, _D, _D, _I, _PD, _PD, _D, _D, _D, _I,
                                      _PD, _I, _D, _I, _PI, _PI, _PI, _PD],
                "oracle_tv_value": [_PD, _I, _I, _I, _D],
                "oracle_tv_grad": [_PD, _I, _I, _I, _D, _PD],
                "oracle_num_threads": [],
                "oracle_set_num_threads": [_I],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = None
            lib.oracle_parker_weight.restype = _D
            lib.oracle_scan_weight.restype = _D
            lib.oracle_pad_length.restype = _I
            lib.oracle_tv_value.restype = _D
            lib.oracle_num_threads.restype = _I
            lib.oracle_set_num_threads.restype = _I
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _p(a: np.ndarray):
    if a is None:
        return None
    if a.dtype == np.int32:
        return a.ctypes.data_as(_PI)
    return a.ctypes.data_as(_PD)


# filter kinds and redundancy modes, same numbering as the product API
RAMLAK, RAMP, SHEPP_LOGAN, CUSTOM = 0, 1, 2, 3
REDUND_FULL, REDUND_PARKER, REDUND_NONE, REDUND_SCAN = 0, 1, 2, 3


def uniform_angles(n_views: int, angular_range: float) -> np.ndarray:
    """beta_j = j * range / n_views (no duplicated view on a 360 degree scan)."""
    return np.arange(n_views, dtype=np.float64) * (angular_range / n_views)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> int:
    """OpenMP threads for later oracle calls; returns the previous count."""
    return int(_load().oracle_set_num_threads(int(n)))


def circular_pmats(angles, sid, sdd, det_shape, det_spacing) -> np.ndarray:
    """[n_views, 3, 4] projection matrices of the circular trajectory."""
    nv, nu = det_shape
    sv, su = det_spacing
    ang = _f64(angles)
    out = np.empty((ang.size, 3, 4))
    _load().oracle_circular_pmats(ang.size, _p(ang), sid, sdd, nu, nv, su, sv, _p(out))
    return out


def default_step(spacing) -> float:
    return 0.5 * float(min(spacing))


# ---------------------------------------------------------------- 2D ----
def fp_par2d(img, spacing, nu, su, angles, step=None):
    img = _f64(img)
    ny, nx = img.shape
    sy, sx = spacing
    ang = _f64(angles)
    dt = default_step(spacing) if step is None else step
    out = np.empty((ang.size, nu))
    _load().oracle_fp_par2d(_p(img), nx, ny, sx, sy, nu, su, ang.size, _p(ang), dt, _p(out))
    return out


def fp_fan2d(img, spacing, nu, su, angles, sid, sdd, step=None):
    img = _f64(img)
    ny, nx = img.shape
    sy, sx = spacing
    ang = _f64(angles)
    dt = default_step(spacing) if step is None else step
    out = np.empty((ang.size, nu))
    _load().oracle_fp_fan2d(_p(img), nx, ny, sx, sy, nu, su, ang.size, _p(ang), sid, sdd, dt, _p(out))
    return out


def fpT_par2d(sino, shape, spacing, su, angles, step=None):
    sino = _f64(sino)
    ny, nx = shape
    sy, sx = spacing
    ang = _f64(angles)
    dt = default_step(spacing) if step is None else step
    out = np.empty((ny, nx))
    _load().oracle_fpT_par2d(_p(sino), nx, ny, sx, sy, sino.shape[1], su, ang.size, _p(ang), dt, _p(out))
    return out


def fpT_fan2d(sino, shape, spacing, su, angles, sid, sdd, step=None):
    sino = _f64(sino)
    ny, nx = shape
    sy, sx = spacing
    ang = _f64(angles)
    dt = default_step(spacing) if step is None else step
    out = np.empty((ny, nx))
    _load().oracle_fpT_fan2d(_p(sino), nx, ny, sx, sy, sino.shape[1], su, ang.size, _p(ang), sid, sdd, dt,
                             _p(out))
    return out


def bp_par2d(sino, shape, spacing, su, angles, scale=1.0):
    sino = _f64(sino)
    ny, nx = shape
    sy, sx = spacing
    ang = _f64(angles)
    out = np.empty((ny, nx))
    _load().oracle_bp_par2d(_p(sino), nx, ny, sx, sy, sino.shape[1], su, ang.size, _p(ang), scale, _p(out))
    return out


def bp_fan2d(sino, shape, spacing, su, angles, sid, sdd, weight=0, scale=1.0):
    sino = _f64(sino)
    ny, nx = shape
    sy, sx = spacing
    ang = _f64(angles)
    out = np.empty((ny, nx))
    _load().oracle_bp_fan2d(_p(sino), nx, ny, sx, sy, sino.shape[1], su, ang.size, _p(ang), sid, sdd, weight,
                            scale, _p(out))
    return out


def bpT_par2d(img, nu, su, angles, spacing, scale=1.0):
    img = _f64(img)
    ny, nx = img.shape
    sy, sx = spacing
    ang = _f64(angles)
    out = np.empty((ang.size, nu))
    _load().oracle_bpT_par2d(_p(img), nx, ny, sx, sy, nu, su, ang.size, _p(ang), scale, _p(out))
    return out


def bpT_fan2d(img, nu, su, angles, spacing, sid, sdd, weight=0, scale=1.0):
    img = _f64(img)
    ny, nx = img.shape
    sy, sx = spacing
    ang = _f64(angles)
    out = np.empty((ang.size, nu))
    _load().oracle_bpT_fan2d(_p(img), nx, ny, sx, sy, nu, su, ang.size, _p(ang), sid, sdd, weight, scale,
                             _p(out))
    return out


# ---------------------------------------------------------------- 3D ----
def fp_cone3d(vol, spacing, det_shape, pmats, step=None):
    vol = _f64(vol)
    nz, ny, nx = vol.shape
    sz, sy, sx = spacing
    nv, nu = det_shape
    P = _f64(pmats)
    dt = default_step(spacing) if step is None else step
    out = np.empty((P.shape[0], nv, nu))
    _load().oracle_fp_cone3d(_p(vol), nx, ny, nz, sx, sy, sz, nu, nv, P.shape[0], _p(P), dt, _p(out))
    return out


def fp_cone3d_rays(vol, spacing, pmats, views, ks, ls, step=None):
    vol = _f64(vol)
    nz, ny, nx = vol.shape
    sz, sy, sx = spacing
    P = _f64(pmats)
    v, k, l = _i32(views), _i32(ks), _i32(ls)
    dt = default_step(spacing) if step is None else step
    out = np.empty(v.size)
    _load().oracle_fp_cone3d_rays(_p(vol), nx, ny, nz, sx, sy, sz, _p(P), dt, v.size, _p(v), _p(k), _p(l), _p(out))
    return out


def fpT_cone3d(sino, shape, spacing, pmats, step=None):
    sino = _f64(sino)
    nz, ny, nx = shape
    sz, sy, sx = spacing
    _, nv, nu = sino.shape
    P = _f64(pmats)
    dt = default_step(spacing) if step is None else step
    out = np.empty((nz, ny, nx))
    _load().oracle_fpT_cone3d(_p(sino), nx, ny, nz, sx, sy, sz, nu, nv, P.shape[0], _p(P), dt, _p(out))
    return out


def fpT_cone3d_voxels(sino, shape, spacing, pmats, ii, jj, kk, step=None):
    """The exact adjoint A^T y at the voxels (ii[r], jj[r], kk[r]) only, from
    its definition (the rays and planes whose samples fall in each voxel's
    interpolation support); equal to fpT_cone3d there."""
    sino = _f64(sino)
    nz, ny, nx = shape
    sz, sy, sx = spacing
    nvw, nv, nu = sino.shape
    P = _f64(pmats)
    dt = default_step(spacing) if step is None else step
    i, j, k = _i32(ii), _i32(jj), _i32(kk)
    out = np.empty(i.size)
    _load().oracle_fpT_cone3d_voxels(_p(sino), nx, ny, nz, sx, sy, sz, nu, nv, nvw, _p(P), dt, i.size, _p(i), _p(j),
                                     _p(k), _p(out))
    return out


def bp_cone3d(sino, shape, spacing, pmats, sid, weight=0, scale=1.0):
    sino = _f64(sino)
    nz, ny, nx = shape
    sz, sy, sx = spacing
    _, nv, nu = sino.shape
    P = _f64(pmats)
    out = np.empty((nz, ny, nx))
    _load().oracle_bp_cone3d(_p(sino), nx, ny, nz, sx, sy, sz, nu, nv, P.shape[0], _p(P), sid, weight, scale, _p(out))
    return out


def bp_cone3d_voxels(sino, shape, spacing, pmats, sid, ii, jj, kk, weight=0, scale=1.0):
    sino = _f64(sino)
    nz, ny, nx = shape
    sz, sy, sx = spacing
    _, nv, nu = sino.shape
    P = _f64(pmats)
    i, j, k = _i32(ii), _i32(jj), _i32(kk)
    out = np.empty(i.size)
    _load().oracle_bp_cone3d_voxels(_p(sino), nx, ny, nz, sx, sy, sz, nu, nv, P.shape[0], _p(P), sid, weight, scale,
                                    i.size, _p(i), _p(j), _p(k), _p(out))
    return out


def bpT_cone3d(vol, det_shape, spacing, pmats, sid, weight=0, scale=1.0):
    vol = _f64(vol)
    nz, ny, nx = vol.shape
    sz, sy, sx = spacing
    nv, nu = det_shape
    P = _f64(pmats)
    out = np.empty((P.shape[0], nv, nu))
    _load().oracle_bpT_cone3d(_p(vol), nx, ny, nz, sx, sy, sz, nu, nv, P.shape[0], _p(P), sid, weight, scale, _p(out))
    return out


# ------------------------------------------------- weights, filters, FBP --
def parker_weight(beta, gamma, delta) -> float:
    return float(_load().oracle_parker_weight(beta, gamma, delta))


def scan_weight(beta, gamma, scan_range) -> float:
    """Redundancy weight of ray (beta, gamma) in a scan over [0, scan_range]."""
    return float(_load().oracle_scan_weight(beta, gamma, scan_range))


def _scan(redund, scan_range):
    if redund == REDUND_SCAN and not (scan_range and 0.0 < scan_range <= 2 * np.pi + 1e-12):
        raise ValueError("REDUND_SCAN needs 0 < scan_range <= 2 pi")
    return float(scan_range or 0.0)


def weights(sino, det_spacing, angles, sdd, cosine=True, redund=REDUND_NONE, scan_range=None):
    """W_red W_cos p for a [V, Nu] (fan) or [V, Nv, Nu] (cone) sinogram;
    scan_range is the scan's angular range for REDUND_SCAN."""
    s = _f64(sino).copy()
    if s.ndim == 2:
        nvw, nu = s.shape
        nv = 1
        su, sv = det_spacing, 0.0
    else:
        nvw, nv, nu = s.shape
        sv, su = det_spacing
    ang = _f64(angles)
    _load().oracle_weights(_p(s), nvw, nv, nu, su, sv, _p(ang), sdd, int(bool(cosine)), redund,
                           _scan(redund, scan_range))
    return s


def pad_length(nu: int) -> int:
    return int(_load().oracle_pad_length(nu))


def filter_rows(rows, tau, kind=RAMLAK, K=None):
    r = _f64(rows)
    shp = r.shape
    nu = shp[-1]
    flat = r.reshape(-1, nu)
    out = np.empty_like(flat)
    Kc = None if K is None else _f64(K)
    _load().oracle_filter_rows(_p(flat), _p(out), flat.shape[0], nu, tau, kind, _p(Kc))
    return out.reshape(shp)


def filter_grad_K(p, g):
    p = _f64(p)
    nu = p.shape[-1]
    pf = p.reshape(-1, nu)
    gf = _f64(g).reshape(-1, nu)
    out = np.empty(pad_length(nu) // 2 + 1)
    _load().oracle_filter_grad_K(_p(pf), _p(gf), pf.shape[0], nu, _p(out))
    return out


def fbp_par2d(sino, shape, spacing, su, angles, kind=RAMLAK, K=None):
    sino = _f64(sino)
    ny, nx = shape
    sy, sx = spacing
    ang = _f64(angles)
    Kc = None if K is None else _f64(K)
    out = np.empty((ny, nx))
    _load().oracle_fbp_par2d(_p(sino), nx, ny, sx, sy, sino.shape[1], su, ang.size, _p(ang), kind, _p(Kc), _p(out))
    return out


def fbp_fan2d(sino, shape, spacing, su, angles, sid, sdd, dbeta, kind=RAMLAK, redund=REDUND_FULL, K=None,
              scan_range=None):
    sino = _f64(sino)
    ny, nx = shape
    sy, sx = spacing
    ang = _f64(angles)
    Kc = None if K is None else _f64(K)
    out = np.empty((ny, nx))
    _load().oracle_fbp_fan2d(_p(sino), nx, ny, sx, sy, sino.shape[1], su, ang.size, _p(ang), dbeta, sid, sdd, kind,
                             _p(Kc), redund, _scan(redund, scan_range), _p(out))
    return out


def fdk(sino, shape, spacing, det_spacing, angles, pmats, sid, sdd, dbeta, kind=SHEPP_LOGAN, redund=REDUND_PARKER,
        K=None, scan_range=None):
    sino = _f64(sino)
    nz, ny, nx = shape
    sz, sy, sx = spacing
    _, nv, nu = sino.shape
    sv, su = det_spacing
    ang = _f64(angles)
    P = _f64(pmats)
    Kc = None if K is None else _f64(K)
    out = np.empty((nz, ny, nx))
    _load().oracle_fdk(_p(sino), nx, ny, nz, sx, sy, sz, nu, nv, su, sv, ang.size, _p(P), _p(ang), dbeta, sid, sdd,
                       kind, _p(Kc), redund, _scan(redund, scan_range), _p(out))
    return out


def fdk_voxels(sino, shape, spacing, det_spacing, angles, pmats, sid, sdd, dbeta, ii, jj, kk, kind=SHEPP_LOGAN,
               redund=REDUND_PARKER, K=None, scan_range=None):
    sino = _f64(sino)
    nz, ny, nx = shape
    sz, sy, sx = spacing
    _, nv, nu = sino.shape
    sv, su = det_spacing
    ang = _f64(angles)
    P = _f64(pmats)
    Kc = None if K is None else _f64(K)
    i, j, k = _i32(ii), _i32(jj), _i32(kk)
    out = np.empty(i.size)
    _load().oracle_fdk_voxels(_p(sino), nx, ny, nz, sx, sy, sz, nu, nv, su, sv, ang.size, _p(P), _p(ang), dbeta, sid,
                              sdd, kind, _p(Kc), redund, _scan(redund, scan_range), i.size, _p(i), _p(j), _p(k),
                              _p(out))
    return out


def tv_value(x, eps) -> float:
    x = _f64(x)
    if x.ndim == 2:
        x = x[None]
    nz, ny, nx = x.shape
    return float(_load().oracle_tv_value(_p(x), nx, ny, nz, eps))


def tv_grad(x, eps):
    x = _f64(x)
    shp = x.shape
    if x.ndim == 2:
        x = x[None]
    nz, ny, nx = x.shape
    out = np.empty_like(x)
    _load().oracle_tv_grad(_p(x), nx, ny, nz, eps, _p(out))
    return out.reshape(shp)


# ------------------------------------------------------ iterative TV (Eq. 7) --
def lipschitz(fwd, adj, shape, iters=20, seed=0) -> float:
    """Largest eigenvalue of 2 A^T A by power iteration (FP64)."""
    v = np.random.default_rng(seed).uniform(size=shape)
    lam = 0.0
    for _ in range(iters):
        w = adj(fwd(v))
        lam = np.linalg.norm(w) / np.linalg.norm(v)
        v = w / np.linalg.norm(w)
    return 2.0 * lam


def tv_solve(p, fwd, adj, lam, eps, n_iter, L_est, clamp=10.0, x0=None):
    """Gradient descent with Barzilai-Borwein steps on J(x) = |A x - p|^2 +
    lam TV(x) (Eq. 7), from x = 0:
      g_k = 2 A^T (A x_k - p) + lam grad TV(x_k),
      alpha_0 = 1/L_est, alpha_k = (s.s)/(s.dy) clamped to [0, clamp/L_est],
      x_{k+1} = x_k - alpha_k g_k.
    Returns (x, objective per iterate including the last)."""
    p = _f64(p)
    x = np.zeros_like(adj(p)) if x0 is None else _f64(x0).copy()
    x_prev = g_prev = None
    obj = []
    for k in range(n_iter):
        r = fwd(x) - p
        g = 2.0 * adj(r) + lam * tv_grad(x, eps)
        obj.append(float(np.sum(r * r)) + lam * tv_value(x, eps))
        if k == 0:
            alpha = 1.0 / L_est
        else:
            s, dy = x - x_prev, g - g_prev
            sy = float(np.sum(s * dy))
            alpha = float(np.sum(s * s)) / sy if sy > 0 else 1.0 / L_est
            alpha = min(max(alpha, 0.0), clamp / L_est)
        x_prev, g_prev = x, g
        x = x - alpha * g
    r = fwd(x) - p
    obj.append(float(np.sum(r * r)) + lam * tv_value(x, eps))
    return x, obj
