"""pyro_fdk_noalloc: FDK for callers that cannot allocate device memory.

Such callers (for instance a reconstruction stage that is handed only the
projection and volume buffers by an acquisition pipeline, or a plug-in whose
host application owns all device memory and forbids allocating more) cannot
supply the workspace pyro_fdk asks for; this entry point uses the library's
static 64 MiB scratch array instead.  The test calls it through the C ABI and
compares it with pyro_fdk (caller workspace) and with the FP64 oracle's FDK
on two calls in a row with different inputs, so a stale scratch array from
the first call would show.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1904_13342_gb300 import binding as B
from paper_1904_13342_gb300 import phantoms as ph
from paper_1904_13342_gb300.geometry import ConeGeometry3D, short_scan_range

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
TOL = 1e-5  # the FP32 parity tolerance of the other tests


def rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def geometry():
    nv, nu, s = 96, 128, 1.0
    return ConeGeometry3D((64, 64, 64), (1.0, 1.0, 1.0), (nv, nu), (s, s), 90, short_scan_range(nu * s, 700.0),
                          400.0, 700.0)


def call_noalloc(sino, g, kind, redund):
    """Direct C-ABI call: only the input and output buffers are passed."""
    out = torch.empty((sino.shape[0], *g.volume_shape), device=DEV, dtype=sino.dtype)
    cg = g.to_c()
    st = B.lib().pyro_fdk_noalloc(ctypes.c_void_p(sino.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  sino.shape[0], ctypes.byref(cg), kind, None, redund, B.PYRO_F32,
                                  ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream))
    assert st == 0, B.lib().pyro_last_error().decode()
    return out


def oracle_fdk(y, g, kind, redund):
    ang = g.view_angles()
    P = oracle.circular_pmats(ang, g.sid, g.sdd, g.detector_shape, g.detector_spacing)
    return np.stack([oracle.fdk(s, g.volume_shape, g.volume_spacing, g.detector_spacing, ang, P, g.sid, g.sdd,
                                g.angular_range / g.number_of_projections, kind, redund)
                     for s in y.double().cpu().numpy()])


def test_noalloc_matches_fdk_on_two_calls_in_a_row():
    g = geometry()
    for seed, kind, redund in ((1, B.SHEPP_LOGAN, B.REDUND_PARKER), (2, B.RAMLAK, B.REDUND_PARKER)):
        y = torch.from_numpy(ph.random_sinogram((2, *g.sinogram_shape), seed, smooth=3)).float().to(DEV)
        y += 5.0 * seed  # make the two inputs differ clearly
        got = call_noalloc(y, g, kind, redund)
        ref = B.pyro_fdk(y, g, kind=kind, redund=redund)
        torch.cuda.synchronize()
        assert rel(got, ref) < TOL
        exact = oracle_fdk(y, g, kind, redund)
        err = np.linalg.norm(got.double().cpu().numpy() - exact) / np.linalg.norm(exact)
        assert err < TOL


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    g = geometry()
    cg = g.to_c()
    need = B.lib().pyro_fdk_workspace_bytes(ctypes.byref(cg), 1)
    batch = (B.NOALLOC_SCRATCH_BYTES // need) + 1
    st = B.lib().pyro_fdk_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), batch, ctypes.byref(cg), B.SHEPP_LOGAN,
                                  None, B.REDUND_PARKER, B.PYRO_F32, None)
    assert st == 5  # PYRO_EWORKSPACE, nothing enqueued
    assert "64 MiB" in B.lib().pyro_last_error().decode()
