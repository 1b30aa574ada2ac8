"""The C-ABI library builds, loads and exports every entry point of
include/pyro.h, and its host-side validation rejects bad arguments before
touching the GPU (runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1904_13342_gb300 import binding as B
from paper_1904_13342_gb300.geometry import CGeom2D, CGeom3D, ConeGeometry3D, FanGeometry2D, ParallelGeometry2D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pyro.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"PYRO_API\s+[\w\s\*]+?\b(pyro_\w+)\s*\(", src)))


def test_header_declares_the_core_calls():
    names = declared_symbols()
    for n in ("pyro_fp_par2d", "pyro_fp_fan2d", "pyro_fp_cone3d", "pyro_bp_par2d", "pyro_bp_fan2d",
              "pyro_bp_cone3d", "pyro_fdk"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.lib()._name)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert B.version().startswith("pyro-gb300")


def test_library_exports_nothing_else():
    out = os.popen(f"nm -D --defined-only {B.library_path()}").read()
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported and exported <= set(declared_symbols()) | {"_init", "_fini"}, exported - set(declared_symbols())


def fake_ptr():
    # 16-byte aligned, never dereferenced: every case below fails validation first
    return ctypes.c_void_p(0x10000)


def call_fp_par(g):
    return B.lib().pyro_fp_par2d(fake_ptr(), fake_ptr(), 1, ctypes.byref(g), 0, None)


def test_validation_rejects_bad_geometry():
    L = B.lib()
    good = ParallelGeometry2D((8, 8), (1.0, 1.0), 9, 1.0, 4).to_c()
    bad = CGeom2D.from_buffer_copy(good)
    bad.nx = 0
    assert call_fp_par(bad) == 1
    assert "positive" in L.pyro_last_error().decode()
    bad = CGeom2D.from_buffer_copy(good)
    bad.su = -1.0
    assert call_fp_par(bad) == 1
    bad = CGeom2D.from_buffer_copy(good)
    bad.su = float("nan")
    assert call_fp_par(bad) == 1
    bad = CGeom2D.from_buffer_copy(good)
    bad.range = 0.0
    assert call_fp_par(bad) == 1
    assert L.pyro_fp_par2d(None, fake_ptr(), 1, ctypes.byref(good), 0, None) == 1
    assert L.pyro_fp_par2d(ctypes.c_void_p(0x10004), fake_ptr(), 1, ctypes.byref(good), 0, None) == 1
    assert "aligned" in L.pyro_last_error().decode()
    assert L.pyro_fp_par2d(fake_ptr(), fake_ptr(), 1, ctypes.byref(good), 7, None) == 1
    assert L.pyro_fp_par2d(fake_ptr(), fake_ptr(), 1, None, 0, None) == 1
    # source inside the image support
    fan = FanGeometry2D((64, 64), (1.0, 1.0), 9, 1.0, 4, 2 * np.pi, sid=40.0, sdd=80.0).to_c()
    assert L.pyro_fp_fan2d(fake_ptr(), fake_ptr(), 1, ctypes.byref(fan), 0, None) == 1
    assert "outside" in L.pyro_last_error().decode()
    fan = FanGeometry2D((8, 8), (1.0, 1.0), 9, 1.0, 4, 2 * np.pi, sid=90.0, sdd=80.0).to_c()
    assert L.pyro_fp_fan2d(fake_ptr(), fake_ptr(), 1, ctypes.byref(fan), 0, None) == 1


def test_validation_rejects_bad_cone_geometry_and_modes():
    L = B.lib()
    g = ConeGeometry3D((8, 8, 8), (1, 1, 1), (6, 7), (1.5, 1.5), 5, 2 * np.pi, 100.0, 160.0)
    P = np.zeros((5, 3, 4))
    g.projection_matrices = P
    assert L.pyro_fp_cone3d(fake_ptr(), fake_ptr(), 1, ctypes.byref(g.to_c()), 0, None) == 1
    P = np.random.default_rng(0).standard_normal((5, 3, 4))
    P[:, 2, 3] = 1e-3  # source next to the iso-centre
    g.projection_matrices = P
    assert L.pyro_fp_cone3d(fake_ptr(), fake_ptr(), 1, ctypes.byref(g.to_c()), 0, None) == 1
    g.projection_matrices = None
    cg = g.to_c()
    # adjoint only in FP32
    assert L.pyro_fpT_cone3d(fake_ptr(), fake_ptr(), 1, ctypes.byref(cg), 1, None) == 4
    assert L.pyro_bpT_cone3d(fake_ptr(), fake_ptr(), 1, ctypes.byref(cg), 0, 1.0, 2, None) == 4
    # unknown weight / filter / redundancy
    assert L.pyro_bp_cone3d(fake_ptr(), fake_ptr(), 1, ctypes.byref(cg), 9, 1.0, 0, None) == 1
    assert L.pyro_filter_rows(fake_ptr(), fake_ptr(), 4, 16, 1.0, 9, None, 0, None) == 1
    assert L.pyro_filter_rows(fake_ptr(), fake_ptr(), 4, 16, 1.0, 3, None, 0, None) == 1
    assert L.pyro_filter_rows(fake_ptr(), fake_ptr(), 4, 5000, 1.0, 0, None, 0, None) == 1
    assert L.pyro_weights3d(fake_ptr(), 1, ctypes.byref(cg), 1, 7, 0, None) == 1
    # FDK with a missing or small workspace
    need = L.pyro_fdk_workspace_bytes(ctypes.byref(cg), 2)
    assert need == 4 * 2 * 5 * 6 * 7
    assert L.pyro_fdk(fake_ptr(), fake_ptr(), 2, ctypes.byref(cg), 0, None, 1, None, 0, 0, None) == 5
    assert L.pyro_fdk(fake_ptr(), fake_ptr(), 2, ctypes.byref(cg), 0, None, 1, fake_ptr(), need - 4, 0, None) == 5
    assert "workspace" in L.pyro_last_error().decode()


def test_pad_length():
    assert [B.pyro_filter_pad_length(n) for n in (1, 64, 65, 183, 620, 1240)] == [2, 128, 256, 512, 2048, 4096]


def test_tensor_wrappers_refuse_cpu_tensors():
    import torch

    g = ParallelGeometry2D((8, 8), (1.0, 1.0), 9, 1.0, 4)
    with pytest.raises(TypeError):
        B.pyro_fp_par2d(torch.zeros(8, 8), g)


def test_missing_library_fails_loudly(monkeypatch):
    """No library and no way to build it: the binding raises (there is no
    CPU fallback to fall into)."""
    monkeypatch.setattr(B, "_lib", None)

    def no_compiler():
        raise RuntimeError("nvcc not found")

    monkeypatch.setattr(B._build, "build", no_compiler)
    with pytest.raises(RuntimeError):
        B.lib()
    with pytest.raises(RuntimeError):
        B.pyro_filter_pad_length(100)


def test_validation_of_scan_weights_staged_2d_and_textures():
    """Host-side checks of the scan-range weights, the staged 2D calls and the
    texture calls fail before any GPU work."""
    L = B.lib()
    fan = FanGeometry2D((8, 8), (1.0, 1.0), 9, 1.0, 4, 7.0, 300.0, 500.0).to_c()  # range above 2 pi
    assert L.pyro_weights2d(fake_ptr(), 1, ctypes.byref(fan), 1, B.REDUND_SCAN, B.PYRO_F32, None) == 1
    assert "2 pi" in L.pyro_last_error().decode()
    assert L.pyro_weights2d(fake_ptr(), 1, ctypes.byref(fan), 1, 9, B.PYRO_F32, None) == 1  # unknown mode
    par = ParallelGeometry2D((8, 8), (1.0, 1.0), 9, 1.0, 4).to_c()
    need = L.pyro_fp2d_workspace_bytes(ctypes.byref(par), 2, B.PYRO_F32)
    assert need == 2 * 8 * 8 * 4
    for fn in (L.pyro_fp_par2d_ws, L.pyro_fpT_par2d_ws):
        assert fn(fake_ptr(), fake_ptr(), 2, ctypes.byref(par), fake_ptr(), need - 16, B.PYRO_F32, None) == 5
        assert fn(fake_ptr(), fake_ptr(), 2, ctypes.byref(par), None, need, B.PYRO_F32, None) == 1
    h = ctypes.c_void_p()
    assert L.pyro_texture_volume_create(0, 4, 4, B.PYRO_F32, ctypes.byref(h)) == 1 and not h.value
    assert L.pyro_texture_sinogram_create(4, 4, -1, B.PYRO_F32, ctypes.byref(h)) == 1 and not h.value
    assert L.pyro_texture_volume_create(4, 4, 4, B.PYRO_BF16, ctypes.byref(h)) == 4 and not h.value
    assert L.pyro_texture_destroy(None) == 0
    assert L.pyro_texture_upload(None, fake_ptr(), None) == 1
    cone = ConeGeometry3D((4, 4, 4), (1.0, 1.0, 1.0), (6, 6), (1.0, 1.0), 3, 6.0, 300.0, 500.0).to_c()
    assert L.pyro_fp_cone3d_tex(None, fake_ptr(), ctypes.byref(cone), B.PYRO_F32, None) == 1
    assert L.pyro_bp_cone3d_tex(None, fake_ptr(), ctypes.byref(cone), 2, 1.0, B.PYRO_F32, None) == 1
