"""Thin ctypes binding of the C ABI (include/pyro.h), same names.

Argument marshalling only: every step runs in the CUDA library.  PyTorch
provides the device memory (outputs are allocated with ``torch.empty`` on
the input's device) and the stream (the current CUDA stream).  Tensors must
be CUDA, contiguous, float32 / float16 / bfloat16; there is no CPU path and
a missing library is an error, never a fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import torch

from . import build as _build
from .geometry import CGeom2D, CGeom3D, ConeGeometry3D, Geometry2D

_lock = threading.Lock()
_lib = None

PYRO_F32, PYRO_F16, PYRO_BF16 = 0, 1, 2
W_NONE, W_INV_L, W_INV_L2 = 0, 1, 2
RAMLAK, RAMP, SHEPP_LOGAN, FILTER_CUSTOM = 0, 1, 2, 3
REDUND_FULL, REDUND_PARKER, REDUND_NONE, REDUND_SCAN = 0, 1, 2, 3

_DTYPES = {torch.float32: PYRO_F32, torch.float16: PYRO_F16, torch.bfloat16: PYRO_BF16}
_STATUS = {1: "EINVAL", 2: "ECUDA", 3: "ETIMEOUT", 4: "EUNSUPPORTED", 5: "EWORKSPACE"}


class PyroError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"pyro {_STATUS.get(status, status)}: {msg}")
        self.status = status


_VP = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_long
_F = ctypes.c_float
_D = ctypes.c_double
_SZ = ctypes.c_size_t
_G2 = ctypes.POINTER(CGeom2D)
_G3 = ctypes.POINTER(CGeom3D)

_SIGS = {
    "pyro_fp_par2d": [_VP, _VP, _I, _G2, _I, _VP],
    "pyro_fp_fan2d": [_VP, _VP, _I, _G2, _I, _VP],
    "pyro_fp_cone3d": [_VP, _VP, _I, _G3, _I, _VP],
    "pyro_fp_cone3d_workspace_bytes": [_G3, _I],
    "pyro_fp_cone3d_ws": [_VP, _VP, _I, _G3, _VP, _SZ, _I, _VP],
    "pyro_fp_cone3d_ws_storage": [_VP, _VP, _I, _G3, _VP, _SZ, _I, _I, _VP],
    "pyro_fpT_par2d": [_VP, _VP, _I, _G2, _I, _VP],
    "pyro_fpT_fan2d": [_VP, _VP, _I, _G2, _I, _VP],
    "pyro_fpT_cone3d": [_VP, _VP, _I, _G3, _I, _VP],
    "pyro_fpT_cone3d_workspace_bytes": [_G3],
    "pyro_fp2d_workspace_bytes": [_G2, _I, _I],
    "pyro_fp_par2d_ws": [_VP, _VP, _I, _G2, _VP, _SZ, _I, _VP],
    "pyro_fp_fan2d_ws": [_VP, _VP, _I, _G2, _VP, _SZ, _I, _VP],
    "pyro_texture_volume_create": [_I, _I, _I, _I, ctypes.POINTER(_VP)],
    "pyro_texture_sinogram_create": [_I, _I, _I, _I, ctypes.POINTER(_VP)],
    "pyro_texture_upload": [_VP, _VP, _VP],
    "pyro_texture_destroy": [_VP],
    "pyro_fp_cone3d_tex": [_VP, _VP, _G3, _I, _VP],
    "pyro_bp_cone3d_tex": [_VP, _VP, _G3, _I, _F, _I, _VP],
    "pyro_fpT_par2d_ws": [_VP, _VP, _I, _G2, _VP, _SZ, _I, _VP],
    "pyro_fpT_fan2d_ws": [_VP, _VP, _I, _G2, _VP, _SZ, _I, _VP],
    "pyro_cone_projection_matrices": [_G3, _VP],
    "pyro_weights3d_table": [_VP, _I, _G3, _VP, _I, _I, _VP],
    "pyro_bb_dots": [_VP, _VP, _VP, _VP, ctypes.c_long, _VP, _VP],
    "pyro_sync_status": [_VP],
    "pyro_selftest_wait_timeout": [_I, _VP],
    "pyro_probe_gather": [_VP, _SZ, _I, ctypes.c_long, _VP, _VP],
    "pyro_bb_update": [_VP, _VP, _VP, _VP, ctypes.c_long, _VP, ctypes.c_float, ctypes.c_float, _I, _VP, _VP],
    "pyro_redundancy_grad": [_VP, _VP, _VP, _I, _I, _I, _I, _VP],
    "pyro_fpT_cone3d_ws": [_VP, _VP, _I, _G3, _VP, _SZ, _I, _VP],
    "pyro_bp_par2d": [_VP, _VP, _I, _G2, _I, _F, _I, _VP],
    "pyro_bp_fan2d": [_VP, _VP, _I, _G2, _I, _F, _I, _VP],
    "pyro_bp_cone3d": [_VP, _VP, _I, _G3, _I, _F, _I, _VP],
    "pyro_bpT_par2d": [_VP, _VP, _I, _G2, _I, _F, _I, _VP],
    "pyro_bpT_fan2d": [_VP, _VP, _I, _G2, _I, _F, _I, _VP],
    "pyro_bpT_cone3d": [_VP, _VP, _I, _G3, _I, _F, _I, _VP],
    "pyro_weights2d": [_VP, _I, _G2, _I, _I, _I, _VP],
    "pyro_weights3d": [_VP, _I, _G3, _I, _I, _I, _VP],
    "pyro_filter_rows": [_VP, _VP, _L, _I, _D, _I, _VP, _I, _VP],
    "pyro_filter_pad_length": [_I],
    "pyro_filter_spectrum": [_I, _I, _D, ctypes.POINTER(ctypes.c_float)],
    "pyro_filter_grad_K": [_VP, _VP, _VP, _L, _I, _VP],
    "pyro_fdk_workspace_bytes": [_G3, _I],
    "pyro_fdk": [_VP, _VP, _I, _G3, _I, _VP, _I, _VP, _SZ, _I, _VP],
    "pyro_fbp2d_workspace_bytes": [_G2, _I],
    "pyro_fbp_par2d": [_VP, _VP, _I, _G2, _I, _VP, _VP, _SZ, _I, _VP],
    "pyro_fbp_fan2d": [_VP, _VP, _I, _G2, _I, _VP, _I, _VP, _SZ, _I, _VP],
    "pyro_fdk_noalloc": [_VP, _VP, _I, _G3, _I, _VP, _I, _I, _VP],
    "pyro_tv": [_VP, _VP, _VP, _F, _F, _VP, _I, _I, _I, _I, _F, _VP],
    "pyro_conv3d": [_VP, _VP, _VP, _VP, _I, _I, _I, _I, _I, _I, _I, _VP],
    "pyro_conv3d_wgrad": [_VP, _VP, _VP, _I, _I, _I, _I, _I, _I, _VP],
    "pyro_conv3d_flip_weights": [_VP, _VP, _I, _I, _VP],
    "pyro_cnn_op": [_I, _VP, _VP, _VP, _VP, _L, _I, _I, _I, _I, _VP],
    "pyro_cnn_bias_grad": [_VP, _VP, _L, _I, _VP],
    "pyro_cnn_mse": [_VP, _VP, _VP, _VP, _L, _VP],
    "pyro_cnn_adam": [_VP, _VP, _VP, _VP, _VP, _L, _F, _F, _F, _F, _I, _VP],
    "pyro_axpby": [_VP, _VP, _L, _F, _F, _VP],
    "pyro_dot": [_VP, _VP, _L, _VP, _VP],
    "pyro_last_error": [],
    "pyro_version": [],
}


def lib():
    """The loaded libpyro.so (built in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = _I
            L.pyro_last_error.restype = ctypes.c_char_p
            L.pyro_version.restype = ctypes.c_char_p
            L.pyro_fdk_workspace_bytes.restype = _SZ
            L.pyro_fp_cone3d_workspace_bytes.restype = _SZ
            L.pyro_fpT_cone3d_workspace_bytes.restype = _SZ
            L.pyro_fp2d_workspace_bytes.restype = _SZ
            L.pyro_fbp2d_workspace_bytes.restype = _SZ
            _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


def _check(status: int):
    if status != 0:
        raise PyroError(status, lib().pyro_last_error().decode())


def _stream(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _dev(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if t.dtype not in _DTYPES:
        raise TypeError(f"{name} must be float32, float16 or bfloat16, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _batched(t: torch.Tensor, ndim: int, name: str):
    """(tensor viewed with a leading batch dim, whether one was added)."""
    if t.dim() == ndim:
        return t.unsqueeze(0), True
    if t.dim() == ndim + 1:
        return t, False
    raise ValueError(f"{name} must have {ndim} or {ndim + 1} dims, got {tuple(t.shape)}")


def _shape_check(t: torch.Tensor, shape, name):
    if tuple(t.shape[1:]) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape[1:])}, geometry expects {tuple(shape)}")


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _out(t, shape, dtype=None):
    return torch.empty((t.shape[0], *shape), device=t.device, dtype=dtype or t.dtype)


# ------------------------------------------------------------ projectors --
def _fp(fn, vol, g, vshape, sshape):
    v, squeeze = _batched(_dev(vol, "volume"), len(vshape), "volume")
    _shape_check(v, vshape, "volume")
    out = _out(v, sshape)
    cg = g.to_c()
    with torch.cuda.device(v.device):
        _check(fn(_ptr(v), _ptr(out), v.shape[0], ctypes.byref(cg), _DTYPES[v.dtype], _stream(v)))
    return out[0] if squeeze else out


def _fpT(fn, sino, g, vshape, sshape):
    s, squeeze = _batched(_dev(sino, "sinogram"), len(sshape), "sinogram")
    _shape_check(s, sshape, "sinogram")
    out = _out(s, vshape)
    cg = g.to_c()
    with torch.cuda.device(s.device):
        _check(fn(_ptr(s), _ptr(out), s.shape[0], ctypes.byref(cg), _DTYPES[s.dtype], _stream(s)))
    return out[0] if squeeze else out


def _bp(fn, sino, g, weight, scale, vshape, sshape):
    s, squeeze = _batched(_dev(sino, "sinogram"), len(sshape), "sinogram")
    _shape_check(s, sshape, "sinogram")
    out = _out(s, vshape)
    cg = g.to_c()
    with torch.cuda.device(s.device):
        _check(fn(_ptr(s), _ptr(out), s.shape[0], ctypes.byref(cg), int(weight), float(scale), _DTYPES[s.dtype],
                  _stream(s)))
    return out[0] if squeeze else out


def _bpT(fn, vol, g, weight, scale, vshape, sshape):
    v, squeeze = _batched(_dev(vol, "volume"), len(vshape), "volume")
    _shape_check(v, vshape, "volume")
    out = _out(v, sshape)
    cg = g.to_c()
    with torch.cuda.device(v.device):
        _check(fn(_ptr(v), _ptr(out), v.shape[0], ctypes.byref(cg), int(weight), float(scale), _DTYPES[v.dtype],
                  _stream(v)))
    return out[0] if squeeze else out


def pyro_fp_par2d(vol: torch.Tensor, g: Geometry2D) -> torch.Tensor:
    return _fp(lib().pyro_fp_par2d, vol, g, g.volume_shape, g.sinogram_shape)


def pyro_fp_fan2d(vol: torch.Tensor, g: Geometry2D) -> torch.Tensor:
    return _fp(lib().pyro_fp_fan2d, vol, g, g.volume_shape, g.sinogram_shape)


def _fp2d_ws(fn, vol, g, workspace, out):
    v, squeeze = _batched(_dev(vol, "volume"), 2, "volume")
    _shape_check(v, g.volume_shape, "volume")
    cg = g.to_c()
    need = lib().pyro_fp2d_workspace_bytes(ctypes.byref(cg), v.shape[0], _DTYPES[v.dtype])
    if workspace is None:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=v.device)
    o = _out(v, g.sinogram_shape) if out is None else _dev(out, "out")
    with torch.cuda.device(v.device):
        _check(fn(_ptr(v), _ptr(o), v.shape[0], ctypes.byref(cg), _ptr(workspace),
                  workspace.numel() * workspace.element_size(), _DTYPES[v.dtype], _stream(v)))
    return o[0] if squeeze and out is None else o


def pyro_fp_par2d_ws(vol: torch.Tensor, g: Geometry2D, workspace: Optional[torch.Tensor] = None,
                     out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Parallel-beam FP that also reads a transposed copy of the batch kept in
    `workspace` (allocated here when not given)."""
    return _fp2d_ws(lib().pyro_fp_par2d_ws, vol, g, workspace, out)


def pyro_fp_fan2d_ws(vol: torch.Tensor, g: Geometry2D, workspace: Optional[torch.Tensor] = None,
                     out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Fan-beam FP that also reads a transposed copy of the batch."""
    return _fp2d_ws(lib().pyro_fp_fan2d_ws, vol, g, workspace, out)


def _fpT2d_ws(fn, sino, g, workspace):
    s, squeeze = _batched(_dev(sino, "sinogram"), 2, "sinogram")
    _shape_check(s, g.sinogram_shape, "sinogram")
    cg = g.to_c()
    need = lib().pyro_fp2d_workspace_bytes(ctypes.byref(cg), s.shape[0], PYRO_F32)
    if workspace is None:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=s.device)
    out = _out(s, g.volume_shape)
    with torch.cuda.device(s.device):
        _check(fn(_ptr(s), _ptr(out), s.shape[0], ctypes.byref(cg), _ptr(workspace),
                  workspace.numel() * workspace.element_size(), _DTYPES[s.dtype], _stream(s)))
    return out[0] if squeeze else out


def pyro_fpT_par2d_ws(sino: torch.Tensor, g: Geometry2D, workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Exact adjoint of the parallel-beam FP with a transposed accumulator."""
    return _fpT2d_ws(lib().pyro_fpT_par2d_ws, sino, g, workspace)


def pyro_fpT_fan2d_ws(sino: torch.Tensor, g: Geometry2D, workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Exact adjoint of the fan-beam FP with a transposed accumulator."""
    return _fpT2d_ws(lib().pyro_fpT_fan2d_ws, sino, g, workspace)


def fp2d_workspace_bytes(g: Geometry2D, batch: int, dtype=torch.float32) -> int:
    cg = g.to_c()
    return int(lib().pyro_fp2d_workspace_bytes(ctypes.byref(cg), int(batch), _DTYPES[dtype]))


def pyro_fp_cone3d(vol: torch.Tensor, g: ConeGeometry3D) -> torch.Tensor:
    return _fp(lib().pyro_fp_cone3d, vol, g, g.volume_shape, g.sinogram_shape)


def fp_cone3d_workspace_bytes(g: ConeGeometry3D, dtype=torch.float32) -> int:
    """Workspace pyro_fp_cone3d_ws needs for one volume of `dtype`."""
    cg = g.to_c()
    return int(lib().pyro_fp_cone3d_workspace_bytes(ctypes.byref(cg), _DTYPES[dtype]))


class Texture:
    """Data in a CUDA array read with hardware filtering (the paper's
    texture mode): a [nz, ny, nx] volume (`kind="volume"`, trilinear) or a
    [n_views, nv, nu] sinogram (`kind="sinogram"`, one layer per view,
    bilinear).  The library allocates it; `close()` (or garbage collection)
    releases it.  `upload(t)` copies a device tensor of the texture's shape
    and dtype (float32 or float16) into it."""

    def __init__(self, shape, dtype=torch.float32, device=None, kind="volume"):
        self.shape = tuple(int(n) for n in shape)
        self.dtype = dtype
        self.kind = kind
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if kind not in ("volume", "sinogram"):
            raise ValueError("kind must be 'volume' or 'sinogram'")
        if dtype not in (torch.float32, torch.float16):
            raise PyroError(4, "textures hold float32 or float16 values")
        a, b_, c = self.shape
        h = _VP()
        create = lib().pyro_texture_volume_create if kind == "volume" else lib().pyro_texture_sinogram_create
        with torch.cuda.device(self.device):
            _check(create(c, b_, a, _DTYPES[dtype], ctypes.byref(h)))
        self._h = h

    def upload(self, t: torch.Tensor) -> "Texture":
        v = _dev(t, self.kind)
        if tuple(v.shape) != self.shape or v.dtype != self.dtype or v.device != self.device:
            raise ValueError(f"{self.kind} {tuple(v.shape)} {v.dtype} on {v.device} does not match the texture "
                             f"{self.shape} {self.dtype} on {self.device}")
        with torch.cuda.device(v.device):
            _check(lib().pyro_texture_upload(self._h, _ptr(v), _stream(v)))
        return self

    def close(self):
        """Release the array (after the device has finished every queued use of it)."""
        if getattr(self, "_h", None) is not None and self._h.value:
            torch.cuda.synchronize(self.device)
            with torch.cuda.device(self.device):
                _check(lib().pyro_texture_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pyro_fp_cone3d_tex(tex: Texture, g: ConeGeometry3D, dtype=torch.float32,
                       out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Cone-beam FP of a volume texture (hardware trilinear filtering)."""
    if tex.kind != "volume" or tuple(g.volume_shape) != tex.shape:
        raise ValueError(f"geometry volume {tuple(g.volume_shape)} does not match the {tex.kind} texture {tex.shape}")
    o = torch.empty(g.sinogram_shape, dtype=dtype, device=tex.device) if out is None else _dev(out, "out")
    cg = g.to_c()
    with torch.cuda.device(tex.device):
        _check(lib().pyro_fp_cone3d_tex(tex._h, _ptr(o), ctypes.byref(cg), _DTYPES[o.dtype], _stream(o)))
    return o


def pyro_bp_cone3d_tex(tex: Texture, g: ConeGeometry3D, weight=W_INV_L2, scale=1.0, dtype=torch.float32,
                       out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Voxel-driven cone-beam BP of a sinogram texture (hardware bilinear filtering)."""
    if tex.kind != "sinogram" or tuple(g.sinogram_shape) != tex.shape:
        raise ValueError(f"geometry sinogram {tuple(g.sinogram_shape)} does not match the {tex.kind} texture "
                         f"{tex.shape}")
    o = torch.empty(g.volume_shape, dtype=dtype, device=tex.device) if out is None else _dev(out, "out")
    cg = g.to_c()
    with torch.cuda.device(tex.device):
        _check(lib().pyro_bp_cone3d_tex(tex._h, _ptr(o), ctypes.byref(cg), int(weight), float(scale),
                                        _DTYPES[o.dtype], _stream(o)))
    return o


def pyro_fp_cone3d_ws(vol: torch.Tensor, g: ConeGeometry3D, workspace: Optional[torch.Tensor] = None,
                      out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Cone-beam FP from a z-major copy of the volume kept in `workspace`
    (allocated here when not given; one volume of the input dtype)."""
    v, squeeze = _batched(_dev(vol, "volume"), 3, "volume")
    _shape_check(v, g.volume_shape, "volume")
    cg = g.to_c()
    need = lib().pyro_fp_cone3d_workspace_bytes(ctypes.byref(cg), _DTYPES[v.dtype])
    if workspace is None:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=v.device)
    o = _out(v, g.sinogram_shape) if out is None else _dev(out, "out")
    with torch.cuda.device(v.device):
        _check(lib().pyro_fp_cone3d_ws(_ptr(v), _ptr(o), v.shape[0], ctypes.byref(cg), _ptr(workspace),
                                       workspace.numel() * workspace.element_size(), _DTYPES[v.dtype], _stream(v)))
    return o[0] if squeeze and out is None else o


def pyro_fp_cone3d_ws_storage(vol: torch.Tensor, g: ConeGeometry3D, storage: torch.dtype,
                              workspace: Optional[torch.Tensor] = None,
                              out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Cone-beam FP of an FP32 volume from a workspace copy held in
    `storage` (torch.float16 or torch.bfloat16); FP32 sinogram."""
    v, squeeze = _batched(_dev(vol, "volume"), 3, "volume")
    _shape_check(v, g.volume_shape, "volume")
    cg = g.to_c()
    need = lib().pyro_fp_cone3d_workspace_bytes(ctypes.byref(cg), _DTYPES[storage])
    if workspace is None:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=v.device)
    o = _out(v, g.sinogram_shape) if out is None else _dev(out, "out")
    with torch.cuda.device(v.device):
        _check(lib().pyro_fp_cone3d_ws_storage(_ptr(v), _ptr(o), v.shape[0], ctypes.byref(cg), _ptr(workspace),
                                               workspace.numel() * workspace.element_size(), _DTYPES[v.dtype],
                                               _DTYPES[storage], _stream(v)))
    return o[0] if squeeze and out is None else o


def pyro_fpT_par2d(sino: torch.Tensor, g: Geometry2D) -> torch.Tensor:
    return _fpT(lib().pyro_fpT_par2d, sino, g, g.volume_shape, g.sinogram_shape)


def pyro_fpT_fan2d(sino: torch.Tensor, g: Geometry2D) -> torch.Tensor:
    return _fpT(lib().pyro_fpT_fan2d, sino, g, g.volume_shape, g.sinogram_shape)


def pyro_fpT_cone3d(sino: torch.Tensor, g: ConeGeometry3D) -> torch.Tensor:
    return _fpT(lib().pyro_fpT_cone3d, sino, g, g.volume_shape, g.sinogram_shape)


def fpT_cone3d_workspace_bytes(g: ConeGeometry3D) -> int:
    """Workspace pyro_fpT_cone3d_ws needs (the ray-weighted sinogram of one
    batch item, transposed to [view][column][row], FP32)."""
    cg = g.to_c()
    return int(lib().pyro_fpT_cone3d_workspace_bytes(ctypes.byref(cg)))


def pyro_fpT_cone3d_ws(sino: torch.Tensor, g: ConeGeometry3D, workspace: Optional[torch.Tensor] = None,
                       out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Exact adjoint of the cone-beam FP, gathered voxel by voxel from the
    transposed, ray-weighted sinogram kept in `workspace` (allocated here
    when not given): the same result bit for bit from run to run."""
    s, squeeze = _batched(_dev(sino, "sinogram"), 3, "sinogram")
    _shape_check(s, g.sinogram_shape, "sinogram")
    cg = g.to_c()
    need = lib().pyro_fpT_cone3d_workspace_bytes(ctypes.byref(cg))
    if workspace is None:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=s.device)
    o = _out(s, g.volume_shape) if out is None else _dev(out, "out")
    with torch.cuda.device(s.device):
        _check(lib().pyro_fpT_cone3d_ws(_ptr(s), _ptr(o), s.shape[0], ctypes.byref(cg), _ptr(workspace),
                                        workspace.numel() * workspace.element_size(), _DTYPES[s.dtype], _stream(s)))
    return o[0] if squeeze and out is None else o


def pyro_bp_par2d(sino, g: Geometry2D, weight=W_NONE, scale=1.0):
    return _bp(lib().pyro_bp_par2d, sino, g, weight, scale, g.volume_shape, g.sinogram_shape)


def pyro_bp_fan2d(sino, g: Geometry2D, weight=W_NONE, scale=1.0):
    return _bp(lib().pyro_bp_fan2d, sino, g, weight, scale, g.volume_shape, g.sinogram_shape)


def pyro_bp_cone3d(sino, g: ConeGeometry3D, weight=W_NONE, scale=1.0):
    return _bp(lib().pyro_bp_cone3d, sino, g, weight, scale, g.volume_shape, g.sinogram_shape)


def pyro_bpT_par2d(vol, g: Geometry2D, weight=W_NONE, scale=1.0):
    return _bpT(lib().pyro_bpT_par2d, vol, g, weight, scale, g.volume_shape, g.sinogram_shape)


def pyro_bpT_fan2d(vol, g: Geometry2D, weight=W_NONE, scale=1.0):
    return _bpT(lib().pyro_bpT_fan2d, vol, g, weight, scale, g.volume_shape, g.sinogram_shape)


def pyro_bpT_cone3d(vol, g: ConeGeometry3D, weight=W_NONE, scale=1.0):
    return _bpT(lib().pyro_bpT_cone3d, vol, g, weight, scale, g.volume_shape, g.sinogram_shape)


# ------------------------------------------------------ weights / filters --
def pyro_weights2d(sino: torch.Tensor, g: Geometry2D, cosine=True, redund=REDUND_NONE) -> torch.Tensor:
    """In place; returns ``sino``."""
    s, _ = _batched(_dev(sino, "sinogram"), 2, "sinogram")
    _shape_check(s, g.sinogram_shape, "sinogram")
    cg = g.to_c()
    with torch.cuda.device(s.device):
        _check(lib().pyro_weights2d(_ptr(s), s.shape[0], ctypes.byref(cg), int(bool(cosine)), int(redund),
                                    _DTYPES[s.dtype], _stream(s)))
    return sino


def pyro_weights3d_table(sino: torch.Tensor, g: ConeGeometry3D, table: torch.Tensor, cosine=True) -> torch.Tensor:
    """In place: sino *= (cosine ? W_cos : 1) * table[view][column]; returns ``sino``."""
    s, _ = _batched(_dev(sino, "sinogram"), 3, "sinogram")
    _shape_check(s, g.sinogram_shape, "sinogram")
    t = _dev(table, "table")
    if t.dtype != torch.float32 or tuple(t.shape) != (g.number_of_projections, g.detector_shape[1]):
        raise ValueError("table must be float32 [n_views, nu]")
    t = t.contiguous()
    cg = g.to_c()
    with torch.cuda.device(s.device):
        _check(lib().pyro_weights3d_table(_ptr(s), s.shape[0], ctypes.byref(cg), _ptr(t), int(bool(cosine)),
                                          _DTYPES[s.dtype], _stream(s)))
    return sino


def pyro_redundancy_grad(a: torch.Tensor, g: torch.Tensor) -> torch.Tensor:
    """[V, nu] = sum over batch and rows of a * g; a, g float32 [..., V, nv, nu]."""
    a_, g_ = _dev(a, "a").contiguous(), _dev(g, "g").contiguous()
    if a_.shape != g_.shape or a_.dtype != torch.float32 or g_.dtype != torch.float32 or a_.dim() < 3:
        raise ValueError("a and g must be float32 tensors of one shape [..., V, nv, nu]")
    V, nv, nu = a_.shape[-3:]
    batch = a_.numel() // (V * nv * nu)
    out = torch.empty((V, nu), device=a_.device, dtype=torch.float32)
    with torch.cuda.device(a_.device):
        _check(lib().pyro_redundancy_grad(_ptr(a_), _ptr(g_), _ptr(out), batch, V, nv, nu, _stream(a_)))
    return out


def pyro_weights3d(sino: torch.Tensor, g: ConeGeometry3D, cosine=True, redund=REDUND_NONE) -> torch.Tensor:
    s, _ = _batched(_dev(sino, "sinogram"), 3, "sinogram")
    _shape_check(s, g.sinogram_shape, "sinogram")
    cg = g.to_c()
    with torch.cuda.device(s.device):
        _check(lib().pyro_weights3d(_ptr(s), s.shape[0], ctypes.byref(cg), int(bool(cosine)), int(redund),
                                    _DTYPES[s.dtype], _stream(s)))
    return sino


def pyro_filter_pad_length(nu: int) -> int:
    return int(lib().pyro_filter_pad_length(nu))


def pyro_filter_spectrum(kind: int, nu: int, tau: float) -> torch.Tensor:
    """K[0..pn/2] of a built-in filter, computed by the library (CPU tensor)."""
    K = torch.empty(pyro_filter_pad_length(nu) // 2 + 1, dtype=torch.float32)
    _check(lib().pyro_filter_spectrum(int(kind), int(nu), float(tau),
                                      ctypes.cast(K.data_ptr(), ctypes.POINTER(ctypes.c_float))))
    return K


def pyro_filter_rows(rows: torch.Tensor, tau: float, kind=RAMLAK, custom_K: Optional[torch.Tensor] = None,
                     out: Optional[torch.Tensor] = None) -> torch.Tensor:
    r = _dev(rows, "rows")
    nu = r.shape[-1]
    o = torch.empty_like(r) if out is None else _dev(out, "out")
    K = None
    if kind == FILTER_CUSTOM:
        K = _dev(custom_K, "custom_K")
        if K.dtype != torch.float32 or K.numel() != pyro_filter_pad_length(nu) // 2 + 1:
            raise ValueError("custom_K must be float32 with pad_length(nu)//2 + 1 entries")
    with torch.cuda.device(r.device):
        _check(lib().pyro_filter_rows(_ptr(r), _ptr(o), r.numel() // nu, nu, float(tau), int(kind), _ptr(K),
                                      _DTYPES[r.dtype], _stream(r)))
    return o


def pyro_filter_grad_K(p: torch.Tensor, g: torch.Tensor) -> torch.Tensor:
    p, g = _dev(p, "p"), _dev(g, "g")
    if p.dtype != torch.float32 or g.dtype != torch.float32 or p.shape != g.shape:
        raise ValueError("p and g must be float32 tensors of one shape")
    nu = p.shape[-1]
    dK = torch.empty(pyro_filter_pad_length(nu) // 2 + 1, device=p.device, dtype=torch.float32)
    with torch.cuda.device(p.device):
        _check(lib().pyro_filter_grad_K(_ptr(p), _ptr(g), _ptr(dK), p.numel() // nu, nu, _stream(p)))
    return dK


# ------------------------------------------------------------------ FBP --
def pyro_fdk(sino: torch.Tensor, g: ConeGeometry3D, kind=SHEPP_LOGAN, redund=REDUND_PARKER,
             custom_K: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None) -> torch.Tensor:
    s, squeeze = _batched(_dev(sino, "sinogram"), 3, "sinogram")
    _shape_check(s, g.sinogram_shape, "sinogram")
    cg = g.to_c()
    need = lib().pyro_fdk_workspace_bytes(ctypes.byref(cg), s.shape[0])
    if workspace is None:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=s.device)
    out = _out(s, g.volume_shape)
    with torch.cuda.device(s.device):
        _check(lib().pyro_fdk(_ptr(s), _ptr(out), s.shape[0], ctypes.byref(cg), int(kind), _ptr(custom_K),
                              int(redund), _ptr(workspace), workspace.numel() * workspace.element_size(),
                              _DTYPES[s.dtype], _stream(s)))
    return out[0] if squeeze else out


NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024


def pyro_fdk_noalloc(sino: torch.Tensor, g: ConeGeometry3D, kind=SHEPP_LOGAN, redund=REDUND_PARKER,
                     custom_K: Optional[torch.Tensor] = None) -> torch.Tensor:
    """FDK whose scratch is the library's static 64 MiB device array (for
    callers that cannot allocate a workspace); the output tensor is still
    allocated here by PyTorch, the C call itself allocates nothing."""
    s, squeeze = _batched(_dev(sino, "sinogram"), 3, "sinogram")
    _shape_check(s, g.sinogram_shape, "sinogram")
    cg = g.to_c()
    out = _out(s, g.volume_shape)
    with torch.cuda.device(s.device):
        _check(lib().pyro_fdk_noalloc(_ptr(s), _ptr(out), s.shape[0], ctypes.byref(cg), int(kind), _ptr(custom_K),
                                      int(redund), _DTYPES[s.dtype], _stream(s)))
    return out[0] if squeeze else out


def _fbp2d(fan, sino, g, kind, redund, custom_K, workspace):
    s, squeeze = _batched(_dev(sino, "sinogram"), 2, "sinogram")
    _shape_check(s, g.sinogram_shape, "sinogram")
    cg = g.to_c()
    need = lib().pyro_fbp2d_workspace_bytes(ctypes.byref(cg), s.shape[0])
    if workspace is None:
        workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=s.device)
    out = _out(s, g.volume_shape)
    nbytes = workspace.numel() * workspace.element_size()
    with torch.cuda.device(s.device):
        if fan:
            st = lib().pyro_fbp_fan2d(_ptr(s), _ptr(out), s.shape[0], ctypes.byref(cg), int(kind), _ptr(custom_K),
                                      int(redund), _ptr(workspace), nbytes, _DTYPES[s.dtype], _stream(s))
        else:
            st = lib().pyro_fbp_par2d(_ptr(s), _ptr(out), s.shape[0], ctypes.byref(cg), int(kind), _ptr(custom_K),
                                      _ptr(workspace), nbytes, _DTYPES[s.dtype], _stream(s))
        _check(st)
    return out[0] if squeeze else out


def pyro_fbp_par2d(sino, g: Geometry2D, kind=RAMLAK, custom_K=None, workspace=None):
    return _fbp2d(False, sino, g, kind, REDUND_NONE, custom_K, workspace)


def pyro_fbp_fan2d(sino, g: Geometry2D, kind=RAMLAK, redund=REDUND_FULL, custom_K=None, workspace=None):
    return _fbp2d(True, sino, g, kind, redund, custom_K, workspace)


# ------------------------------------------------------------ TV / vectors --
def _f32(t, name):
    t = _dev(t, name)
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    return t


def pyro_tv(x: torch.Tensor, eps: float, lam: float = 1.0, base: Optional[torch.Tensor] = None, alpha: float = 0.0,
            want_grad: bool = True, want_value: bool = True):
    """(grad, value): grad = alpha * base + lam * dTV/dx, value = TV(x) per
    batch item; x is [nz, ny, nx] or [batch, nz, ny, nx] (2D: nz = 1)."""
    xv = _f32(x, "x")
    shp = xv.shape
    if xv.dim() == 2:
        xv = xv.reshape(1, 1, *shp)
    elif xv.dim() == 3:
        xv = xv.unsqueeze(0)
    bsz, nz, ny, nx = xv.shape
    grad = torch.empty_like(xv) if want_grad else None
    value = torch.empty(bsz, device=xv.device, dtype=torch.float32) if want_value else None
    b = None if base is None else _f32(base, "base")
    with torch.cuda.device(xv.device):
        _check(lib().pyro_tv(_ptr(xv), _ptr(grad), _ptr(b), float(alpha), float(lam), _ptr(value), bsz, nz, ny, nx,
                             float(eps), _stream(xv)))
    return (None if grad is None else grad.reshape(shp)), value


def pyro_axpby(x: torch.Tensor, y: torch.Tensor, a: float, b: float) -> torch.Tensor:
    """y <- a x + b y in place."""
    x, y = _f32(x, "x"), _f32(y, "y")
    if x.numel() != y.numel():
        raise ValueError("x and y must have the same size")
    with torch.cuda.device(y.device):
        _check(lib().pyro_axpby(_ptr(x), _ptr(y), y.numel(), float(a), float(b), _stream(y)))
    return y


def pyro_dot(a: torch.Tensor, b: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """sum a_i b_i as a one-element float32 device tensor (FP32 reduction)."""
    a, b = _f32(a, "a"), _f32(b, "b")
    if a.numel() != b.numel():
        raise ValueError("a and b must have the same size")
    o = torch.empty(1, device=a.device, dtype=torch.float32) if out is None else out
    with torch.cuda.device(a.device):
        _check(lib().pyro_dot(_ptr(a), _ptr(b), a.numel(), _ptr(o), _stream(a)))
    return o


def pyro_bb_dots(x, x_prev, g, g_prev, dots: Optional[torch.Tensor] = None) -> torch.Tensor:
    """[|x - x_prev|^2, (x - x_prev).(g - g_prev)] as a float32 device tensor of 2."""
    t = [_f32(a, n) for a, n in ((x, "x"), (x_prev, "x_prev"), (g, "g"), (g_prev, "g_prev"))]
    if len({a.numel() for a in t}) != 1:
        raise ValueError("x, x_prev, g, g_prev must have one size")
    o = torch.empty(2, device=t[0].device, dtype=torch.float32) if dots is None else dots
    with torch.cuda.device(t[0].device):
        _check(lib().pyro_bb_dots(*(_ptr(a) for a in t), t[0].numel(), _ptr(o), _stream(t[0])))
    return o


def pyro_bb_update(x, x_prev, g, g_prev, dots: Optional[torch.Tensor], alpha0: float, alpha_max: float, first: bool,
                   alpha_out: Optional[torch.Tensor] = None):
    """x_prev = x, g_prev = g, x -= alpha g with alpha chosen on the device."""
    t = [_f32(a, n) for a, n in ((x, "x"), (x_prev, "x_prev"), (g, "g"), (g_prev, "g_prev"))]
    if len({a.numel() for a in t}) != 1:
        raise ValueError("x, x_prev, g, g_prev must have one size")
    with torch.cuda.device(t[0].device):
        _check(lib().pyro_bb_update(_ptr(t[0]), _ptr(t[1]), _ptr(t[2]), _ptr(t[3]), t[0].numel(), _ptr(dots),
                                    float(alpha0), float(alpha_max), int(bool(first)), _ptr(alpha_out),
                                    _stream(t[0])))


def pyro_sync_status(device=None) -> None:
    """Wait for the current stream of `device`; raise PyroError if it faulted."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    with torch.cuda.device(dev):
        _check(lib().pyro_sync_status(ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)))


def pyro_selftest_wait_timeout(limit_ms: int = 20, device=None) -> None:
    """Enqueue the bounded-wait self-test (see include/pyro.h)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    with torch.cuda.device(dev):
        _check(lib().pyro_selftest_wait_timeout(int(limit_ms),
                                                ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)))


def pyro_probe_gather(buf: torch.Tensor, loads_per_thread: int, threads: int, sink: torch.Tensor) -> None:
    """Enqueue the 16-byte random-gather probe over the bytes of `buf`."""
    b = _dev_any(buf, "buf")
    with torch.cuda.device(b.device):
        _check(lib().pyro_probe_gather(_ptr(b), b.numel() * b.element_size(), int(loads_per_thread), int(threads),
                                       _ptr(sink), _stream(b)))


def _dev_any(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA tensor")
    return t


# ------------------------------------------------------------ residual CNN --
CNN_RELU_BWD, CNN_AVGPOOL2, CNN_AVGPOOL2_BWD, CNN_UPSAMPLE2, CNN_UPSAMPLE2_BWD, CNN_ADD = 0, 1, 2, 3, 4, 5
CNN_F32_TO_BF16, CNN_BF16_TO_F32, CNN_RESIDUAL = 6, 7, 8


def _cuda(t, name, dtype):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous() or t.dtype != dtype:
        raise TypeError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t


def pyro_conv3d(x: torch.Tensor, w: torch.Tensor, bias: Optional[torch.Tensor], relu: bool,
                out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """x [B, D, H, W, cin] bf16, w [27, cout, cin] bf16, bias [cout] f32 -> [B, D, H, W, cout] bf16."""
    _cuda(x, "x", torch.bfloat16)
    _cuda(w, "w", torch.bfloat16)
    B_, D, H, W, cin = x.shape
    cout = w.shape[1]
    if w.shape != (27, cout, cin):
        raise ValueError("w must be [27, cout, cin]")
    if bias is not None:
        _cuda(bias, "bias", torch.float32)
    y = torch.empty((B_, D, H, W, cout), device=x.device, dtype=torch.bfloat16) if out is None else out
    with torch.cuda.device(x.device):
        _check(lib().pyro_conv3d(_ptr(x), _ptr(w), _ptr(bias), _ptr(y), B_, D, H, W, cin, cout, int(relu), _stream(x)))
    return y


def pyro_conv3d_wgrad(x: torch.Tensor, dy: torch.Tensor) -> torch.Tensor:
    _cuda(x, "x", torch.bfloat16)
    _cuda(dy, "dy", torch.bfloat16)
    B_, D, H, W, cin = x.shape
    cout = dy.shape[-1]
    dw = torch.empty((27, cout, cin), device=x.device, dtype=torch.float32)
    with torch.cuda.device(x.device):
        _check(lib().pyro_conv3d_wgrad(_ptr(x), _ptr(dy), _ptr(dw), B_, D, H, W, cin, cout, _stream(x)))
    return dw


def pyro_conv3d_flip_weights(w: torch.Tensor) -> torch.Tensor:
    _cuda(w, "w", torch.bfloat16)
    _, cout, cin = w.shape
    wf = torch.empty((27, cin, cout), device=w.device, dtype=torch.bfloat16)
    with torch.cuda.device(w.device):
        _check(lib().pyro_conv3d_flip_weights(_ptr(w), _ptr(wf), cin, cout, _stream(w)))
    return wf


def pyro_cnn_op(op: int, a: torch.Tensor, y: torch.Tensor, b: Optional[torch.Tensor] = None,
                f: Optional[torch.Tensor] = None, dims=(0, 0, 0, 0)) -> torch.Tensor:
    nz, ny, nx, c = dims
    with torch.cuda.device(a.device):
        _check(lib().pyro_cnn_op(int(op), _ptr(a), _ptr(b), _ptr(y), _ptr(f), y.numel(), nz, ny, nx, c, _stream(a)))
    return y


def pyro_cnn_bias_grad(dy: torch.Tensor) -> torch.Tensor:
    _cuda(dy, "dy", torch.bfloat16)
    c = dy.shape[-1]
    db = torch.empty(c, device=dy.device, dtype=torch.float32)
    with torch.cuda.device(dy.device):
        _check(lib().pyro_cnn_bias_grad(_ptr(dy), _ptr(db), dy.numel() // c, c, _stream(dy)))
    return db


def pyro_cnn_mse(out: torch.Tensor, target: torch.Tensor, grad: Optional[torch.Tensor] = None) -> torch.Tensor:
    _cuda(out, "out", torch.float32)
    _cuda(target, "target", torch.float32)
    loss = torch.empty(1, device=out.device, dtype=torch.float32)
    with torch.cuda.device(out.device):
        _check(lib().pyro_cnn_mse(_ptr(out), _ptr(target), _ptr(grad), _ptr(loss), out.numel(), _stream(out)))
    return loss


def pyro_cnn_adam(p, g, m, v, p16, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    with torch.cuda.device(p.device):
        _check(lib().pyro_cnn_adam(_ptr(p), _ptr(g), _ptr(m), _ptr(v), _ptr(p16), p.numel(), float(lr), float(beta1),
                                   float(beta2), float(eps), int(step), _stream(p)))


def version() -> str:
    return lib().pyro_version().decode()
