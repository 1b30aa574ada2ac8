"""Geometry descriptions (paper, Section "Reconstruction & Geometry").

A geometry holds the attributes the paper lists: volume shape and spacing,
detector shape and spacing, number of projections, angular range, and for
fan / cone beam the source-to-iso-centre (SID) and source-to-detector (SDD)
distances; the trajectory is one central-ray direction per view (2D, given
by the view angles) or one 3x4 projection matrix per view (3D, Section
"Trajectories"; ``None`` means the circular trajectory built inside the
library).  Shapes are given slowest axis first, like the tensors:
(ny, nx) / (nz, ny, nx) for volumes, nu / (nv, nu) for detectors.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field, replace
from typing import Optional, Sequence

import numpy as np


class CGeom2D(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("sx", ctypes.c_double), ("sy", ctypes.c_double),
        ("nu", ctypes.c_int), ("su", ctypes.c_double),
        ("n_views", ctypes.c_int), ("angles", ctypes.POINTER(ctypes.c_double)),
        ("range", ctypes.c_double), ("sid", ctypes.c_double), ("sdd", ctypes.c_double),
        ("step", ctypes.c_double),
    ]


class CGeom3D(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("sx", ctypes.c_double), ("sy", ctypes.c_double), ("sz", ctypes.c_double),
        ("nu", ctypes.c_int), ("nv", ctypes.c_int),
        ("su", ctypes.c_double), ("sv", ctypes.c_double),
        ("n_views", ctypes.c_int),
        ("proj_mats", ctypes.POINTER(ctypes.c_double)),
        ("angles", ctypes.POINTER(ctypes.c_double)),
        ("range", ctypes.c_double), ("sid", ctypes.c_double), ("sdd", ctypes.c_double),
        ("step", ctypes.c_double),
    ]


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Geometry2D:
    """2D parallel-beam (sid/sdd None) or fan-beam geometry."""
    volume_shape: Sequence[int]  # (ny, nx)
    volume_spacing: Sequence[float]  # (sy, sx) mm
    detector_shape: int  # nu
    detector_spacing: float  # su mm
    number_of_projections: int
    angular_range: float  # rad
    sid: Optional[float] = None
    sdd: Optional[float] = None
    angles: Optional[np.ndarray] = None  # explicit view angles (rad)
    step: float = 0.0  # FP sampling step (mm), 0: half the smallest spacing
    _keep: list = field(default_factory=list, repr=False, compare=False)

    @property
    def fan(self) -> bool:
        return self.sid is not None

    @property
    def sinogram_shape(self):
        return (self.number_of_projections, self.detector_shape)

    def view_angles(self) -> np.ndarray:
        if self.angles is not None:
            return np.asarray(self.angles, dtype=np.float64)
        return np.arange(self.number_of_projections) * (self.angular_range / self.number_of_projections)

    def central_ray_vectors(self) -> np.ndarray:
        """[V, 2] unit central-ray direction c = (cos b, sin b) of every view
        (the 2D trajectory as the paper describes it)."""
        b = self.view_angles()
        return np.stack([np.cos(b), np.sin(b)], axis=1)

    def with_central_ray_vectors(self, vectors) -> "Geometry2D":
        """The same geometry on a trajectory given by central-ray vectors [V, 2]."""
        v = np.asarray(vectors, dtype=np.float64)
        if v.ndim != 2 or v.shape[1] != 2 or not np.all(np.linalg.norm(v, axis=1) > 0):
            raise ValueError("central ray vectors must be a nonzero [V, 2] array")
        return replace(self, number_of_projections=v.shape[0], angles=np.arctan2(v[:, 1], v[:, 0]), _keep=[])

    def to_c(self) -> CGeom2D:
        ang = None if self.angles is None else np.ascontiguousarray(self.angles, dtype=np.float64)
        if ang is not None and ang.size != self.number_of_projections:
            raise ValueError("angles must have number_of_projections entries")
        self._keep = [ang]
        ny, nx = self.volume_shape
        sy, sx = self.volume_spacing
        return CGeom2D(nx, ny, sx, sy, self.detector_shape, self.detector_spacing, self.number_of_projections,
                       _dptr(ang), self.angular_range, self.sid or 0.0, self.sdd or 0.0, self.step)


def ParallelGeometry2D(volume_shape, volume_spacing, detector_shape, detector_spacing, number_of_projections,
                       angular_range=math.pi, angles=None, step=0.0) -> Geometry2D:
    return Geometry2D(tuple(volume_shape), tuple(volume_spacing), int(detector_shape), float(detector_spacing),
                      int(number_of_projections), float(angular_range), None, None, angles, step)


def FanGeometry2D(volume_shape, volume_spacing, detector_shape, detector_spacing, number_of_projections,
                  angular_range, sid, sdd, angles=None, step=0.0) -> Geometry2D:
    return Geometry2D(tuple(volume_shape), tuple(volume_spacing), int(detector_shape), float(detector_spacing),
                      int(number_of_projections), float(angular_range), float(sid), float(sdd), angles, step)


@dataclass
class ConeGeometry3D:
    volume_shape: Sequence[int]  # (nz, ny, nx)
    volume_spacing: Sequence[float]  # (sz, sy, sx) mm
    detector_shape: Sequence[int]  # (nv, nu)
    detector_spacing: Sequence[float]  # (sv, su) mm
    number_of_projections: int
    angular_range: float
    sid: float
    sdd: float
    projection_matrices: Optional[np.ndarray] = None  # [V, 3, 4]
    angles: Optional[np.ndarray] = None
    step: float = 0.0
    _keep: list = field(default_factory=list, repr=False, compare=False)

    @property
    def sinogram_shape(self):
        return (self.number_of_projections, *self.detector_shape)

    def view_angles(self) -> np.ndarray:
        if self.angles is not None:
            return np.asarray(self.angles, dtype=np.float64)
        return np.arange(self.number_of_projections) * (self.angular_range / self.number_of_projections)

    def trajectory(self) -> np.ndarray:
        """[V, 3, 4] projection matrices the library uses for this geometry:
        the given ones normalised, or the circular trajectory's (computed by
        the library from the geometry)."""
        from .shard import projection_matrices

        return projection_matrices(self)

    def to_c(self) -> CGeom3D:
        P = None
        if self.projection_matrices is not None:
            P = np.ascontiguousarray(self.projection_matrices, dtype=np.float64)
            if P.shape != (self.number_of_projections, 3, 4):
                raise ValueError("projection_matrices must be [number_of_projections, 3, 4]")
        ang = None if self.angles is None else np.ascontiguousarray(self.angles, dtype=np.float64)
        if ang is not None and ang.size != self.number_of_projections:
            raise ValueError("angles must have number_of_projections entries")
        self._keep = [P, ang]
        nz, ny, nx = self.volume_shape
        sz, sy, sx = self.volume_spacing
        nv, nu = self.detector_shape
        sv, su = self.detector_spacing
        return CGeom3D(nx, ny, nz, sx, sy, sz, nu, nv, su, sv, self.number_of_projections, _dptr(P), _dptr(ang),
                       self.angular_range, self.sid, self.sdd, self.step)


def short_scan_range(detector_width_mm: float, sdd: float) -> float:
    """pi + 2 delta, delta = atan(width / (2 SDD)): the Parker short scan."""
    return math.pi + 2.0 * math.atan(0.5 * detector_width_mm / sdd)
