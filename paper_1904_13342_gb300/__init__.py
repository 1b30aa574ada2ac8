"""GB300-native known-operator CT layers (PYRO-NN hot path, sm_103a).

``binding`` exposes the C ABI of include/pyro.h one-to-one on CUDA tensors;
``geometry`` describes parallel / fan / cone-beam set-ups; ``autograd``
registers the operators as differentiable layers; ``phantoms`` draws the
seeded synthetic inputs.  The CUDA library is loaded on first use.
"""
from . import geometry
from .geometry import ConeGeometry3D, FanGeometry2D, Geometry2D, ParallelGeometry2D, short_scan_range

__all__ = ["geometry", "ConeGeometry3D", "FanGeometry2D", "Geometry2D", "ParallelGeometry2D", "short_scan_range"]
