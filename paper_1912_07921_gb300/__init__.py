"""GB300-native real-time TDDFT propagation: Kohn-Sham H psi on a uniform 3D grid inside
a 4th-order Taylor exp(-i dt H), with FP64 density, norm, energy and dipole/current
reductions (arXiv:1912.07921, Sec. "New propagators for real-time TDDFT").

The compute path is the CUDA library ``_build/libtdks.so`` (C interface in
``include/tdks.h``); this package only marshals arguments to it.
"""
from .system import System  # noqa: F401
from . import inputs  # noqa: F401
