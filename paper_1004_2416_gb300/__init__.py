"""GB300-native (sm_103a) implementation of the immersed-boundary lattice
Boltzmann finite-element time step of Krueger, Varnik and Raabe
(arXiv:1004.2416): D3Q19 BGK collide-and-stream with Guo forcing and shear
walls, IBM spreading and interpolation, Skalak membrane forces and the Taylor
deformation, behind the C ABI of ``include/iblbm.h``.
"""
from .iblbm import Sim, IblbmError, LIB_PATH  # noqa: F401
