"""GB300-native (sm_103a) implementation of the immersed-boundary lattice
Boltzmann finite-element time step of Krueger, Varnik and Raabe
(arXiv:1004.2416): D3Q19 BGK collide-and-stream with Guo forcing and shear
walls, IBM spreading and interpolation, Skalak membrane forces and the Taylor
deformation, behind the C ABI of ``include/iblbm.h``.

The CUDA library is loaded on first use of ``Sim``, ``IblbmError`` or
``LIB_PATH`` (or on ``import paper_1004_2416_gb300.iblbm``), so that the
seeded input generators of ``workloads`` and the build script import without
mapping it.
"""

_BINDING = ("Sim", "IblbmError", "LIB_PATH")


def __getattr__(name):
    if name in _BINDING:
        from . import iblbm

        return getattr(iblbm, name)
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")
