"""GB300-native 2D TMz FDTD of leaf light scattering (arXiv 2512.17132).

The computation lives in libfdtd.so (CUDA, sm_103a; C ABI in include/fdtd.h);
`fdtd` is its ctypes binding and `build` compiles it in-tree.
"""
from . import fdtd  # noqa: F401
from .fdtd import Simulation, load_library  # noqa: F401
