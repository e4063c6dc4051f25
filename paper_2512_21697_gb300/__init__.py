"""GB300-native Crank-Nicolson step of the 3D time-dependent Dirac equation (arXiv 2512.21697).

The method runs in libdirac_gb300.so (C ABI in include/dirac.h): host C++ for the basis and
operator setup, hand-written sm_103a CUDA kernels for every part of the time step.
``binding`` exposes the C ABI to Python; ``workloads`` holds the seeded synthetic inputs.
"""
from . import workloads  # noqa: F401
