"""B300-native split-step Fourier propagation through a three-waveguide
potential (Morgan et al., "Coherent transport by adiabatic passage on atom
chips", Sec. IV-V).

The compute path is libctap.so (CUDA, sm_103a) behind the C ABI in
include/ctap.h; ``ctap`` is its thin ctypes binding and ``workloads`` builds
seeded synthetic inputs.  Importing the package does not load the library;
the first Plan does, and raises if it has not been built.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "ctap", "build"]
