"""GB300-native sparse-state quantum-walk simulator (arXiv 2303.06890).

Submodules are imported on demand: ``qwalk`` (ctypes binding of the C ABI in
include/qwalk.h, loads libqwalk.so), ``build`` (nvcc build of the library) and
``workloads`` (seeded synthetic inputs).  Importing the package itself loads no
native code.
"""
