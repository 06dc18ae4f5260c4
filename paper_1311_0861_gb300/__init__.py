"""GB300-native two-fluid FlIC/Godunov step (Kulikov 2013, GPUPEGAS), behind a C ABI.

The compute path is the CUDA library ``libflic.so`` (built by ``build``); this
package holds its thin ctypes binding (``flic``) and the seeded input generators
(``inputs``).  Importing the package does not load the library.
"""
__all__ = ["flic", "inputs", "build"]
