"""GB300-native Newton step of the VMS / generalized-alpha hyper-elastodynamics
scheme with nested block preconditioning (Liu & Marsden, arXiv:1809.06350).

* ``hyel``   -- ctypes binding of the CUDA library libhyel.so (include/hyel.h)
* ``inputs`` -- seeded synthetic meshes, boundary sets, materials and states
* ``build``  -- in-tree nvcc build of libhyel.so for sm_103a

Importing the package loads nothing; ``hyel.lib()`` loads the library on first
use and raises if it is missing.
"""
