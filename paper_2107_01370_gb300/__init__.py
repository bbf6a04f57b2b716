"""GB300 implementation of the two-population compressible semi-Lagrangian
lattice Boltzmann step with rigid-body coupling on blended body-fitted meshes
(Bhadauria, Dorschner & Karlin, "Lattice Boltzmann method for fluid-structure
interaction in compressible flow").

  inputs   seeded synthetic meshes and initial fields
  lbfsi    ctypes binding of liblbfsi.so (the C ABI of include/lbfsi.h)
  build    in-tree nvcc build of liblbfsi.so for sm_103a

The binding is imported lazily so that the input generators can be used
without the compiled library.
"""

__all__ = ["inputs", "lbfsi", "build"]
