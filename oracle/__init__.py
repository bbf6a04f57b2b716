"""FP64 CPU oracle of the two-population compressible semi-Lagrangian LBM
step on a moving, blended, body-fitted mesh (Bhadauria, Dorschner & Karlin,
"Lattice Boltzmann method for fluid-structure interaction in compressible
flow").

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never calls it and shares no code with it: the two meet only in the
seeded input arrays (mesh tables, initial fields) that the callers hand to
both.

Plain numpy, float64, vectorised over nodes only.  Each function cites the
section / equation of the paper it follows.  Readings of passages that are
silent, garbled or ambiguous are labelled R<n> in the docstrings.

Parity status per part (what pins each function):
  kinetics   pinned: closed-form moments, textbook D2Q9 at T = 1/3,
             conservation, Chapman-Enskog decay rates; the Grad terms'
             stress equals the Navier-Stokes stress, their heat flux and
             energy moment at a no-slip wall (tests).
  mesh       pinned: brute-force element search, polynomial exactness,
             textbook streaming on a lattice-matched mesh.
  ale        pinned: r5 closed form, rigid/stationary limits, translation
             and rotation identities.
  boundary   pinned: rest state around a wall is a fixed point; Grad
             moments equal the prescribed P(1), q(1), R(1); radial wall
             normals of a circle; the missing set of a static wall is
             exactly {c . n0 > 0}; wall targets exact on linear fields at
             B = A + dt n0 and taken from the previous step's field; the
             inlet set of O- and C-grids is exactly {U_inf . n_out < 0},
             outlet targets exact on linear fields at B = A - dt n_out.
  forces     pinned: uniform stress -> 0, linear pressure -> -A grad p.
  structure  pinned: RK4 Taylor identity, forced-oscillator solution,
             nondimensional 1-DOF form.
  unstructured  pinned: a relabelled O-grid reproduces the structured
             departures and step; gradients exact for linear fields (and
             quadratics on affine elements); Taylor-Green decay on an
             unstructured box; symmetric flow kept symmetric on a C-grid
             element list.
  solver     whole coupled run: parity unpinned beyond the per-part pins and
             the free-stream / decay-rate invariants.
"""
from . import kinetics, mesh, ale, boundary, forces, structure, solver  # noqa: F401
