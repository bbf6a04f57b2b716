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
             conservation, Chapman-Enskog decay rates (tests).
  mesh       pinned: brute-force element search, polynomial exactness,
             textbook streaming on a lattice-matched mesh.
  ale        pinned: r5 closed form, rigid/stationary limits, translation
             and rotation identities.
  boundary   pinned: rest state around a wall is a fixed point; Grad
             moments equal the prescribed P(1), q(1), R(1).
  forces     pinned: uniform stress -> 0, linear pressure -> -A grad p.
  structure  pinned: RK4 Taylor identity, forced-oscillator solution,
             nondimensional 1-DOF form.
  solver     whole coupled run: parity unpinned beyond the per-part pins and
             the free-stream / decay-rate invariants.
"""
from . import kinetics, mesh, ale, boundary, forces, structure, solver  # noqa: F401
