"""FP64 CPU oracle for the neural-SDF collision query.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may use it.  It shares no code with the CUDA library;
the only common module is ``synth`` (seeded inputs, none of the method's
arithmetic).

Contents, each function citing the passage of the paper it follows:

* ``mlp``  - the SDF network f (Eq. 1), its analytic input gradient (the
  back-propagated normal, Eq. 2), the collision test f < eps (Sec. 3.2),
  the contact point (Eq. 3) with the naive solve, the rigid-transform rule
  (Sec. 4.2), and the parameter / input gradients of a loss that depends on
  f and on its gradient (used for fitting and for collision penalties).
* ``mesh`` - exact signed distance to a watertight triangle mesh by brute
  force (the ground truth a network is fitted to, Sec. 3.1): closest point on
  a triangle, sign from the generalized winding number.
* ``rounded`` - the Fourier-feature ReLU network of Sec. 4.3 with its
  tensor-core operands rounded to a 16-bit format, so that the ReLU
  decisions are taken in the precision of the 16-bit kernels.
* ``cloth`` - one explicit Verlet step of a mass-spring quad cloth followed
  by the collision solve (Sec. 4.1).
* ``voxel`` - the voxel SDF baseline of Sec. 4.3 (Table 1): trilinear
  interpolation of a grid of signed distances, its gradient and the same
  collision query.

Parity status: every function here is pinned by closed forms, brute force or
finite differences in ``tests/test_oracle_*.py``; the paper prints no worked
numerical example, so nothing is pinned to a printed value.
"""

from . import mlp, mesh, cloth, rounded, voxel  # noqa: F401
