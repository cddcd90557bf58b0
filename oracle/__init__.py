"""CPU FP64 oracle for the graph-based FEM fracture step (test infrastructure).

This package is test infrastructure, not part of the product.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg
of ``bench.py`` may import it.  It shares no code with the CUDA path: the
two meet only at the seeded input generators in ``workloads/``.

It is deliberately plain and slow: numpy/scipy in float64, one function per
step of the method, each citing the passage of the paper it follows
(Mandal, Chaudhuri & Chaudhuri, "Remeshing-Free Graph-Based Finite Element
Method for Ductile and Brittle Fracture").

Modules
  mesh     -- edges, tet->edge map, rest geometry, lumped mass, neighbourhoods
  elastic  -- C from edge lengths by the least squares of Thm 3.1 (Eq. 27-31),
              StVK (Eq. 37), stable Neo-Hookean (Eq. 35), edge forces (Eq. 12),
              tangent (Eq. 10/33), chi
              scaling (Eq. 32-34)
  damage   -- stress (Eq. 14), edge projection (Eq. 16-19), non-local average
              (Eq. 20), relabel (Eq. 21), chi (Eq. 22-25)
  step     -- linearised backward-Euler step (Eq. 2, Algorithm 1, Sec. 4.3),
              Newton iterations, consistent mass (Eq. 5), the quasi-static
              load step (Eq. 36)
  solve    -- preconditioned conjugate gradients and the direct solve
  surface  -- split visualisation mesh and crack quads (Sec. 4.1, Fig. 6)
  gnn      -- the learned warm start / block preconditioner network

Parity pins live in ``tests/test_oracle_*.py``.
"""
from . import mesh, elastic, damage, step, solve, surface  # noqa: F401
