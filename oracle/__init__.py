"""Plain FP64 CPU multigrid oracle for the resilient HHG multigrid path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import anything from this
package.  The product path (the CUDA library and its Python binding) never
imports it, and this package imports nothing from the product.

What it computes follows Huber, Gmeiner, Ruede, Wohlmuth, "Resilience for
Multigrid Software at the Extreme Scale":

* the model problem and its P1 discretisation on a uniformly refined
  tetrahedral macro mesh, §2.1 Eq. (1)-(2);
* the multigrid correction-scheme V-cycle with linear interpolation, its
  adjoint, Gauss-Seidel smoothing (3 pre / 3 post) and a CG coarse solver,
  §2.1;
* the fault model (one or more macro-tetrahedra lose their volume unknowns
  after a complete cycle; they are re-initialised with zero), §2.2, and the
  cycle advantage kappa, Eq. (3);
* the local recovery (LR) and Dirichlet-Dirichlet recovery (DD) of §4.2,
  Algorithm 1, with n_F = ceil(eta * n_I) from §4.4.

Every function works on the global structured node grid of the cube family:
the fine mesh of a cube split into Kuhn macro-tetrahedra and refined
uniformly is the Freudenthal triangulation of that grid.  The macro vertices
may also sit at arbitrary physical positions (general tetrahedral shapes of a
polyhedral domain with the same connectivity, §2.1): each macro is then the
image of its reference lattice under its own affine map.  Per-macro blocked
storage is a GPU concern and is deliberately absent here.

``oracle/unstructured.py`` (imported as ``oracle.unstructured``) is the same
method on a macro mesh of general connectivity (vertex and tetrahedron
arrays), with its own smoother reading for that case.

Parity status of each function is listed in ``oracle/hhg_oracle.py`` and
``oracle/unstructured.py``.
"""

from .hhg_oracle import *  # noqa: F401,F403
