"""GB300-native resilient hierarchical-hybrid multigrid (HHG).

Matrix-free P1 multigrid V-cycles on uniformly refined tetrahedral macro
meshes with fault injection and local / Dirichlet-Dirichlet recovery, after
Huber, Gmeiner, Ruede, Wohlmuth, "Resilience for Multigrid Software at the
Extreme Scale".  The compute path is the CUDA library ``_lib/libhhg.so``
(C ABI in ``include/hhg.h``); ``paper_1506_06185_gb300.hhg`` binds it and
``paper_1506_06185_gb300.build`` compiles it.
"""

from .build import build, LIB  # noqa: F401
