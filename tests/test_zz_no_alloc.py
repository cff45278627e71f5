"""The allocation-free V-cycle entry point against the ordinary one.

hhg_vcycle_noalloc serves callers that cannot call cudaMalloc once they run
(their device memory is owned by another allocator, or allocation is banned
on their path): its coarse-grid CG takes its work vectors from a fixed static
device array instead of allocated memory.  It must give the same iterate as
hhg_vcycle, call after call, and refuse meshes whose coarse problem does not
fit the array.  This file is collected last on purpose.
"""

import numpy as np
import pytest

import hhg_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1506_06185_gb300 import build
    from paper_1506_06185_gb300 import hhg
    build()
    return hhg


def test_noalloc_vcycle_matches_vcycle_on_two_calls(H):
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=6)
    u0 = I.initial_guess(sub, R, I.harmonic_boundary(sub, R))
    a, b = H.Mesh(sub, R), H.Mesh(sub, R)
    a.set_problem(f, u0)
    b.set_problem(f, u0)
    for call in range(2):
        H.hhg_vcycle(a.h, 3, 3, want_residual=False)
        H.hhg_vcycle_noalloc(b.h, 3, 3)
        ua, ub = a.get_solution(), b.get_solution()
        rel = np.linalg.norm(ua - ub) / np.linalg.norm(ua)
        assert rel <= 1e-12, (call, rel)
    a.close()
    b.close()


def test_noalloc_rejects_coarse_problems_beyond_the_array(H):
    # 7x7x7 sub-cubes: the coarsest level has 27^3 = 19683 > 16384 unknowns
    m = H.Mesh((7, 7, 7), 3)
    with pytest.raises(H.HHGError) as e:
        H.hhg_vcycle_noalloc(m.h, 3, 3)
    assert e.value.code == H.HHG_ERR_ARG
    assert "16384" in str(e.value)
    m.close()
