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
from parity import assert_close

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
        assert_close(b.get_solution(), a.get_solution(), 1e-12, what=f"call {call}")
    a.close()
    b.close()


def test_noalloc_allocates_nothing_on_repeated_calls(H):
    """After the first call (which looks up the static array's address and may
    load the library's device code), further calls leave the device's free
    memory and the mesh's own allocations unchanged."""
    import torch
    sub, R = (2, 2, 2), 5
    m = H.Mesh(sub, R)
    m.set_problem(I.random_load(sub, R, seed=2), I.initial_guess(sub, R))
    H.hhg_vcycle_noalloc(m.h, 3, 3)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    bytes0 = m.bytes()
    for _ in range(3):
        H.hhg_vcycle_noalloc(m.h, 3, 3)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and m.bytes() == bytes0, (free0 - free1, m.bytes() - bytes0)
    m.close()


def test_noalloc_vcycle_on_a_general_mesh(H):
    """A macro mesh of general connectivity (five tetrahedra per sub-cube):
    the allocation-free cycle equals the ordinary one there too."""
    v, t = I.five_tet_macro_mesh((2, 2, 1), seed=3, amp=0.12)
    R = 4
    a, b = H.Mesh.general(v, t, R), H.Mesh.general(v, t, R)
    rng = np.random.default_rng(9)
    f = rng.uniform(-1.0, 1.0, a.n_nodes)
    u0 = np.zeros(a.n_nodes)
    a.set_problem(f, u0)
    b.set_problem(f, u0)
    for call in range(2):
        H.hhg_vcycle(a.h, 3, 3, want_residual=False)
        H.hhg_vcycle_noalloc(b.h, 3, 3)
        assert_close(b.get_solution(), a.get_solution(), 1e-12, what=f"general mesh, call {call}")
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
