"""The streaming Gauss-Seidel kernel (7-point structure, levels refined 6 or
more times): neighbour colours staged in shared memory by bulk asynchronous
copies on mbarriers, slice by slice (§2.1 smoother).

* Against the oracle node by node (parity.assert_close) for V-cycles and for
  solves with DD / DN recovery.
* Against the row-pair tile kernel (the default; the streaming kernel is
  switched on per mesh with hhg_set_streaming): a colour's update is the same
  arithmetic in the same order, so the iterates agree bit for bit, in FP64
  and in the FP32 cycles of mixed precision.
* Bounded waits: with hhg_set_wait_limit(mesh, 0) every wait of the kernel
  runs out at once; the CTAs report it through the mesh's error flag, let
  their copies in flight land and stop, and the next synchronising call
  returns HHG_ERR_TIMEOUT.  Only the streaming kernel waits, so this also
  shows that it ran.  Afterwards the mesh works as before.
"""

import numpy as np
import pytest

import hhg_inputs as I
import oracle as O
from parity import assert_close

pytestmark = pytest.mark.gpu

ATOL_HIST = 1e-12


@pytest.fixture(scope="module")
def hhg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1506_06185_gb300 import build
    from paper_1506_06185_gb300 import hhg as H
    build()
    return H


def _assert_streams(hhg, M):
    """The mesh's Gauss-Seidel streams: with no tries left every wait runs out."""
    hhg.hhg_set_wait_limit(M.h, 0)
    with pytest.raises(hhg.HHGError) as e:
        M.vcycle()
    assert e.value.code == hhg.HHG_ERR_TIMEOUT
    hhg.hhg_set_wait_limit(M.h, -1)


@pytest.mark.parametrize("sub,R", [((2, 2, 2), 6), ((1, 1, 1), 7)])
def test_streaming_vcycles_match_oracle_and_tile_kernel(hhg, sub, R):
    f = I.random_load(sub, R, seed=11)
    u0 = I.initial_guess(sub, R, I.harmonic_boundary(sub, R))
    coeff = np.exp(np.random.default_rng(12).standard_normal(6 * int(np.prod(sub))))
    S, T = hhg.Mesh(sub, R, coeff=coeff), hhg.Mesh(sub, R, coeff=coeff)
    hhg.hhg_set_streaming(S.h, 1)
    S.set_problem(f, u0)
    T.set_problem(f, u0)
    m = O.Mesh(sub, R, coeff=coeff)
    uo, fo = O.pad(u0.copy()), O.pad(f)
    r0 = O.resnorm(m, uo, fo)
    top = len(m.levels) - 1
    for k in range(3):
        rs = S.vcycle()
        T.vcycle()
        O.vcycle(m, m.global_problem, top, uo, fo)
        us = S.get_solution()
        assert_close(us, O.interior(uo), what=f"cycle {k}")
        assert np.array_equal(us, T.get_solution()), f"cycle {k}: streaming and tile kernels differ"
        assert abs(rs - O.resnorm(m, uo, fo)) <= ATOL_HIST * r0
    _assert_streams(hhg, S)
    # usable again after the timeout: a fresh start gives the tile kernel's bits
    S.set_problem(f, u0)
    T.set_problem(f, u0)
    S.vcycle()
    T.vcycle()
    assert np.array_equal(S.get_solution(), T.get_solution())
    S.close()
    T.close()


@pytest.mark.parametrize("recovery", [2, 3])
def test_streaming_solve_with_recovery_matches_oracle(hhg, recovery):
    """DD (Algorithm 1) and DN (Algorithm 2) on a sub-cube at refinement 6."""
    sub, R = (2, 2, 2), 6
    f = I.random_load(sub, R, seed=13)
    u0 = I.initial_guess(sub, R)
    kw = dict(rtol=1e-9, max_cycles=40, fault_cycle=3, fault_ids=I.subcube_macros(sub, 1, 1, 0),
              recovery=recovery, n_global=2, eta=3.0)
    S, T = hhg.Mesh(sub, R), hhg.Mesh(sub, R)
    hhg.hhg_set_streaming(S.h, 1)
    S.set_problem(f, u0)
    T.set_problem(f, u0)
    hs, cs, _ = S.solve(**kw)
    ht, ct, _ = T.solve(**kw)
    m = O.Mesh(sub, R)
    uo = O.pad(u0.copy())
    ref = O.solve(m, uo, O.pad(f), **kw)
    assert cs == ct == ref["cycles"]
    assert np.abs(hs - ref["hist"]).max() <= ATOL_HIST
    us = S.get_solution()
    assert_close(us, O.interior(uo), what="solve")
    assert np.array_equal(us, T.get_solution())
    S.close()
    T.close()


def test_streaming_fp32_cycles_match_tile_kernel(hhg):
    """Mixed precision (FP32 cycles in FP64 refinement) at refinement 6 with
    a DD recovery: the streaming FP32 sweeps give the tile kernel's bits."""
    sub, R = (2, 2, 2), 6
    f = I.random_load(sub, R, seed=14)
    u0 = I.initial_guess(sub, R)
    kw = dict(rtol=1e-9, max_cycles=40, fault_cycle=3, fault_ids=I.subcube_macros(sub), recovery=2, n_global=2,
              eta=4.0, mixed_precision=True)
    S, T = hhg.Mesh(sub, R, precision=32), hhg.Mesh(sub, R, precision=32)
    hhg.hhg_set_streaming(S.h, 1)
    S.set_problem(f, u0)
    T.set_problem(f, u0)
    hs, cs, _ = S.solve(**kw)
    ht, ct, _ = T.solve(**kw)
    assert cs == ct and hs[-1] <= 1e-9 and np.array_equal(hs, ht)
    assert np.array_equal(S.get_solution(), T.get_solution())
    S.close()
    T.close()


def test_bounded_wait_reports_timeout_and_mesh_recovers(hhg):
    """A wait that runs out is an error status, not a hang or a fault; the
    mesh (and the GPU context) stay usable."""
    sub, R = (2, 2, 2), 6
    f = I.random_load(sub, R, seed=15)
    u0 = I.initial_guess(sub, R)
    M = hhg.Mesh(sub, R)
    hhg.hhg_set_streaming(M.h, 1)
    M.set_problem(f, u0)
    hhg.hhg_set_wait_limit(M.h, 0)
    with pytest.raises(hhg.HHGError) as e:
        M.solve(rtol=1e-8, max_cycles=5)
    assert e.value.code == hhg.HHG_ERR_TIMEOUT and "wait" in str(e.value)
    hhg.hhg_set_wait_limit(M.h, -1)
    M.set_problem(None, u0)
    m = O.Mesh(sub, R)
    uo, fo = O.pad(u0.copy()), O.pad(f)
    for _ in range(2):
        M.vcycle()
        O.vcycle(m, m.global_problem, len(m.levels) - 1, uo, fo)
    assert_close(M.get_solution(), O.interior(uo), what="after the timeout")
    M.close()
