"""The dynamic unit walk of the level-wide kernels, at sizes the oracle checks.

A level-wide launch (Gauss-Seidel colour, residual, restriction,
prolongation, the FP32/FP64 hand-over of mixed precision) walks its work
units with a grid stride when it has fewer than 4 units per CTA and hands
them out through a per-problem atomic counter otherwise.  With the grid the
GPU holds at once, only meshes refined 8 or more times reach the dynamic walk
(the benchmark's size); hhg_set_launch_limit caps the CTAs per launch so that
refinements 4-6 take it as well.  Each test
  * asserts through hhg_walk_counts that the dynamic walk ran (and that
    without the cap it did not, at these sizes),
  * compares the iterates with the oracle node by node (parity.assert_close),
  * and compares them with a twin mesh that takes the grid-stride walk: the
    iterate of a V-cycle does not depend on the order in which the units are
    handed out (a colour's nodes only read other colours, the transfers are
    gathers per node, the coarse CG runs in one CTA), so the two must agree
    bit for bit.  A unit skipped or handed out twice would change the
    prolongation's sums or the residual norm.
(§2.1 V-cycle; §4.2 Algorithm 1; §4.3 Algorithm 2.)
"""

import numpy as np
import pytest

import hhg_inputs as I
import oracle as O
from parity import assert_close

pytestmark = pytest.mark.gpu

SHEAR = np.array([[1.0, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.1]])
ATOL_HIST = 1e-12


@pytest.fixture(scope="module")
def hhg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1506_06185_gb300 import build
    from paper_1506_06185_gb300 import hhg as H
    build()
    return H


def _twins(hhg, sub, R, f, u0, cap, **mesh_kw):
    """A mesh limited to `cap` CTAs per launch (dynamic walk) and a twin with
    the default grid (grid-stride walk at these sizes), same problem."""
    D = hhg.Mesh(sub, R, **mesh_kw)
    S = hhg.Mesh(sub, R, **mesh_kw)
    hhg.hhg_set_launch_limit(D.h, cap)
    for M in (D, S):
        M.set_problem(f, u0)
    return D, S


@pytest.mark.parametrize("sub,R,cap,shear", [((2, 2, 2), 5, 8, False), ((3, 2, 2), 6, 24, False),
                                             ((2, 1, 2), 5, 4, True)])
def test_dynamic_walk_vcycles(hhg, sub, R, cap, shear):
    f = I.random_load(sub, R, seed=3)
    u0 = I.initial_guess(sub, R, I.harmonic_boundary(sub, R))
    kw = dict(affine=SHEAR, coeff=np.exp(np.random.default_rng(2).standard_normal(6 * np.prod(sub)))) if shear \
        else {}
    D, S = _twins(hhg, sub, R, f, u0, cap, **kw)
    m = O.Mesh(sub, R, **kw)
    uo, fo = O.pad(u0.copy()), O.pad(f)
    r0 = O.resnorm(m, uo, fo)
    top = len(m.levels) - 1
    for k in range(4):
        rd = D.vcycle()
        rs = S.vcycle()
        O.vcycle(m, m.global_problem, top, uo, fo)
        ud, us = D.get_solution(), S.get_solution()
        assert_close(ud, O.interior(uo), what=f"cycle {k}")
        assert np.array_equal(ud, us), f"cycle {k}: dynamic and grid-stride walks differ"
        ro = O.resnorm(m, uo, fo)
        assert abs(rd - ro) <= ATOL_HIST * r0 and abs(rs - ro) <= ATOL_HIST * r0, k
    dyn = hhg.hhg_walk_counts(D.h)
    stride = hhg.hhg_walk_counts(S.h)
    # per cycle and level at least the 4 x 6 Gauss-Seidel launches walk dynamically
    assert dyn[0] >= 4 * 24, dyn
    assert stride[0] == 0, stride
    D.close()
    S.close()


def _solve_both(hhg, sub, R, f, u0, cap, kw, mesh_kw=None):
    mesh_kw = mesh_kw or {}
    D, S = _twins(hhg, sub, R, f, u0, cap, **mesh_kw)
    hd, cd, _ = D.solve(**kw)
    hs, cs, _ = S.solve(**kw)
    m = O.Mesh(sub, R, **mesh_kw)
    uo = O.pad(u0.copy())
    okw = dict(rtol=kw["rtol"], max_cycles=kw["max_cycles"], fault_cycle=kw.get("fault_cycle", -1),
               fault_ids=kw.get("fault_ids", ()), recovery=kw.get("recovery", 0), n_local=kw.get("n_local", 0),
               n_global=kw.get("n_global", 0), eta=kw.get("eta", 1.0))
    ref = O.solve(m, uo, O.pad(f), **okw)
    assert cd == cs == ref["cycles"]
    assert np.abs(hd - ref["hist"]).max() <= ATOL_HIST
    ud, us = D.get_solution(), S.get_solution()
    assert_close(ud, O.interior(uo), what="solve")
    assert np.array_equal(ud, us)
    counts = hhg.hhg_walk_counts(D.h)
    D.close()
    S.close()
    return counts


def test_dynamic_walk_local_recovery(hhg):
    """LR after a fault of two macros: n_F = 3 local cycles on Omega_F (4
    tiles per macro at refinement 5, so 2 CTAs walk 8 units dynamically)."""
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=4)
    counts = _solve_both(hhg, sub, R, f, I.initial_guess(sub, R), 2,
                         dict(rtol=1e-10, max_cycles=40, fault_cycle=4, fault_ids=[13, 14], recovery=1,
                              n_local=3))
    assert counts[0] > 0 and counts[1] > 0, counts


def test_dynamic_walk_dirichlet_dirichlet(hhg):
    """DD (Algorithm 1) on a sub-cube: both concurrent sides take the dynamic walk."""
    sub, R = (2, 2, 2), 6
    f = I.random_load(sub, R, seed=5)
    counts = _solve_both(hhg, sub, R, f, I.initial_guess(sub, R), 4,
                         dict(rtol=1e-9, max_cycles=40, fault_cycle=3, fault_ids=I.subcube_macros(sub, 1, 0, 1),
                              recovery=2, n_global=2, eta=3.0))
    assert counts[0] > 0 and counts[1] > 0 and counts[2] > 0, counts


def test_dynamic_walk_dirichlet_neumann_sheared(hhg):
    """DN (Algorithm 2) on a sheared 15-point mesh with coefficients."""
    sub, R = (3, 2, 2), 5
    f = I.random_load(sub, R, seed=6)
    coeff = np.exp(np.random.default_rng(7).standard_normal(72))
    counts = _solve_both(hhg, sub, R, f, I.initial_guess(sub, R), 3,
                         dict(rtol=1e-9, max_cycles=40, fault_cycle=3, fault_ids=[13, 14, 30, 31], recovery=3,
                              n_global=2, eta=2.0), dict(affine=SHEAR, coeff=coeff))
    assert counts[0] > 0 and counts[1] > 0 and counts[3] > 0, counts


def test_dynamic_walk_mixed_precision(hhg):
    """FP32 cycles inside FP64 refinement (the FP32/FP64 hand-over kernels walk
    dynamically too): both walks give the same bits, the same cycle count and
    the stopping test of the FP64 oracle."""
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=8)
    u0 = I.initial_guess(sub, R)
    kw = dict(rtol=1e-10, max_cycles=40, fault_cycle=4, fault_ids=I.subcube_macros(sub), recovery=2, n_global=2,
              eta=4.0, mixed_precision=True)
    D, S = _twins(hhg, sub, R, f, u0, 6, precision=32)
    hd, cd, _ = D.solve(**kw)
    hs, cs, _ = S.solve(**kw)
    # the norms' partial sums follow the grid, so the histories agree to rounding
    assert cd == cs and np.abs(hd - hs).max() <= 1e-14 and hd[-1] <= 1e-10
    assert np.array_equal(D.get_solution(), S.get_solution())
    assert hhg.hhg_walk_counts(D.h)[0] > 0
    D.close()
    S.close()


def test_launch_limit_rejects_negative(hhg):
    M = hhg.Mesh((1, 1, 1), 3)
    with pytest.raises(hhg.HHGError) as e:
        hhg.hhg_set_launch_limit(M.h, -1)
    assert e.value.code == hhg.HHG_ERR_ARG
    M.close()
