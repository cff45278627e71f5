"""GPU parity on a macro mesh of general connectivity (five tetrahedra per
sub-cube, corners moved): the CUDA path through the C ABI
(hhg_mesh_create_general) against the general-mesh oracle
(oracle/unstructured.py), V-cycle by V-cycle (§2.1).  Library and oracle
order the nodes differently; the test maps them through the node keys
(interface nodes in the same key order, then the volume nodes macro by macro
in local (k, j, i) order)."""

import numpy as np
import pytest

import hhg_inputs as I
from parity import assert_close
from oracle import unstructured as U

pytestmark = pytest.mark.gpu

RTOL_U = 1e-12


@pytest.fixture(scope="module")
def hhg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1506_06185_gb300 import build
    from paper_1506_06185_gb300 import hhg as H
    build()
    return H


def lib_to_oracle(om, tets):
    """Library node order -> oracle node id."""
    lv = om.levels[-1]
    N = lv.N
    n_if = int((lv.dim < 4).sum())
    okeys = {tuple(k): q for q, k in enumerate(lv.keys.tolist())}
    perm = list(range(n_if))
    for t in tets:
        for k in range(1, N):
            for j in range(1, N - k):
                for i in range(1, N - j - k):
                    w = [N - i - j - k, i, j, k]
                    perm.append(okeys[(4, *sorted(int(g) * (N + 1) + ww for g, ww in zip(t, w)))])
    return np.array(perm)


def test_general_mesh_vcycles_match_oracle(hhg):
    v, t = I.five_tet_macro_mesh((2, 2, 1), seed=3, amp=0.12)
    R = 4
    om = U.UMesh(v, t, R)
    lv = om.levels[-1]
    perm = lib_to_oracle(om, t)
    fo = np.where(lv.boundary, 0.0, np.random.default_rng(5).uniform(-1, 1, lv.n))
    uo = np.where(lv.boundary, np.exp(np.pi * lv.X[:, 0]) * np.sin(np.pi * lv.X[:, 1]), 0.0)
    M = hhg.Mesh.general(v, t, R)
    assert M.n_nodes == lv.n and M.n_dof == int((~lv.boundary).sum())
    M.set_problem(np.ascontiguousarray(fo[perm]), np.ascontiguousarray(uo[perm]))
    masks = om.global_masks()
    r0 = U.resnorm(om, uo, fo)
    assert abs(M.residual_norm() - r0) <= 1e-13 * r0
    for c in range(3):
        rg = M.vcycle()
        U.vcycle(om, len(om.levels) - 1, uo, fo, masks)
        ug = M.get_solution()
        assert_close(ug, uo[perm], RTOL_U, what=f"cycle {c}")
        assert abs(rg - U.resnorm(om, uo, fo)) <= 1e-12 * r0, c
    M.close()


@pytest.mark.parametrize("recovery,ids", [("LR", [5, 6, 7, 8, 9]), ("DD", [5, 6, 7, 8, 9]), ("DN", [5, 6, 7, 8, 9]),
                                          ("DD", [7, 12]), ("DN", [0, 13])])
def test_general_mesh_fault_recovery_matches_oracle(hhg, recovery, ids):
    """A fault after global cycle 2 (§2.2) on one sub-cube's five macros or on
    scattered macros, recovered by LR, DD (Algorithm 1) or DN (Algorithm 2),
    then global cycles to 1e-10: the same cycle count, residual history and
    iterate, node by node, as the general-mesh oracle's solve."""
    v, t = I.five_tet_macro_mesh((2, 2, 1), seed=3, amp=0.12)
    R = 4
    om = U.UMesh(v, t, R)
    lv = om.levels[-1]
    perm = lib_to_oracle(om, t)
    fo = np.where(lv.boundary, 0.0, np.random.default_rng(8).uniform(-1, 1, lv.n))
    uo = np.zeros(lv.n)
    M = hhg.Mesh.general(v, t, R)
    M.set_problem(np.ascontiguousarray(fo[perm]), np.ascontiguousarray(uo[perm]))
    kw = {"LR": dict(recovery=U.LR, n_local=3), "DD": dict(recovery=U.DD, n_local=3, n_global=2),
          "DN": dict(recovery=U.DN, n_global=2, eta=2.5)}[recovery]
    hist, cyc, _ = M.solve(rtol=1e-10, max_cycles=40, fault_cycle=2, fault_ids=ids, **kw)
    hist_o = U.solve(om, uo, fo, rtol=1e-10, max_cycles=40, fault_cycle=2, fault_ids=ids, **kw)
    assert len(hist) == len(hist_o) and cyc == len(hist_o) - 2
    assert np.abs(hist - hist_o).max() <= 1e-12, np.abs(hist - hist_o).max()
    assert_close(M.get_solution(), uo[perm], RTOL_U, what=f"{recovery} solve")
    M.close()
