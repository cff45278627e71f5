"""Dirichlet-Neumann recovery (§4.3, Algorithm 2) on the GPU against the
oracle's ``dn_recover``: the Omega_I Neumann problem under A_I with the
frozen interface flux, Omega_F Dirichlet blocks of ceil(j eta) - ceil((j-1)
eta) cycles on the Gamma values of the previous Omega_I cycle.  FP64 iterates
must agree within a relative 1e-12, residual histories within 1e-12."""

import numpy as np
import pytest

import hhg_inputs as I
import oracle as O
from parity import assert_close

pytestmark = pytest.mark.gpu

SHEAR = np.array([[1.0, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.1]])
RTOL_U = 1e-12
ATOL_HIST = 1e-12


@pytest.fixture(scope="module")
def hhg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1506_06185_gb300 import build
    from paper_1506_06185_gb300 import hhg as H
    build()
    return H


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _recover(hhg, sub, R, ids, n_global, eta, coeff=None, affine=None, seed=5, before=3):
    f = I.random_load(sub, R, seed=seed)
    M = hhg.Mesh(sub, R, coeff=coeff, affine=affine)
    M.set_problem(f, I.initial_guess(sub, R))
    m = O.Mesh(sub, R, coeff=coeff, affine=affine)
    uo, fo = O.pad(I.initial_guess(sub, R)), O.pad(f)
    top = len(m.levels) - 1
    for _ in range(before):
        M.vcycle()
        O.vcycle(m, m.global_problem, top, uo, fo)
    M.inject_fault(ids)
    O.inject_fault(m, uo, ids)
    nf, tl, tg = M.recover_dn(ids, n_global, eta, timed=True)
    nf_o = O.dn_recover(m, uo, fo, ids, n_global, eta)
    assert nf == nf_o
    assert_close(M.get_solution(), O.interior(uo), RTOL_U, what="after DN recovery")
    # the global iteration resumes from consistent ghost copies
    M.vcycle()
    O.vcycle(m, m.global_problem, top, uo, fo)
    assert_close(M.get_solution(), O.interior(uo), RTOL_U, what="next global cycle")
    M.close()
    return nf, tl, tg


def test_dn_subcube_matches_oracle(hhg):
    sub, R = (2, 2, 2), 5
    nf, tl, tg = _recover(hhg, sub, R, I.subcube_macros(sub, 1, 0, 1), n_global=3, eta=1.5)
    assert nf == 5 and tl > 0 and tg > 0


def test_dn_sheared_coefficients_scattered_faults(hhg):
    """15-point stencils, per-macro coefficients, two separate faulty regions
    and interface nodes with several faulty and healthy copies."""
    sub, R = (3, 2, 2), 5
    coeff = np.exp(np.random.default_rng(3).standard_normal(72))
    _recover(hhg, sub, R, [13, 14, 30, 31, 50], n_global=4, eta=2.0, coeff=coeff, affine=SHEAR, seed=2)


def test_dn_degenerate_schedules(hhg):
    """eta = 0 (Omega_F never runs), n_global = 0 (nothing runs) and a fault
    of every macro (Omega_I is empty)."""
    sub, R = (2, 2, 2), 4
    assert _recover(hhg, sub, R, [13], n_global=2, eta=0.0)[0] == 0
    assert _recover(hhg, sub, R, [13], n_global=0, eta=3.0)[0] == 0
    assert _recover(hhg, (1, 1, 1), 3, list(range(6)), n_global=2, eta=2.0)[0] == 4


def test_dn_invalid_arguments(hhg):
    M = hhg.Mesh((1, 1, 1), 3)
    for args in (([0], -1, 1.0), ([0], 1, -1.0), ([0], 1, float("nan")), ([6], 1, 1.0), ([], 1, 1.0)):
        with pytest.raises(hhg.HHGError) as e:
            M.recover_dn(*args)
        assert e.value.code == hhg.HHG_ERR_ARG
    M.close()


def test_solve_dn_history_matches_oracle(hhg):
    """hhg_solve with DN after cycle 5 on a sub-cube: identical cycle counts,
    residual histories and final iterate."""
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=0)
    ids = I.subcube_macros(sub)
    kw = dict(rtol=1e-10, max_cycles=40, fault_cycle=5, fault_ids=ids, recovery=3, n_global=2, eta=4.0)
    M = hhg.Mesh(sub, R)
    M.set_problem(f, I.initial_guess(sub, R))
    hist, cyc, _ = M.solve(**kw)
    m = O.Mesh(sub, R)
    uo = O.pad(I.initial_guess(sub, R))
    ref = O.solve(m, uo, O.pad(f), **kw)
    assert cyc == ref["cycles"] and len(hist) == len(ref["hist"])
    assert np.abs(hist - ref["hist"]).max() <= ATOL_HIST
    assert_close(M.get_solution(), O.interior(uo), RTOL_U, what="DN solve")
    M.close()


def test_mixed_precision_dn(hhg):
    """DN inside FP64 iterative refinement with FP32 inner cycles: same stopping
    test and cycle count within one of the FP64 oracle."""
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=4)
    ids = I.subcube_macros(sub, 0, 1, 0)
    kw = dict(rtol=1e-10, max_cycles=40, fault_cycle=5, fault_ids=ids, recovery=3, n_global=2, eta=4.0)
    M = hhg.Mesh(sub, R, precision=32)
    M.set_problem(f, I.initial_guess(sub, R))
    hist, cyc, _ = M.solve(mixed_precision=True, **kw)
    m = O.Mesh(sub, R)
    uo = O.pad(I.initial_guess(sub, R))
    ref = O.solve(m, uo, O.pad(f), **kw)
    assert hist[-1] <= 1e-10 and abs(cyc - ref["cycles"]) <= 1
    # right after the recovery the FP32 inner cycles leave the residual within
    # a few per cent of the FP64 one
    k = kw["fault_cycle"] + 1
    assert abs(hist[k] / ref["hist"][k] - 1.0) < 0.05, (hist[k], ref["hist"][k])
    assert_close(M.get_solution(), O.interior(uo), 1e-8, what="mixed DN solve")
    M.close()


@pytest.mark.parametrize("recovery", [2, 3])
def test_two_faults_match_oracle(hhg, recovery):
    """A second fault at another location after the first recovery (§5),
    DD and DN: same cycle count, residual history and iterate as the oracle."""
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=8)
    kw = dict(rtol=1e-10, max_cycles=40, fault_cycle=3, fault_ids=[13], recovery=recovery, n_global=2, eta=2.0,
              faults=[(6, I.subcube_macros(sub, 1, 1, 1))])
    M = hhg.Mesh(sub, R)
    M.set_problem(f, I.initial_guess(sub, R))
    hist, cyc, _ = M.solve(**kw)
    m = O.Mesh(sub, R)
    uo = O.pad(I.initial_guess(sub, R))
    ref = O.solve(m, uo, O.pad(f), **kw)
    assert cyc == ref["cycles"] and len(hist) == len(ref["hist"]) == cyc + 3
    assert np.abs(hist - ref["hist"]).max() <= ATOL_HIST
    assert_close(M.get_solution(), O.interior(uo), RTOL_U, what="two faults")
    with pytest.raises(hhg.HHGError) as e:
        M.solve(rtol=1e-10, max_cycles=5, faults=[(0, [1])])
    assert e.value.code == hhg.HHG_ERR_ARG
    M.close()


def test_dn_after_new_coefficients(hhg):
    """The Neumann-side operator A_I follows hhg_set_coefficients: a DN recovery
    after a coefficient change matches the oracle built with the new ones."""
    sub, R = (2, 2, 2), 4
    ids = [13, 14]
    k1 = np.exp(np.random.default_rng(1).standard_normal(48))
    k2 = np.exp(np.random.default_rng(2).standard_normal(48))
    f = I.random_load(sub, R, seed=9)
    M = hhg.Mesh(sub, R, coeff=k1)
    M.set_problem(f, I.initial_guess(sub, R))
    M.vcycle()
    M.inject_fault(ids)
    M.recover_dn(ids, 2, 2.0)
    M.set_coefficients(k2)
    M.set_problem(f, I.initial_guess(sub, R))
    m = O.Mesh(sub, R, coeff=k2)
    uo, fo = O.pad(I.initial_guess(sub, R)), O.pad(f)
    top = len(m.levels) - 1
    for _ in range(2):
        M.vcycle()
        O.vcycle(m, m.global_problem, top, uo, fo)
    M.inject_fault(ids)
    O.inject_fault(m, uo, ids)
    M.recover_dn(ids, 2, 2.0)
    O.dn_recover(m, uo, fo, ids, 2, 2.0)
    assert_close(M.get_solution(), O.interior(uo), RTOL_U, what="DN after new coefficients")
    M.close()


def test_fault_sets_replace_each_other_without_growing_memory(hhg):
    """Arming the mesh for another fault set frees the previous set's
    sub-problems: device memory returns to the same size for the same set."""
    sub, R = (2, 2, 2), 4
    M = hhg.Mesh(sub, R)
    M.set_problem(I.random_load(sub, R, seed=1), I.initial_guess(sub, R))
    sizes = []
    for ids in ([13], I.subcube_macros(sub, 1, 1, 1), [3, 4, 40], [13]):
        M.vcycle()
        M.inject_fault(ids)
        M.recover_local(ids, 2, 1)
        M.recover_dn(ids, 1, 2.0)
        sizes.append(M.bytes())
    assert sizes[3] == sizes[0], sizes
    M.close()
