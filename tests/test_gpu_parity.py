"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 iterates must agree cycle by cycle within a relative 1e-12 (the
tolerance the method's FP64 path is held to); relative residual histories
within 1e-12 absolute (they are normalised by the initial residual, so this
is a relative bound on the residual vector's rounding noise, which is of order
1e-16 * ||A|| ||u||).  Cycle counts and the fault / recovery schedule must be
identical.
"""

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


def _coeff(n, seed):
    return np.exp(np.random.default_rng(seed).standard_normal(n))


def _compare_cycles(hhg, sub, R, f, u0, coeff=None, affine=None, cycles=6, device_ptrs=False):
    import torch
    M = hhg.Mesh(sub, R, coeff=coeff, affine=affine)
    if device_ptrs:
        M.set_problem(torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda())
    else:
        M.set_problem(f, u0)
    m = O.Mesh(sub, R, coeff=coeff, affine=affine)
    uo, fo = O.pad(u0.copy()), O.pad(f)
    r0 = O.resnorm(m, uo, fo)
    assert abs(M.residual_norm() - r0) <= 1e-13 * r0
    top = len(m.levels) - 1
    for k in range(cycles):
        rg = M.vcycle()
        O.vcycle(m, m.global_problem, top, uo, fo)
        if device_ptrs:
            ug = torch.zeros(M.shape, dtype=torch.float64, device="cuda")
            M.get_solution(ug)
            ug = ug.cpu().numpy()
        else:
            ug = M.get_solution()
        assert_close(ug, O.interior(uo), RTOL_U, what=f"cycle {k}")
        assert abs(rg - O.resnorm(m, uo, fo)) <= ATOL_HIST * r0, k
    M.close()


def test_vcycles_config1_harmonic(hhg):
    """2x2x2x6 macros refined 4 times, harmonic Dirichlet data, f = 0."""
    sub, R = (2, 2, 2), 4
    g = I.harmonic_boundary(sub, R)
    _compare_cycles(hhg, sub, R, np.zeros(g.shape), I.initial_guess(sub, R, g), cycles=8)


def test_vcycles_device_pointers_random_load(hhg):
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=0)
    _compare_cycles(hhg, sub, R, f, I.initial_guess(sub, R), cycles=5, device_ptrs=True)


def test_vcycles_fifteen_point_sheared_coefficients(hhg):
    """Sheared mesh: all 15 stencil weights non-zero; per-macro coefficients."""
    sub, R = (2, 1, 2), 5
    f = I.random_load(sub, R, seed=4)
    g = I.harmonic_boundary(sub, R)
    _compare_cycles(hhg, sub, R, f, I.initial_guess(sub, R, g), coeff=_coeff(24, 5), affine=SHEAR, cycles=5)


def test_vcycles_larger_mesh_ragged_tiles(hhg):
    sub, R = (3, 2, 2), 6
    f = I.random_load(sub, R, seed=7)
    _compare_cycles(hhg, sub, R, f, I.initial_guess(sub, R), coeff=_coeff(72, 8), cycles=3)


def _compare_solve(hhg, sub, R, f, u0, coeff=None, affine=None, **kw):
    M = hhg.Mesh(sub, R, coeff=coeff, affine=affine)
    M.set_problem(f, u0)
    hist, cyc, _ = M.solve(**kw)
    m = O.Mesh(sub, R, coeff=coeff, affine=affine)
    uo = O.pad(u0.copy())
    okw = dict(rtol=kw["rtol"], max_cycles=kw["max_cycles"], fault_cycle=kw.get("fault_cycle", -1),
               fault_ids=kw.get("fault_ids", ()), recovery=kw.get("recovery", 0), n_local=kw.get("n_local", 0),
               n_global=kw.get("n_global", 0), eta=kw.get("eta", 1.0))
    ref = O.solve(m, uo, O.pad(f), **okw)
    assert cyc == ref["cycles"]
    assert len(hist) == len(ref["hist"])
    assert np.abs(hist - ref["hist"]).max() <= ATOL_HIST, np.abs(hist - ref["hist"]).max()
    ug = M.get_solution()
    assert_close(ug, O.interior(uo), RTOL_U, what="solve")
    M.close()
    return hist, ref


def test_solve_config1_fault_local_recovery(hhg):
    """Config 1 end to end: fault after cycle 5 zeroes macro-tet 0, LR with
    2 local V-cycles, stop at 1e-10."""
    sub, R = (2, 2, 2), 4
    g = I.harmonic_boundary(sub, R)
    hist, ref = _compare_solve(hhg, sub, R, np.zeros(g.shape), I.initial_guess(sub, R, g), rtol=1e-10,
                               max_cycles=40, fault_cycle=5, fault_ids=[0], recovery=1, n_local=2)
    assert hist[-1] <= 1e-10


def test_solve_dirichlet_dirichlet_subcube(hhg):
    """DD recovery (Algorithm 1) of a whole sub-cube, eta = 4, n_I = 2."""
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=0)
    _compare_solve(hhg, sub, R, f, I.initial_guess(sub, R), rtol=1e-10, max_cycles=40, fault_cycle=5,
                   fault_ids=I.subcube_macros(sub), recovery=2, n_global=2, eta=4.0)


def test_solve_do_nothing_interior_tet(hhg):
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=1)
    _compare_solve(hhg, sub, R, f, I.initial_guess(sub, R), rtol=1e-10, max_cycles=40, fault_cycle=4,
                   fault_ids=[13], recovery=0)


def test_solve_dd_sheared_scattered_faults(hhg):
    sub, R = (3, 2, 2), 5
    f = I.random_load(sub, R, seed=2)
    _compare_solve(hhg, sub, R, f, I.initial_guess(sub, R), coeff=_coeff(72, 3), affine=SHEAR, rtol=1e-9,
                   max_cycles=40, fault_cycle=3, fault_ids=[13, 14, 30, 31], recovery=2, n_global=1, n_local=3)


def test_fault_everything_and_degenerate_calls(hhg):
    """All macros faulty: the healthy problem is empty and DD still works;
    invalid fault lists are rejected."""
    sub, R = (1, 1, 1), 3
    f = I.random_load(sub, R, seed=3)
    _compare_solve(hhg, sub, R, f, I.initial_guess(sub, R), rtol=1e-9, max_cycles=40, fault_cycle=2,
                   fault_ids=list(range(6)), recovery=2, n_global=2, n_local=3)
    M = hhg.Mesh(sub, R)
    for bad in ([], [6], [1, 1], [-1]):
        with pytest.raises(hhg.HHGError) as e:
            M.inject_fault(bad)
        assert e.value.code == hhg.HHG_ERR_ARG
    M.close()


def test_recover_local_matches_oracle_and_reports_times(hhg):
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=5)
    M = hhg.Mesh(sub, R)
    M.set_problem(f, I.initial_guess(sub, R))
    m = O.Mesh(sub, R)
    uo, fo = O.pad(I.initial_guess(sub, R)), O.pad(f)
    top = len(m.levels) - 1
    for _ in range(3):
        M.vcycle()
        O.vcycle(m, m.global_problem, top, uo, fo)
    ids = I.subcube_macros(sub, 1, 0, 1)
    M.inject_fault(ids)
    O.inject_fault(m, uo, ids)
    assert_close(M.get_solution(), O.interior(uo), RTOL_U, what="after the fault")
    tl, tg = M.recover_local(ids, 4, 2, timed=True)
    assert tl > 0 and tg > 0
    lp, hp = m.local_problem(ids), m.healthy_problem(ids)
    for _ in range(4):
        O.vcycle(m, lp, top, uo, fo)
    for _ in range(2):
        O.vcycle(m, hp, top, uo, fo)
    assert_close(M.get_solution(), O.interior(uo), RTOL_U, what="after DD recovery")
    M.close()


def test_replayed_local_cycles_match_oracle_and_count_launches(hhg):
    # the later local cycles of a recovery replay one captured cycle; a second
    # recovery on the same fault set reuses it, and every replayed kernel
    # counts as a launch
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=6)
    M = hhg.Mesh(sub, R)
    M.set_problem(f, I.initial_guess(sub, R))
    m = O.Mesh(sub, R)
    uo, fo = O.pad(I.initial_guess(sub, R)), O.pad(f)
    top = len(m.levels) - 1
    M.vcycle()
    O.vcycle(m, m.global_problem, top, uo, fo)
    ids = I.subcube_macros(sub, 0, 1, 1)
    M.inject_fault(ids)
    O.inject_fault(m, uo, ids)
    lp = m.local_problem(ids)
    deltas = []
    for n in (1, 3, 5, 3):
        l0 = hhg.hhg_launch_count()
        M.recover_local(ids, n, 0)
        deltas.append(hhg.hhg_launch_count() - l0)
        for _ in range(n):
            O.vcycle(m, lp, top, uo, fo)
        assert_close(M.get_solution(), O.interior(uo), RTOL_U, what=f"{n} local cycles")
    per_cycle = (deltas[1] - deltas[0]) // 2
    assert per_cycle > 0
    assert deltas[1] - deltas[0] == 2 * per_cycle
    assert deltas[2] - deltas[1] == 2 * per_cycle
    assert deltas[3] == deltas[1]
    M.close()


@pytest.mark.slow
def test_full_size_config2_sampled_residual(hhg):
    """2x2x2x6 macros refined 8 times (1.3e8 unknowns): converge on the GPU,
    then the oracle's residual, assembled row by row at sampled nodes, must be
    at the converged level (a wrong stencil anywhere sampled would leave O(1)
    residuals), and the per-cycle factors must stay in the V(3,3) band."""
    sub, R = (2, 2, 2), 8
    f = I.random_load(sub, R, seed=0)
    M = hhg.Mesh(sub, R)
    M.set_problem(f, I.initial_guess(sub, R))
    hist, cyc, _ = M.solve(rtol=1e-10, max_cycles=30)
    factors = hist[1:] / hist[:-1]
    assert np.all(factors[1:] < 0.2) and hist[-1] <= 1e-10, hist
    u = M.get_solution()
    r0 = np.linalg.norm(f[~I.boundary_mask(sub, R)])
    rng = np.random.default_rng(11)
    n = 1 << R
    nodes = rng.integers(1, 2 * n, size=(300, 3))
    # include nodes on macro faces / edges / vertices (interior of the domain)
    nodes[:40] = np.maximum((nodes[:40] // 4) * 4, 4)
    nodes[40:60, 0] = n
    assert nodes.min() >= 1 and nodes.max() <= 2 * n - 1
    r = O.local_residual(sub, R, np.ones(48), None, u, f, nodes)
    assert np.abs(r).max() <= 2e-10 * r0, np.abs(r).max() / r0
    M.close()
