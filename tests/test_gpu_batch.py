"""Batched recovery in one CUDA-graph launch, and the tile autotuner.

A batch runs its tasks with the same kernels as the one-at-a-time calls, so
its results must equal those of hhg_inject_fault + hhg_recover_local (and of
hhg_vcycle for the global task) on twin meshes; the autotuner only changes
tile shapes, so V-cycles after tuning still match the oracle."""

import numpy as np
import pytest

import hhg_inputs as I
import oracle as O
from parity import assert_close

pytestmark = pytest.mark.gpu


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


def test_batch_matches_sequential_recovery(hhg):
    specs = [((1, 1, 1), 4, [2], 3), ((2, 1, 1), 5, I.grow_fault_set((2, 1, 1), 5, 7), 2),
             ((2, 2, 1), 4, I.grow_fault_set((2, 2, 1), 10, 8), 3)]
    tasks, twins = [], []
    for q, (sub, R, ids, cyc) in enumerate(specs):
        f = I.random_load(sub, R, seed=10 + q)
        u0 = np.random.default_rng(q).standard_normal(f.shape) * (~I.boundary_mask(sub, R))
        a, b = hhg.Mesh(sub, R), hhg.Mesh(sub, R)
        a.set_problem(f, u0)
        b.set_problem(f, u0)
        tasks.append((a, ids, cyc))
        twins.append((b, ids, cyc))
    gsub, gR = (2, 2, 2), 5
    gf = I.random_load(gsub, gR, seed=20)
    G, G2 = hhg.Mesh(gsub, gR), hhg.Mesh(gsub, gR)
    G.set_problem(gf, I.initial_guess(gsub, gR))
    G2.set_problem(gf, I.initial_guess(gsub, gR))
    batch = hhg.Batch(tasks, G, 2)
    ms = batch.launch()
    assert len(ms) == 4 and all(t > 0 for t in ms)
    for (a, ids, cyc), (b, _, _) in zip(tasks, twins):
        b.inject_fault(ids)
        b.recover_local(ids, cyc)
        assert _rel(a.get_solution(), b.get_solution()) <= 1e-13
    for _ in range(4):   # two cycles at creation (the uncaptured pass) and two per launch
        G2.vcycle()
    assert _rel(G.get_solution(), G2.get_solution()) <= 1e-13
    batch.close()


def test_batch_matches_oracle(hhg):
    """Every task of an FP64 batch against the oracle: the fault of §2.2
    (O.inject_fault) followed by the same number of V-cycles of the local
    Dirichlet problem (O.local_problem); the global task against the same
    number of global V-cycles.  The creation pass and each launch both start
    a task from the fault, which erases what the previous pass recovered, so
    after any number of launches a task holds fault + cycles from its
    initial iterate; the global task has run 2 + 2 cycles after one launch."""
    specs = [((1, 1, 1), 4, [2], 3), ((2, 1, 1), 5, I.grow_fault_set((2, 1, 1), 5, 7), 2),
             ((2, 2, 1), 4, I.grow_fault_set((2, 2, 1), 10, 8), 4), ((2, 2, 2), 4, I.subcube_macros((2, 2, 2)), 3)]
    tasks, refs = [], []
    for q, (sub, R, ids, cyc) in enumerate(specs):
        f = I.random_load(sub, R, seed=30 + q)
        u0 = np.random.default_rng(40 + q).standard_normal(f.shape) * (~I.boundary_mask(sub, R))
        a = hhg.Mesh(sub, R)
        a.set_problem(f, u0)
        tasks.append((a, ids, cyc))
        m = O.Mesh(sub, R)
        uo, fo = O.pad(u0.copy()), O.pad(f)
        O.inject_fault(m, uo, ids)
        lp = m.local_problem(ids)
        for _ in range(cyc):
            O.vcycle(m, lp, len(m.levels) - 1, uo, fo)
        refs.append(O.interior(uo))
    gsub, gR = (2, 2, 2), 5
    gf = I.random_load(gsub, gR, seed=50)
    G = hhg.Mesh(gsub, gR)
    G.set_problem(gf, I.initial_guess(gsub, gR))
    gm = O.Mesh(gsub, gR)
    gu, gfo = O.pad(I.initial_guess(gsub, gR)), O.pad(gf)
    for _ in range(4):
        O.vcycle(gm, gm.global_problem, len(gm.levels) - 1, gu, gfo)
    batch = hhg.Batch(tasks, G, 2)
    batch.launch()
    for q, ((a, _, _), ref) in enumerate(zip(tasks, refs)):
        assert_close(a.get_solution(), ref, 1e-12, what=f"task {q}")
    assert_close(G.get_solution(), O.interior(gu), 1e-12, what="global task")
    # a second launch repeats the tasks from their faults: same iterates
    batch.launch()
    for q, ((a, _, _), ref) in enumerate(zip(tasks, refs)):
        assert_close(a.get_solution(), ref, 1e-12, what=f"task {q}, second launch")
    batch.close()


def test_batch_mixed_precision_matches_oracle(hhg):
    """A mixed-precision batch (FP32 cycles inside FP64 refinement): after ten
    local cycles from the fault, the recovered iterate agrees with ten FP64
    oracle cycles of the same local problem to the level both have reached
    (the local V(3,3) cycles contract the error by 0.1 or better per cycle, so
    each is within 1e-9 of the local solution), and the residual returns to
    its level before the fault."""
    sub, R = (2, 1, 1), 5
    f = I.random_load(sub, R, seed=3)
    M = hhg.Mesh(sub, R, precision=32)
    M.set_problem(f, I.initial_guess(sub, R))
    M.solve(rtol=1e-6, max_cycles=20)
    u_start = M.get_solution()
    r_before = M.residual_norm()
    ids = I.grow_fault_set(sub, 4, 3)
    cyc = 10
    m = O.Mesh(sub, R)
    uo, fo = O.pad(u_start.copy()), O.pad(f)
    O.inject_fault(m, uo, ids)
    lp = m.local_problem(ids)
    for _ in range(cyc):
        O.vcycle(m, lp, len(m.levels) - 1, uo, fo)
    batch = hhg.Batch([(M, ids, cyc)], mixed=True)
    ms = batch.launch()
    assert ms[0] > 0
    assert_close(M.get_solution(), O.interior(uo), 1e-8, what="mixed batch task")
    assert M.residual_norm() <= 10 * r_before
    batch.close()


def test_batch_mixed_precision_runs(hhg):
    sub, R = (2, 1, 1), 5
    f = I.random_load(sub, R, seed=3)
    M = hhg.Mesh(sub, R, precision=32)
    M.set_problem(f, I.initial_guess(sub, R))
    M.solve(rtol=1e-6, max_cycles=20)
    r_before = M.residual_norm()
    ids = I.grow_fault_set(sub, 4, 3)
    batch = hhg.Batch([(M, ids, 6)], mixed=True)
    ms = batch.launch()
    assert ms[0] > 0
    # six local cycles after the fault bring the residual back near its old level
    assert M.residual_norm() <= 10 * r_before
    batch.close()


def test_autotune_keeps_parity(hhg):
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=1)
    M = hhg.Mesh(sub, R, precision=32)
    chosen = hhg.hhg_autotune(M.h, R - 1, reps=2)
    assert chosen[0] == -1 and all(0 <= c < 8 for c in chosen[1:])
    M.set_problem(f, I.initial_guess(sub, R))
    m = O.Mesh(sub, R)
    uo, fo = O.pad(I.initial_guess(sub, R)), O.pad(f)
    for _ in range(3):
        M.vcycle()
        O.vcycle(m, m.global_problem, len(m.levels) - 1, uo, fo)
    assert_close(M.get_solution(), O.interior(uo), 1e-12, what="after autotuning")
    M.close()
