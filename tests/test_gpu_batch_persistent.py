"""Batched recovery as ONE launch of the persistent scheduler kernel.

hhg_batch_launch_persistent runs the operations that the batch's CUDA graph
runs (recorded once at creation) inside one kernel whose CTAs take work units
from the tasks' current operations.  Each unit does the arithmetic of the
corresponding unit of the stand-alone kernel, and within an operation the
result does not depend on which CTA runs which unit (a colour's nodes only
read other colours, the transfers gather per node, the coarse CG runs in one
CTA), so the iterates must equal the graph launch's bit for bit; both are
also checked against the oracle (the fault of §2.2 followed by V-cycles of
the local Dirichlet problem, §4; the global task's V-cycles, §2.1).
"""

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


SPECS = [((1, 1, 1), 4, [2], 3), ((2, 1, 1), 5, I.grow_fault_set((2, 1, 1), 5, 7), 2),
         ((2, 2, 1), 4, I.grow_fault_set((2, 2, 1), 10, 8), 4), ((2, 2, 2), 5, I.subcube_macros((2, 2, 2)), 3)]
SHEAR = np.array([[1.0, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.1]])


def _make(hhg, specs, precision=64, mesh_kw=None):
    mesh_kw = mesh_kw or {}
    tasks, problems = [], []
    for q, (sub, R, ids, cyc) in enumerate(specs):
        f = I.random_load(sub, R, seed=60 + q)
        u0 = np.random.default_rng(70 + q).standard_normal(f.shape) * (~I.boundary_mask(sub, R))
        a = hhg.Mesh(sub, R, precision=precision, **mesh_kw)
        a.set_problem(f, u0)
        tasks.append((a, ids, cyc))
        problems.append((f, u0))
    return tasks, problems


def _reset(tasks, problems):
    for (a, _, _), (f, u0) in zip(tasks, problems):
        a.set_problem(f, u0)


def _oracle_task(sub, R, ids, cyc, f, u0, mesh_kw=None):
    m = O.Mesh(sub, R, **(mesh_kw or {}))
    uo, fo = O.pad(u0.copy()), O.pad(f)
    O.inject_fault(m, uo, ids)
    lp = m.local_problem(ids)
    for _ in range(cyc):
        O.vcycle(m, lp, len(m.levels) - 1, uo, fo)
    return O.interior(uo)


def test_persistent_equals_graph_and_oracle(hhg):
    tasks, problems = _make(hhg, SPECS)
    gsub, gR = (2, 2, 2), 5
    gf, gu0 = I.random_load(gsub, gR, seed=80), I.initial_guess(gsub, gR)
    G = hhg.Mesh(gsub, gR)
    G.set_problem(gf, gu0)
    batch = hhg.Batch(tasks, G, 2)
    n_tasks, n_ops, n_units, n_kernels = batch.info()
    assert n_tasks == len(SPECS) + 1
    # one recorded operation per kernel of the graph, plus the fault's
    # memsets (one per erased macro) that the graph holds as memset nodes
    n_erased = sum(len(ids) for _, _, ids, _ in SPECS)
    assert n_ops == n_kernels + n_erased, (n_ops, n_kernels, n_erased)
    assert n_units >= n_ops

    _reset(tasks, problems)
    G.set_problem(gf, gu0)
    batch.launch()
    graph = [a.get_solution() for a, _, _ in tasks] + [G.get_solution()]

    _reset(tasks, problems)
    G.set_problem(gf, gu0)
    ms = batch.launch_persistent()
    assert len(ms) == n_tasks and all(t > 0 for t in ms), ms
    pers = [a.get_solution() for a, _, _ in tasks] + [G.get_solution()]
    for q, (x, y) in enumerate(zip(graph, pers)):
        assert np.array_equal(x, y), f"task {q}: persistent and graph launches differ"

    for q, ((sub, R, ids, cyc), (f, u0)) in enumerate(zip(SPECS, problems)):
        assert_close(pers[q], _oracle_task(sub, R, ids, cyc, f, u0), what=f"task {q}")
    gm = O.Mesh(gsub, gR)
    gu, gfo = O.pad(gu0.copy()), O.pad(gf)
    for _ in range(2):
        O.vcycle(gm, gm.global_problem, len(gm.levels) - 1, gu, gfo)
    assert_close(pers[-1], O.interior(gu), what="global task")

    # priority classes change which CTA runs which unit when, not the results
    for prio in ([0] * len(SPECS) + [1], [1] * len(SPECS) + [0], [3, 1, 2, 0, 1]):
        batch.set_priority(prio)
        _reset(tasks, problems)
        G.set_problem(gf, gu0)
        batch.launch_persistent()
        again = [a.get_solution() for a, _, _ in tasks] + [G.get_solution()]
        for q, (x, y) in enumerate(zip(pers, again)):
            assert np.array_equal(x, y), f"task {q}, priorities {prio}"
    batch.set_priority(None)
    _reset(tasks, problems)
    G.set_problem(gf, gu0)
    batch.launch_persistent()

    # a second persistent launch repeats each task from its fault; the global
    # task runs two more cycles
    batch.launch_persistent(timed=False)
    for q, ((sub, R, ids, cyc), (f, u0)) in enumerate(zip(SPECS, problems)):
        assert np.array_equal(tasks[q][0].get_solution(), pers[q]), f"task {q}, second launch"
    for _ in range(2):
        O.vcycle(gm, gm.global_problem, len(gm.levels) - 1, gu, gfo)
    assert_close(G.get_solution(), O.interior(gu), what="global task, second launch")
    batch.close()


def test_persistent_fifteen_point_coefficients(hhg):
    """Sheared macros with per-macro coefficients: the 15-point stencil in
    every unit kind (Gauss-Seidel, residual, interface tables)."""
    specs = [((2, 1, 2), 4, I.grow_fault_set((2, 1, 2), 3, 6), 3), ((1, 2, 1), 5, [4, 5], 2)]
    tasks, problems = [], []
    for q, (sub, R, ids, cyc) in enumerate(specs):
        coeff = np.exp(np.random.default_rng(90 + q).standard_normal(6 * int(np.prod(sub))))
        kw = dict(affine=SHEAR, coeff=coeff)
        f = I.random_load(sub, R, seed=91 + q)
        u0 = np.random.default_rng(92 + q).standard_normal(f.shape) * (~I.boundary_mask(sub, R))
        a = hhg.Mesh(sub, R, **kw)
        a.set_problem(f, u0)
        tasks.append((a, ids, cyc))
        problems.append((f, u0, kw))
    batch = hhg.Batch(tasks)
    for (a, _, _), (f, u0, _) in zip(tasks, problems):
        a.set_problem(f, u0)
    batch.launch()
    graph = [a.get_solution() for a, _, _ in tasks]
    for (a, _, _), (f, u0, _) in zip(tasks, problems):
        a.set_problem(f, u0)
    batch.launch_persistent()
    for q, ((sub, R, ids, cyc), (f, u0, kw)) in enumerate(zip(specs, problems)):
        u = tasks[q][0].get_solution()
        assert np.array_equal(u, graph[q]), f"task {q}"
        assert_close(u, _oracle_task(sub, R, ids, cyc, f, u0, kw), what=f"task {q}")
    batch.close()


def test_persistent_mixed_precision_equals_graph(hhg):
    """FP32 cycles in FP64 refinement: the FP64 residual handed to FP32, the
    zeroed FP32 correction, the FP32 cycle and the FP64 update as units."""
    specs = [((2, 1, 1), 5, I.grow_fault_set((2, 1, 1), 4, 3), 4), ((2, 2, 1), 4, [9, 10, 11], 3)]
    tasks, problems = _make(hhg, specs, precision=32)
    batch = hhg.Batch(tasks, mixed=True)
    _reset(tasks, problems)
    batch.launch()
    graph = [a.get_solution() for a, _, _ in tasks]
    _reset(tasks, problems)
    batch.launch_persistent()
    for q, (a, _, _) in enumerate(tasks):
        assert np.array_equal(a.get_solution(), graph[q]), f"task {q}"
    # and close to the FP64 oracle's local cycles
    for q, ((sub, R, ids, cyc), (f, u0)) in enumerate(zip(specs, problems)):
        ref = _oracle_task(sub, R, ids, cyc, f, u0)
        assert_close(graph[q], ref, 1e-5, what=f"mixed task {q}")
    batch.close()


def test_persistent_wait_limit_reports_timeout(hhg):
    """With a wait limit of one idle round, CTAs that find no work stop and
    set the flag: the timed launch reports HHG_ERR_TIMEOUT.  The CTA that
    completes an operation always finds the next one, so the work still
    completes (the iterate equals the graph launch's), and the flag is
    cleared after it was reported."""
    tasks, problems = _make(hhg, SPECS[:2])
    for a, _, _ in tasks:
        hhg.hhg_set_wait_limit(a.h, 1)
    batch = hhg.Batch(tasks)
    _reset(tasks, problems)
    batch.launch()
    graph = [a.get_solution() for a, _, _ in tasks]
    _reset(tasks, problems)
    with pytest.raises(hhg.HHGError) as e:
        batch.launch_persistent()
    assert e.value.code == hhg.HHG_ERR_TIMEOUT
    for q, (a, _, _) in enumerate(tasks):
        assert np.array_equal(a.get_solution(), graph[q]), f"task {q}"
    batch.close()
