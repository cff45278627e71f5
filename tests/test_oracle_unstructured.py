"""Pins of the general-mesh oracle (oracle/unstructured.py) against facts the
mathematics fixes: the cube family given as a general mesh reproduces the
structured oracle; node counts of the macro mesh's primitives; linear
functions and the energy-volume identity; the Galerkin identity; proper
smoother classes and a brute-force Gauss-Seidel sweep; V-cycles = direct
solve; second-order discretisation error (§2.1); fault sets equal to the
structured ones on the cube family, a faulty macro losing exactly its volume
nodes, LR / DD / DN sub-problems = direct solves, recovery beating
do-nothing (§2.2, Algorithms 1 and 2)."""

import itertools

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import hhg_inputs as I
import oracle as O
from oracle import unstructured as U


def _coeff(n, seed):
    return np.exp(np.random.default_rng(seed).standard_normal(n))


@pytest.fixture(scope="module")
def five():
    v, t = I.five_tet_macro_mesh((2, 2, 2), seed=3, amp=0.12)
    return U.UMesh(v, t, 4, coeff=_coeff(len(t), 2))


def test_cube_family_as_a_general_mesh_reproduces_the_structured_oracle():
    sub, R = (2, 1, 2), 3
    coeff = _coeff(24, 1)
    v, t = I.kuhn_macro_mesh(sub)
    um = U.UMesh(v, t, R, coeff=coeff)
    sm = O.Mesh(sub, R, coeff=coeff)
    for lu, ls in zip(um.levels, sm.levels):
        nx, ny, nz = ls.n
        g = np.rint(lu.X * np.array([nx, ny, nz])).astype(np.int64)
        gid = (g[:, 2] * (ny + 1) + g[:, 1]) * (nx + 1) + g[:, 0]
        assert len(np.unique(gid)) == lu.n == (nx + 1) * (ny + 1) * (nz + 1)
        A_s = O.dia_to_csr(ls)[gid][:, gid]
        assert abs(lu.A - A_s).max() <= 1e-14 * abs(A_s).max()
        assert np.array_equal(lu.boundary, ls.boundary.ravel()[gid])
    # interpolation: the same as the structured grid's
    lc, lf = sm.levels[0], sm.levels[1]
    ec = np.random.default_rng(2).standard_normal(lc.shape)
    gc = np.rint(um.levels[0].X * np.array(lc.n)).astype(np.int64)
    gf = np.rint(um.levels[1].X * np.array(lf.n)).astype(np.int64)
    eu = um.P[0] @ ec[gc[:, 2], gc[:, 1], gc[:, 0]]
    assert np.abs(eu - O.prolong(ec)[gf[:, 2], gf[:, 1], gf[:, 0]]).max() <= 1e-15


@pytest.mark.parametrize("kind", ["five", "kuhn-moved"])
def test_node_counts_match_the_macro_primitives(kind):
    if kind == "five":
        v, t = I.five_tet_macro_mesh((2, 1, 2))
    else:
        v, t = I.kuhn_macro_mesh((2, 2, 1))
        v = I.jittered_vertices((2, 2, 1), seed=4).reshape(-1, 3)
    E = {e for tt in t for e in itertools.combinations(sorted(tt), 2)}
    F = {f for tt in t for f in itertools.combinations(sorted(tt), 3)}
    m = U.UMesh(v, t, 3)
    for lv in m.levels:
        N = lv.N
        assert lv.n == len(v) + len(E) * (N - 1) + len(F) * (N - 1) * (N - 2) // 2 + \
            len(t) * (N - 1) * (N - 2) * (N - 3) // 6
        assert len(np.unique(np.round(lv.X, 12), axis=0)) == lv.n     # no two nodes coincide
    # the macros tile the domain: their volumes add up to its volume
    vol = sum(abs(np.linalg.det((v[tt[1:]] - v[tt[0]]).T)) / 6.0 for tt in t)
    if kind == "five":
        assert abs(vol - 1.0) < 1e-12


def test_linear_functions_and_energy(five):
    lv = five.levels[-1]
    c = np.array([0.8, -1.3, 0.5])
    m1 = U.UMesh(five.verts, five.tets, 3)                # unit coefficient
    l1 = m1.levels[-1]
    u = 0.2 + l1.X @ c
    Au = l1.A @ u
    assert np.abs(Au[~l1.boundary]).max() <= 1e-13 * l1.diag.max() * np.abs(u).max()
    vol = sum(abs(np.linalg.det((five.verts[t[1:]] - five.verts[t[0]]).T)) / 6.0 for t in five.tets)
    assert abs(u @ Au - (c @ c) * vol) <= 1e-12 * (c @ c) * vol
    assert abs(lv.A - lv.A.T).max() <= 1e-15 * abs(lv.A).max()


def test_galerkin_identity_and_linear_interpolation(five):
    for l in range(1, len(five.levels)):
        P = five.P[l - 1]
        G = (P.T @ five.levels[l].A @ P).toarray()
        Ac = five.levels[l - 1].A.toarray()
        assert np.abs(G - Ac).max() <= 1e-13 * np.abs(Ac).max()
        lin = lambda X: 0.3 + X @ np.array([1.7, -0.4, 2.2])
        assert np.abs(P @ lin(five.levels[l - 1].X) - lin(five.levels[l].X)).max() <= 1e-13


def test_smoother_classes_are_independent_and_cover_the_free_nodes(five):
    for lv in five.levels:
        allc = np.concatenate(lv.classes)
        assert np.array_equal(np.sort(allc), np.nonzero(~lv.boundary)[0])
        for cls in lv.classes:
            block = lv.A[cls][:, cls]
            assert (block != 0).sum() == len(cls)        # only the diagonal couples a class
        assert lv.n_interface_classes >= 3


def test_gs_step_equals_a_node_by_node_sweep(five):
    lv = five.levels[0]
    rng = np.random.default_rng(7)
    u0, f = rng.standard_normal(lv.n), rng.standard_normal(lv.n)
    free = ~lv.boundary
    u = u0.copy()
    U.gs_step(lv, u, f, free)
    ref = u0.copy()
    A = lv.A.toarray()
    for cls in lv.classes:
        for i in cls[::-1]:                                # any order within a class
            ref[i] = (f[i] - A[i] @ ref + A[i, i] * ref[i]) / A[i, i]
    assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max()


def test_vcycles_converge_to_the_direct_solve(five):
    lv = five.levels[-1]
    free = ~lv.boundary
    rng = np.random.default_rng(3)
    f = rng.uniform(-1, 1, lv.n) * 1e-3
    f[~free] = 0.0
    g = np.exp(np.pi * lv.X[:, 0]) * np.sin(np.pi * lv.X[:, 1])
    u = np.where(free, 0.0, g)
    hist = U.solve(five, u, f, rtol=1e-12, max_cycles=40)
    ref = u.copy()
    ref[free] = spla.spsolve(lv.A[free][:, free].tocsc(), f[free] - lv.A[free][:, ~free] @ g[~free])
    assert np.abs(u - ref).max() <= 1e-9 * np.abs(ref).max()
    factors = hist[1:] / hist[:-1]
    assert factors[1:].max() < 0.35, factors


def test_second_order_error_on_a_general_mesh():
    v, t = I.five_tet_macro_mesh((1, 1, 1), seed=5, amp=0.0)
    errs = []
    for R in (3, 4, 5):
        m = U.UMesh(v, t, R)
        lv = m.levels[-1]
        ex = np.exp(np.pi * lv.X[:, 0]) * np.sin(np.pi * lv.X[:, 1])
        u = np.where(lv.boundary, ex, 0.0)
        U.solve(m, u, np.zeros(lv.n), rtol=1e-12, max_cycles=60)
        errs.append(np.sqrt(np.mean((u - ex) ** 2)))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.4 < q < 4.4 for q in ratios), ratios


# --------------------------------------------------------------------------
# faults and recovery (§2.2, Algorithms 1 and 2) on general meshes
# --------------------------------------------------------------------------

def test_fault_sets_on_the_cube_family_equal_the_structured_ones():
    sub, R = (2, 2, 1), 3
    v, t = I.kuhn_macro_mesh(sub)
    um, sm = U.UMesh(v, t, R), O.Mesh(sub, R)
    ids = [3, 4, 5, 9]
    for lu, ls, (ou, cu), (os_, cs) in zip(um.levels, sm.levels, um.fault_masks(ids), sm.fault_masks(ids)):
        nx, ny, nz = ls.n
        g = np.rint(lu.X * np.array([nx, ny, nz])).astype(np.int64)
        gid = (g[:, 2] * (ny + 1) + g[:, 1]) * (nx + 1) + g[:, 0]
        assert np.array_equal(ou, os_.ravel()[gid]) and np.array_equal(cu, cs.ravel()[gid])


def test_one_faulty_macro_loses_exactly_its_volume_nodes(five):
    for lv, (o, c) in zip(five.levels, five.fault_masks([7])):
        N = lv.N
        assert o.sum() == (N - 1) * (N - 2) * (N - 3) // 6
        assert c.sum() == (N + 1) * (N + 2) * (N + 3) // 6      # its closed lattice
        assert np.all(lv.dim[o] == 4)


def _direct_sub(lv, u, f, free):
    ref = u.copy()
    ref[free] = spla.spsolve(lv.A[free][:, free].tocsc(), f[free] - lv.A[free][:, ~free] @ u[~free])
    return ref


@pytest.mark.parametrize("which", ["local", "healthy"])
def test_recovery_subproblems_converge_to_direct_solves(five, which):
    lv = five.levels[-1]
    rng = np.random.default_rng(11)
    u = np.where(lv.boundary, 0.0, rng.standard_normal(lv.n))
    f = rng.uniform(-1, 1, lv.n)
    ids = [0, 1, 2, 3, 4]                                  # one sub-cube's five macros
    masks = five.local_masks(ids) if which == "local" else five.healthy_masks(ids)
    ref = _direct_sub(lv, u, f, masks[-1])
    for _ in range(30):
        U.vcycle(five, len(five.levels) - 1, u, f, masks)
    assert np.abs(u - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.array_equal(u[~masks[-1]], ref[~masks[-1]])    # frozen nodes untouched


def test_dn_neumann_subproblem_converges_to_its_direct_solve(five):
    lv = five.levels[-1]
    rng = np.random.default_rng(12)
    u = np.where(lv.boundary, 0.0, rng.standard_normal(lv.n))
    f = rng.uniform(-1, 1, lv.n)
    ids = [5, 6, 7, 8, 9]
    hm = five.healthy(ids)
    o, c = five.fault_masks(ids)[-1]
    gamma = c & ~o & ~lv.boundary
    b = f.copy()
    b[gamma] = (hm.levels[-1].A @ u)[gamma]
    free_i = ~lv.boundary & ~o
    U.inject_fault(five, u, ids)
    ref_i = _direct_sub(hm.levels[-1], u, b, free_i)
    U.dn_recover(five, u, f, ids, n_global=30, eta=1.0)
    assert np.abs(u[free_i] - ref_i[free_i]).max() <= 1e-10 * np.abs(ref_i).max()
    ref_f = _direct_sub(lv, u, f, o)
    assert np.abs(u[o] - ref_f[o]).max() <= 1e-9 * np.abs(ref_f).max()


def test_recovery_beats_do_nothing_on_a_general_mesh(five):
    lv = five.levels[-1]
    f = np.where(lv.boundary, 0.0, np.random.default_rng(13).uniform(-1, 1, lv.n))
    ids = [10, 11, 12, 13, 14]
    runs = {}
    for name, kw in [("free", {}), ("none", dict(recovery=U.NONE)), ("lr", dict(recovery=U.LR, n_local=4)),
                     ("dd", dict(recovery=U.DD, n_global=2, eta=3.0)), ("dn", dict(recovery=U.DN, n_global=2, eta=3.0))]:
        u = np.zeros(lv.n)
        fk = dict(fault_cycle=4, fault_ids=ids) if name != "free" else {}
        h = U.solve(five, u, f, rtol=1e-10, max_cycles=40, **fk, **kw)
        runs[name] = len(h) - 1 - (1 if fk else 0)          # global cycles
    assert runs["none"] > runs["free"]
    assert runs["dd"] <= runs["lr"] <= runs["none"] and runs["dn"] <= runs["none"]
    assert runs["dd"] < runs["none"]
