"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these compare the oracle with itself: each checks it against a closed
form, a dense / sparse direct solve, an algebraic identity, a geometric
definition evaluated by brute force, or values the paper prints (tests/golden).
"""

import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import hhg_inputs as I
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SHEAR = np.array([[1.0, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.1]])


def _rand_coeff(n, seed=5):
    return np.exp(np.random.default_rng(seed).standard_normal(n))


# --------------------------------------------------------------------------
# operator (§2.1 Eq. (2))
# --------------------------------------------------------------------------

@pytest.mark.parametrize("sub,r,affine", [((1, 1, 1), 2, None), ((2, 1, 1), 2, SHEAR), ((1, 2, 2), 1 + 1, SHEAR)])
def test_dia_equals_per_element_assembly(sub, r, affine):
    m_coeff = _rand_coeff(6 * sub[0] * sub[1] * sub[2])
    lv = O.Level(sub, r, m_coeff, affine)
    A_dia = O.dia_to_csr(lv)
    A_coo = O.assemble_coo(lv, m_coeff)
    assert abs(A_dia - A_coo).max() <= 1e-14 * abs(A_coo).max()


def test_element_macro_map_geometric():
    """Each fine tetrahedron's centroid lies inside the macro-tetrahedron the
    oracle assigns it to (barycentric coordinates all positive), the macro
    being spanned by 0, e_pi0, e_pi0+e_pi1, (1,1,1) in its sub-cube."""
    sub, r = (2, 1, 2), 2
    lv = O.Level(sub, r, np.ones(24))
    N = lv.N
    nx, ny, nz = lv.n
    for s, sigma in enumerate(O.PERMS):
        offs = O.hhg_oracle._kuhn_offsets(sigma)
        for cz in range(nz):
            for cy in range(ny):
                for cx in range(nx):
                    cen = np.array([cx, cy, cz], float) + np.mean(np.array(offs, float), axis=0)
                    mid = int(lv.emacro[s][cz, cy, cx])
                    sl, p = divmod(mid, 6)
                    a, rest = sl % sub[0], sl // sub[0]
                    b, c = rest % sub[1], rest // sub[1]
                    pi = O.PERMS[p]
                    v0 = np.array([a, b, c], float) * N
                    e = np.eye(3) * N
                    V = np.array([v0, v0 + e[pi[0]], v0 + e[pi[0]] + e[pi[1]], v0 + N])
                    lam = np.linalg.solve(np.vstack([V.T, np.ones(4)]), np.append(cen, 1.0))
                    assert np.all(lam > 0), (s, cx, cy, cz, mid, lam)


def test_cube_stencil_is_scaled_seven_point():
    """On the un-sheared cube with k = 2.5 the Kuhn P1 matrix is k*h times the
    7-point Laplacian at interior nodes (h = mesh width)."""
    lv = O.Level((2, 2, 2), 3, np.full(48, 2.5))
    rng = np.random.default_rng(0)
    u = rng.standard_normal(lv.pshape)
    Au = O.apply_A(lv, u)
    h = 1.0 / lv.n[0]
    c = O.interior(u)
    s = np.zeros_like(c)
    s[1:-1, 1:-1, 1:-1] = (6 * c[1:-1, 1:-1, 1:-1] - c[2:, 1:-1, 1:-1] - c[:-2, 1:-1, 1:-1]
                           - c[1:-1, 2:, 1:-1] - c[1:-1, :-2, 1:-1] - c[1:-1, 1:-1, 2:] - c[1:-1, 1:-1, :-2])
    assert np.allclose(Au[1:-1, 1:-1, 1:-1], 2.5 * h * s[1:-1, 1:-1, 1:-1], rtol=1e-13, atol=1e-13)
    assert sorted(d for d in lv.A if d != (0, 0, 0)) == sorted(
        [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)])


def test_sheared_mesh_uses_all_fifteen_offsets():
    lv = O.Level((1, 1, 1), 3, np.ones(6), SHEAR)
    assert len(lv.A) == 15


def test_symmetry_and_constants():
    lv = O.Level((2, 1, 1), 3, _rand_coeff(12), SHEAR)
    rng = np.random.default_rng(1)
    u, v = rng.standard_normal(lv.shape), rng.standard_normal(lv.shape)
    uAv = np.sum(u * O.apply_A(lv, O.pad(v)))
    vAu = np.sum(v * O.apply_A(lv, O.pad(u)))
    assert abs(uAv - vAu) <= 1e-12 * abs(uAv)
    ones = O.pad(np.ones(lv.shape))
    assert np.abs(O.apply_A(lv, ones)).max() <= 1e-13 * np.abs(lv.A[(0, 0, 0)]).max()


def test_colouring_is_proper():
    lv = O.Level((1, 1, 1), 3, np.ones(6), SHEAR)
    col = O.pad(lv.colour.astype(float) + 1.0)     # 0 in the padding
    for d, a in lv.A.items():
        if d == (0, 0, 0):
            continue
        nb = O.hhg_oracle._shift(col, d, lv)
        coupled = O.interior(a) != 0
        assert not np.any(coupled & (nb == O.interior(col)))


# --------------------------------------------------------------------------
# general macro shapes: moved macro vertices (§2.1, unstructured base mesh of a
# polyhedral domain; each macro refined uniformly through its own affine map)
# --------------------------------------------------------------------------

JSUB = (2, 2, 1)


def _jittered(sub=JSUB, move_boundary=True):
    return I.jittered_vertices(sub, seed=4, amp=0.12, move_boundary=move_boundary)


def _domain_volume(sub, vp):
    """Sum of the macro volumes from the corner positions (determinants)."""
    vol = 0.0
    for v in I.macro_vertices(sub):
        P = [np.asarray(vp[c[2], c[1], c[0]]) for c in v]
        vol += abs(np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]]))) / 6.0
    return vol


def test_moved_vertices_keep_every_macro_proper():
    for sub in [JSUB, (1, 1, 1), (3, 2, 2)]:
        vp = _jittered(sub)
        for v in I.macro_vertices(sub):
            P = [np.asarray(vp[c[2], c[1], c[0]]) for c in v]
            ref = np.linalg.det(np.stack([np.subtract(v[q], v[0]) for q in (1, 2, 3)]).astype(float))
            det = np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]]))
            assert np.sign(det) == np.sign(ref) and abs(det) > 0.2 * abs(ref) / np.prod(sub)


def test_corner_positions_of_the_cube_reproduce_the_cube_operator():
    sub = (2, 1, 2)
    k, j, i = np.meshgrid(np.arange(3), np.arange(2), np.arange(3), indexing="ij")
    vp = np.stack([i / 2, j / 1, k / 2], axis=-1)
    coeff = _rand_coeff(24, 8)
    a, b = O.Level(sub, 3, coeff), O.Level(sub, 3, coeff, vertex_pos=vp)
    assert abs(O.dia_to_csr(a) - O.dia_to_csr(b)).max() <= 1e-15 * abs(O.dia_to_csr(a)).max()


def test_moved_vertices_dia_equals_per_element_assembly():
    coeff = _rand_coeff(6 * 4)
    lv = O.Level(JSUB, 2, coeff, vertex_pos=_jittered())
    A_dia, A_coo = O.dia_to_csr(lv), O.assemble_coo(lv, coeff)
    assert abs(A_dia - A_coo).max() <= 1e-14 * abs(A_coo).max()


def test_moved_vertices_linear_kernel_and_energy_equal_the_volume():
    """For u linear in the physical coordinates, (A u)_i = 0 at every interior
    node and u^T A u = |grad u|^2 |Omega| (unit coefficient): pins the node
    positions and the element geometry against the corner positions alone."""
    vp = _jittered()
    lv = O.Level(JSUB, 3, np.ones(24), vertex_pos=vp)
    X, Y, Z = O.node_coords(lv)
    c = np.array([1.1, -0.7, 0.4])
    u = 0.3 + c[0] * X + c[1] * Y + c[2] * Z
    Au = O.apply_A(lv, O.pad(u))
    assert np.abs(Au[~lv.boundary]).max() <= 1e-13 * np.abs(lv.A[(0, 0, 0)]).max() * np.abs(u).max()
    energy = float(np.sum(u * Au))
    assert abs(energy - c @ c * _domain_volume(JSUB, vp)) <= 1e-12 * energy
    # the boundary nodes lie on the moved boundary: the cube's corners moved
    assert abs(_domain_volume(JSUB, vp) - 1.0) > 1e-3


def test_moved_vertices_general_shapes():
    lv = O.Level(JSUB, 3, np.ones(24), vertex_pos=_jittered())
    assert len(lv.A) == 15                                    # all 15 offsets
    K = lv.Kel[0]
    assert K.shape == (24, 4, 4) and np.abs(K[1:] - K[:1]).max() > 1e-3 * np.abs(K).max()
    rng = np.random.default_rng(1)
    u, v = rng.standard_normal(lv.shape), rng.standard_normal(lv.shape)
    uAv, vAu = np.sum(u * O.apply_A(lv, O.pad(v))), np.sum(v * O.apply_A(lv, O.pad(u)))
    assert abs(uAv - vAu) <= 1e-12 * abs(uAv)


def test_moved_vertices_galerkin_identity():
    coeff = _rand_coeff(24, 9)
    vp = _jittered()
    lc = O.Level(JSUB, 2, coeff, vertex_pos=vp)
    lf = O.Level(JSUB, 3, coeff, vertex_pos=vp)
    P = _prolong_matrix(lc)
    G = (P.T @ O.dia_to_csr(lf) @ P).toarray()
    Ac = O.dia_to_csr(lc).toarray()
    assert np.abs(G - Ac).max() <= 1e-13 * np.abs(Ac).max()


def test_moved_vertices_second_order_on_a_polyhedral_domain():
    """Harmonic u* = exp(pi x) sin(pi y) with Dirichlet data at the moved
    boundary nodes: the discrete L2 nodal error drops ~4x per refinement."""
    sub, errs = (1, 1, 1), []
    vp = _jittered(sub)
    for R in (4, 5, 6):
        m = O.Mesh(sub, R, vertex_pos=vp)
        X, Y, _ = O.node_coords(m.fine)
        ex = np.exp(np.pi * X) * np.sin(np.pi * Y)
        u = O.pad(I.initial_guess(sub, R, ex))
        O.solve(m, u, np.zeros(m.fine.pshape), rtol=1e-12, max_cycles=60)
        errs.append(np.sqrt(np.mean((O.interior(u) - ex) ** 2)))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.5 < q < 4.3 for q in ratios), ratios


def test_moved_vertices_vcycles_converge_to_direct_solve():
    R = 4
    m = O.Mesh(JSUB, R, coeff=_rand_coeff(24, 10), vertex_pos=_jittered(move_boundary=False))
    g = I.harmonic_boundary(JSUB, R)
    u = O.pad(I.initial_guess(JSUB, R, g))
    f = O.pad(I.random_load(JSUB, R, seed=0) * 1e-3)
    res = O.solve(m, u, f, rtol=1e-13, max_cycles=40)
    ref = _direct(m.fine, I.initial_guess(JSUB, R, g), O.interior(f), ~m.fine.boundary)
    assert np.abs(O.interior(u) - ref).max() <= 1e-10 * np.abs(ref).max()
    assert res["hist"][-1] <= 1e-13


# --------------------------------------------------------------------------
# smoother (§2.1: Gauss-Seidel, here in the 4-colour order of the reading)
# --------------------------------------------------------------------------

def _smoother_case(seed=11):
    """A small sheared mesh with random coefficients (all 15 stencil offsets),
    the oracle's colour lists of its free nodes, the per-element CSR matrix, and
    a random iterate (boundary values included) and load."""
    sub, r = (1, 2, 1), 3
    coeff = _rand_coeff(6 * 2, seed)
    m = O.Mesh(sub, r, coeff=coeff, affine=SHEAR)
    lv = m.fine
    A = O.assemble_coo(lv, coeff).tocsr()
    rng = np.random.default_rng(seed)
    u0 = rng.standard_normal(lv.shape)
    f = rng.standard_normal(lv.shape)
    f[lv.boundary] = 0.0
    return m, lv, A, u0, f


def test_gs_step_equals_a_node_by_node_sweep():
    """One step of the oracle's vectorised colour sweep equals the textbook
    Gauss-Seidel loop, u_i <- (f_i - sum_{j != i} a_ij u_j) / a_ii node after
    node, over the same nodes in colour order 0, 1, 2, 3 with the per-element
    matrix (nodes of one colour are not coupled, so only rounding differs)."""
    m, lv, A, u0, f = _smoother_case()
    u_or = O.pad(u0.copy())
    O.gs_step(lv, u_or, O.pad(f), m.global_problem.lists[-1])
    u = u0.ravel().copy()
    fr = f.ravel()
    free = (~lv.boundary).ravel()
    col = lv.colour.ravel()
    for c in range(4):
        for i in np.nonzero(free & (col == c))[0]:
            lo, hi = A.indptr[i], A.indptr[i + 1]
            js, vs = A.indices[lo:hi], A.data[lo:hi]
            aii = vs[js == i].sum()
            s = vs.dot(u[js]) - aii * u[i]
            u[i] = (fr[i] - s) / aii
    got = O.interior(u_or).ravel()
    assert np.abs(got - u).max() <= 1e-13 * np.abs(u).max()
    assert np.array_equal(got[~free], u0.ravel()[~free])      # Dirichlet nodes untouched


def test_residual_after_a_step_is_the_later_colours_updates():
    """After a full step in colour order 0..3, the residual of a colour-c node
    is -sum over later colours c' > c of a_{c c'} (u_new - u_old)_{c'}: the node
    was exact when swept, and only colours swept after it moved.  Colour 3's
    residual vanishes.  A wrong colour order or a stale neighbour value breaks
    this identity."""
    m, lv, A, u0, f = _smoother_case(seed=12)
    u = O.pad(u0.copy())
    O.gs_step(lv, u, O.pad(f), m.global_problem.lists[-1])
    un = O.interior(u).ravel()
    delta = un - u0.ravel()
    free = (~lv.boundary).ravel()
    col = lv.colour.ravel()
    r = f.ravel() - A @ un
    scale = np.abs(A @ un).max()
    for c in range(4):
        later = np.where(col > c, delta, 0.0)
        expect = -(A @ later)
        sel = free & (col == c)
        assert np.abs(r[sel] - expect[sel]).max() <= 1e-12 * scale, c
    assert np.abs(r[free & (col == 3)]).max() <= 1e-12 * scale


# --------------------------------------------------------------------------
# transfers (§2.1)
# --------------------------------------------------------------------------

def _prolong_matrix(lc):
    nz, ny, nx = lc.shape
    cols = []
    for i in range(nz * ny * nx):
        e = np.zeros(nz * ny * nx)
        e[i] = 1.0
        cols.append(O.prolong(e.reshape(lc.shape)).ravel())
    return sp.csr_matrix(np.array(cols).T)


def test_galerkin_identity():
    """P^T A_l P = A_{l-1} for nested P1 spaces with per-macro constant k."""
    coeff = _rand_coeff(12, 3)
    lc = O.Level((1, 2, 1), 2, coeff, SHEAR)
    lf = O.Level((1, 2, 1), 3, coeff, SHEAR)
    P = _prolong_matrix(lc)
    G = (P.T @ O.dia_to_csr(lf) @ P).toarray()
    Ac = O.dia_to_csr(lc).toarray()
    assert np.abs(G - Ac).max() <= 1e-13 * np.abs(Ac).max()


def test_prolongation_reproduces_linear_functions():
    lc = O.Level((2, 1, 1), 2, np.ones(12))
    z, y, x = np.indices(lc.shape).astype(float)
    lin = lambda x, y, z: 0.3 + 1.7 * x - 0.4 * y + 2.2 * z
    zf, yf, xf = np.indices(tuple(2 * s - 1 for s in lc.shape)).astype(float)
    assert np.allclose(O.prolong(lin(x, y, z)), lin(xf / 2, yf / 2, zf / 2), rtol=0, atol=1e-13)


def test_restriction_is_adjoint_of_prolongation():
    rng = np.random.default_rng(2)
    ec = rng.standard_normal((5, 9, 5))
    rf = rng.standard_normal((9, 17, 9))
    assert abs(np.sum(O.prolong(ec) * rf) - np.sum(ec * O.restrict(rf))) < 1e-12


# --------------------------------------------------------------------------
# solvers against direct solves (§2.1)
# --------------------------------------------------------------------------

def _direct(lv, u_full, f_full, free):
    A = O.dia_to_csr(lv)
    fr = free.ravel()
    ub = u_full.ravel().copy()
    rhs = f_full.ravel()[fr] - A[fr][:, ~fr] @ ub[~fr]
    ub[fr] = spla.spsolve(A[fr][:, fr].tocsc(), rhs)
    return ub.reshape(lv.shape)


def test_cg_matches_direct_solve():
    lv = O.Level((2, 2, 2), 2, _rand_coeff(48, 4))
    free = ~lv.boundary
    b = O.pad(np.random.default_rng(3).standard_normal(lv.shape))
    x, it = O.cg(lv, b, free, rtol=1e-14)
    ref = _direct(lv, np.zeros(lv.shape), O.interior(b), free)
    assert np.abs(O.interior(x) - ref).max() <= 1e-11 * np.abs(ref).max()
    assert 0 < it <= free.sum()


@pytest.mark.parametrize("coeff_seed,affine", [(None, None), (7, SHEAR)])
def test_vcycles_converge_to_direct_solve(coeff_seed, affine):
    sub, R = (2, 2, 2), 4
    coeff = None if coeff_seed is None else _rand_coeff(48, coeff_seed)
    m = O.Mesh(sub, R, coeff=coeff, affine=affine)
    g = I.harmonic_boundary(sub, R)
    u = O.pad(I.initial_guess(sub, R, g))
    f = O.pad(I.random_load(sub, R, seed=0) * 1e-3)
    res = O.solve(m, u, f, rtol=1e-13, max_cycles=40)
    ref = _direct(m.fine, I.initial_guess(sub, R, g), O.interior(f), ~m.fine.boundary)
    assert np.abs(O.interior(u) - ref).max() <= 1e-10 * np.abs(ref).max()
    assert res["hist"][-1] <= 1e-13


def test_discretisation_error_is_second_order():
    """Harmonic u* = exp(pi x) sin(pi y): max-norm error drops ~4x per refinement."""
    errs = []
    for R in (3, 4, 5):
        sub = (1, 1, 1)
        m = O.Mesh(sub, R)
        g = I.harmonic_boundary(sub, R)
        u = O.pad(I.initial_guess(sub, R, g))
        O.solve(m, u, np.zeros(m.fine.pshape), rtol=1e-12, max_cycles=40)
        errs.append(np.abs(O.interior(u) - g).max())
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.4 < q < 4.6 for q in ratios), ratios


def test_vcycle_factor_is_h_independent():
    """Textbook V(3,3) Gauss-Seidel on P1 Poisson: per-cycle residual factor
    well below 0.2 and essentially independent of the mesh size."""
    worst = []
    for R in (3, 4, 5, 6):
        sub = (2, 2, 2)
        m = O.Mesh(sub, R)
        u = O.pad(np.zeros(m.fine.shape))
        f = O.pad(I.random_load(sub, R, seed=1))
        res = O.solve(m, u, f, rtol=1e-30, max_cycles=8)
        h = res["hist"]
        worst.append(max(h[i + 1] / h[i] for i in range(2, 8)))
    assert max(worst) < 0.2, worst
    assert max(worst) / min(worst) < 2.0, worst


def test_residual_history_matches_paper_band():
    """Fault-free history of Fig. 2: every per-cycle factor of the oracle's
    V(3,3) on the 2x2x2x6 cube lies within 2x of the paper's printed factor."""
    data = np.loadtxt(os.path.join(GOLDEN, "fig2_residual_history.txt"))
    paper = data[:, 1]
    pf = paper[1:10] / paper[0:9]
    sub, R = (2, 2, 2), 5
    m = O.Mesh(sub, R)
    g = I.harmonic_boundary(sub, R)
    u = O.pad(I.initial_guess(sub, R, g))
    res = O.solve(m, u, np.zeros(m.fine.pshape), rtol=1e-30, max_cycles=9)
    h = res["hist"]
    of = h[1:10] / h[0:9]
    assert np.all(of < 2 * pf) and np.all(of > 0.5 * pf), (of, pf)


# --------------------------------------------------------------------------
# fault model and recovery (§2.2, §4.1, §4.2 Algorithm 1, Eq. (3))
# --------------------------------------------------------------------------

def test_fault_sets_integer_facts():
    m = O.Mesh((2, 2, 2), 4)
    # one macro-tetrahedron: its coarsest level (r = 2) has exactly one inner
    # node (§2.1 / §4.1); at r = 4 it has 15*14*13/6 = 455 inner nodes.
    masks = m.fault_masks([13])
    assert masks[0][0].sum() == 1
    assert masks[-1][0].sum() == 15 * 14 * 13 // 6
    # a whole interior sub-cube: (N-1)^3 inner nodes on each level
    sub = I.subcube_macros((2, 2, 2), 1, 1, 1)
    for lv, (o, c) in zip(m.levels, m.fault_masks(sub)):
        assert o.sum() == (lv.N - 1) ** 3
        assert c.sum() == (lv.N + 1) ** 3
    # fine-grid DoF of the whole problem = (2N - 1)^3
    assert (~m.fine.boundary).sum() == 31 ** 3


def _local_direct(m, u, f, ids, healthy=False):
    o, c = m.fault_masks(ids)[-1]
    free = (~m.fine.boundary & ~c) if healthy else o
    return _direct(m.fine, O.interior(u).copy(), O.interior(f), free), free


@pytest.mark.parametrize("healthy,moved", [(False, False), (True, False), (False, True), (True, True)])
def test_recovery_subproblems_converge_to_direct_solve(healthy, moved):
    """Algorithm 1: step a solves A_FF u_F = f_F - A_FG u_G, step b solves
    A_II u_I = f_I - A_IG u_G with the interface G frozen (also with moved
    sub-cube corners)."""
    sub, R = (2, 2, 2), 4
    vp = _jittered(sub) if moved else None
    m = O.Mesh(sub, R, coeff=_rand_coeff(48, 9), vertex_pos=vp)
    rng = np.random.default_rng(4)
    u = O.pad(I.initial_guess(sub, R))
    O.interior(u)[~m.fine.boundary] = rng.standard_normal((~m.fine.boundary).sum())
    f = O.pad(I.random_load(sub, R, seed=2))
    ids = I.subcube_macros(sub, 0, 0, 0) if healthy else [13]
    prob = m.healthy_problem(ids) if healthy else m.local_problem(ids)
    ref, free = _local_direct(m, u, f, ids, healthy)
    for _ in range(30):
        O.vcycle(m, prob, len(m.levels) - 1, u, f)
    assert np.abs(O.interior(u) - ref).max() <= 1e-10 * np.abs(ref).max()
    # frozen nodes untouched
    assert np.array_equal(O.interior(u)[~free], ref[~free])


def _run(m, f, rtol, **kw):
    u = O.pad(np.zeros(m.fine.shape))
    return O.solve(m, u, f, rtol=rtol, max_cycles=60, **kw)


def test_do_nothing_costs_about_kF_minus_one_cycles():
    """§2.2 / Fig. 2: after a fault at k_F = 5 the do-nothing job needs about
    k_F - 1 extra cycles; kappa close to the Tab. 1 do-nothing row."""
    sub, R = (2, 2, 2), 5
    m = O.Mesh(sub, R)
    f = O.pad(I.random_load(sub, R, seed=0))
    free = _run(m, f, 1e-10)
    dn = _run(m, f, 1e-10, fault_cycle=5, fault_ids=[13])
    extra = dn["k_faulty"] - free["cycles"]
    assert 3 <= extra <= 5, extra
    tab = np.loadtxt(os.path.join(GOLDEN, "tab1_kappa_do_nothing.txt"))
    k_dn = O.kappa(dn["k_faulty"], free["cycles"], 5)
    assert tab[0, 1] - 0.01 <= k_dn <= 1.0
    # the fault makes the residual jump by orders of magnitude (Fig. 2)
    assert dn["hist"][6] > 1e3 * dn["hist"][5]


def test_recovery_beats_do_nothing():
    sub, R = (2, 2, 2), 5
    m = O.Mesh(sub, R)
    f = O.pad(I.random_load(sub, R, seed=0))
    ids = I.subcube_macros(sub, 0, 0, 0)
    free = _run(m, f, 1e-10)["cycles"]
    dn = _run(m, f, 1e-10, fault_cycle=5, fault_ids=ids)["k_faulty"]
    lr = _run(m, f, 1e-10, fault_cycle=5, fault_ids=ids, recovery=O.LR, n_local=6)["k_faulty"]
    dd = _run(m, f, 1e-10, fault_cycle=5, fault_ids=ids, recovery=O.DD, n_global=2, eta=4.0)
    assert dd["n_F"] == 8
    kd = O.kappa(dn, free, 5)
    assert O.kappa(lr, free, 5) < kd
    assert O.kappa(dd["k_faulty"], free, 5) < kd


def test_dd_with_zero_healthy_cycles_is_do_nothing():
    sub, R = (2, 2, 2), 4
    m = O.Mesh(sub, R)
    f = O.pad(I.random_load(sub, R, seed=0))
    a = _run(m, f, 1e-10, fault_cycle=4, fault_ids=[13])
    b = _run(m, f, 1e-10, fault_cycle=4, fault_ids=[13], recovery=O.DD, n_global=0, eta=4.0)
    assert np.array_equal(a["hist"], b["hist"])


# --------------------------------------------------------------------------
# adjoint gradient
# --------------------------------------------------------------------------

def test_coefficient_gradient_matches_finite_differences():
    sub, R = (1, 1, 1), 3
    k0 = _rand_coeff(6, 11)
    f = I.random_load(sub, R, seed=3)
    tgt = I.smooth_target(sub, R)

    def fwd(k):
        lv = O.Level(sub, R, k)
        return _direct(lv, np.zeros(lv.shape), f, ~lv.boundary), lv

    u, lv = fwd(k0)
    lam = _direct(lv, np.zeros(lv.shape), u - tgt, ~lv.boundary)
    m = O.Mesh(sub, R, coeff=k0)
    g = O.grad_coeff(m, O.pad(u), O.pad(lam))
    L = lambda k: 0.5 * np.sum((fwd(k)[0] - tgt)[~lv.boundary] ** 2)
    for i in range(6):
        e = np.zeros(6)
        e[i] = 1e-6
        fd = (L(k0 + e) - L(k0 - e)) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


# --------------------------------------------------------------------------
# planted mistakes: each must be caught by one of the pins above
# --------------------------------------------------------------------------

def test_planted_restriction_mistake_is_caught(monkeypatch):
    orig = O.hhg_oracle.FREUDENTHAL
    monkeypatch.setattr(O.hhg_oracle, "FREUDENTHAL", orig[:-1])   # drop one term
    with pytest.raises(AssertionError):
        test_galerkin_identity()


def test_planted_stiffness_mistake_is_caught(monkeypatch):
    orig = O.hhg_oracle.element_stiffness
    monkeypatch.setattr(O.hhg_oracle, "element_stiffness", lambda X: orig(X).T * np.array([1, 1, 1, 1.01]))
    with pytest.raises(AssertionError):
        test_cube_stencil_is_scaled_seven_point()


def test_planted_colour_order_mistake_is_caught(monkeypatch):
    orig = O.gs_step
    monkeypatch.setattr(O, "gs_step", lambda lv, u, f, lists: orig(lv, u, f, lists[::-1]))   # colours 3..0
    with pytest.raises(AssertionError):
        test_residual_after_a_step_is_the_later_colours_updates()
    with pytest.raises(AssertionError):
        test_gs_step_equals_a_node_by_node_sweep()


def test_planted_dropped_neighbour_is_caught(monkeypatch):
    orig = O.gs_step

    def dropped(lv, u, f, lists):
        d = next(k for k in lv.A if k != (0, 0, 0))
        saved = lv.A.pop(d)                       # the sweep forgets one neighbour
        try:
            orig(lv, u, f, lists)
        finally:
            lv.A[d] = saved

    monkeypatch.setattr(O, "gs_step", dropped)
    with pytest.raises(AssertionError):
        test_gs_step_equals_a_node_by_node_sweep()


def test_local_residual_equals_assembled_residual():
    """The per-node row assembly used for sampled checks on large meshes agrees
    with the full DIA residual (itself pinned to the per-element COO above)."""
    sub, R = (2, 1, 2), 3
    c = _rand_coeff(24, 0)
    m = O.Mesh(sub, R, coeff=c, affine=SHEAR)
    rng = np.random.default_rng(1)
    u, f = rng.standard_normal(m.fine.shape), rng.standard_normal(m.fine.shape)
    r = O.residual(m.fine, O.pad(u), O.pad(f), ~m.fine.boundary)
    nodes = np.array([[1, 1, 1], [5, 3, 7], [8, 4, 8], [15, 7, 15], [8, 1, 9]])
    got = O.local_residual(sub, R, c, SHEAR, u, f, nodes)
    assert np.abs(got - np.array([r[z, y, x] for x, y, z in nodes])).max() <= 1e-14


# --------------------------------------------------------------------------
# Dirichlet-Neumann recovery (§4.3, Algorithm 2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("moved", [False, True])
def test_dn_neumann_subproblem_converges_to_direct_solve(moved):
    """With many cycles, Omega_I solves A_I [u_I; u_G] = [f_I; b_G] (A_I from
    the healthy macros' elements, b_G = (A_I u)_G at the fault) and Omega_F
    the Dirichlet problem with the final interface values (also with moved
    sub-cube corners)."""
    sub, R = (2, 2, 2), 4
    m = O.Mesh(sub, R, coeff=_rand_coeff(48, 12), vertex_pos=_jittered(sub) if moved else None)
    rng = np.random.default_rng(5)
    u = O.pad(I.initial_guess(sub, R))
    O.interior(u)[~m.fine.boundary] = rng.standard_normal((~m.fine.boundary).sum())
    f = O.pad(I.random_load(sub, R, seed=4))
    ids = I.subcube_macros(sub, 1, 0, 0)
    hm = O.hhg_oracle.healthy_mesh(m, ids)
    o, c = m.fault_masks(ids)[-1]
    gamma = c & ~o & ~m.fine.boundary
    b = O.interior(f).copy()
    b[gamma] = O.apply_A(hm.fine, u)[gamma]
    free_i = ~m.fine.boundary & ~o
    O.inject_fault(m, u, ids)
    ref_i = _direct(hm.fine, O.interior(u).copy(), b, free_i)
    O.dn_recover(m, u, f, ids, n_global=30, eta=1.0, hmesh=hm)
    assert np.abs(O.interior(u)[free_i] - ref_i[free_i]).max() <= 1e-10 * np.abs(ref_i).max()
    ref_f = _direct(m.fine, O.interior(u).copy(), O.interior(f), o)
    assert np.abs(O.interior(u)[o] - ref_f[o]).max() <= 1e-9 * np.abs(ref_f).max()


def test_dn_recovers_an_exact_solution():
    """A fault on the exact discrete solution: the frozen flux is the exact one,
    so Omega_I stays exact and Omega_F is rebuilt to it."""
    sub, R = (2, 2, 2), 4
    m = O.Mesh(sub, R)
    f = O.pad(I.random_load(sub, R, seed=9))
    ustar = O.pad(_direct(m.fine, np.zeros(m.fine.shape), O.interior(f), ~m.fine.boundary))
    u = ustar.copy()
    ids = [13, 14]
    O.inject_fault(m, u, ids)
    O.dn_recover(m, u, f, ids, n_global=12, eta=3.0)
    assert np.abs(O.interior(u) - O.interior(ustar)).max() <= 1e-9 * np.abs(ustar).max()


def test_dn_beats_do_nothing():
    sub, R = (2, 2, 2), 5
    m = O.Mesh(sub, R)
    f = O.pad(I.random_load(sub, R, seed=0))
    ids = I.subcube_macros(sub, 0, 0, 0)
    free = _run(m, f, 1e-10)["cycles"]
    dn = _run(m, f, 1e-10, fault_cycle=5, fault_ids=ids)["k_faulty"]
    r = _run(m, f, 1e-10, fault_cycle=5, fault_ids=ids, recovery=O.DN, n_global=2, eta=4.0)
    assert r["n_F"] == 8
    assert O.kappa(r["k_faulty"], free, 5) < O.kappa(dn, free, 5)


def test_two_faults_equal_the_sequence_of_single_fault_steps():
    """A second fault after the first recovery (§5): the listed faults give the
    iterate of running cycles, fault, recovery, cycles, fault, recovery by
    hand."""
    sub, R = (2, 2, 2), 4
    m = O.Mesh(sub, R)
    f = O.pad(I.random_load(sub, R, seed=6))
    u = O.pad(I.initial_guess(sub, R))
    r = O.solve(m, u, f, rtol=1e-30, max_cycles=8, fault_cycle=3, fault_ids=[13], recovery=O.DD, n_global=1,
                eta=2.0, faults=[(6, [40, 41])])
    assert len(r["hist"]) == 8 + 1 + 2 and r["k_faulty"] == 8 + 2
    v = O.pad(I.initial_guess(sub, R))
    top = len(m.levels) - 1
    for k in range(1, 9):
        O.vcycle(m, m.global_problem, top, v, f)
        if k in (3, 6):
            ids = [13] if k == 3 else [40, 41]
            O.inject_fault(m, v, ids)
            for _ in range(2):
                O.vcycle(m, m.local_problem(ids), top, v, f)
            O.vcycle(m, m.healthy_problem(ids), top, v, f)
    assert np.abs(O.interior(v) - O.interior(u)).max() == 0.0


def test_strategy_ordering_of_the_cycle_advantage():
    """§4.4 and Tab. 1: for every superman factor and n_I, DN is at least as
    good as DD and DD at least as good as LR, none is worse than do-nothing
    (n_I = 0), and with n_I >= 1 each beats do-nothing; scenarios I (refined
    5 times) and II (refined 4 times), fault after 5 cycles."""
    import math
    for si, (name, sub, ids) in enumerate(I.kappa_scenarios()[:2]):
        R = 5 if si == 0 else 4
        m = O.Mesh(sub, R)
        f = O.pad(I.random_load(sub, R, seed=0))
        u0 = O.pad(I.initial_guess(sub, R))
        free = O.solve(m, u0.copy(), f, rtol=1e-10, max_cycles=60)["cycles"]
        for eta in (2.0, 5.0):
            nothing = None
            for n_I in range(4):
                kap = []
                for rec in (O.LR, O.DD, O.DN):
                    kw = dict(fault_cycle=5, fault_ids=ids, recovery=rec)
                    if rec == O.LR:
                        kw["n_local"] = int(math.ceil(eta * n_I))
                    else:
                        kw.update(n_global=n_I, eta=eta)
                    r = O.solve(m, u0.copy(), f, rtol=1e-10, max_cycles=60, **kw)
                    kap.append(O.kappa(r["cycles"] + n_I, free, 5))
                if n_I == 0:
                    nothing = kap[0]
                    assert kap == [nothing] * 3
                else:
                    assert kap[2] <= kap[1] <= kap[0] < nothing, (name, eta, n_I, kap)
