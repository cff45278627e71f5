"""Plain FP64 CPU multigrid oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this module.  It shares no code with the CUDA path.

Reference: Huber, Gmeiner, Ruede, Wohlmuth, "Resilience for Multigrid Software
at the Extreme Scale".  Each function names the passage it follows.

Representation
--------------
A level is the global node grid of the cube family: ``sub = (sx, sy, sz)``
sub-cubes, each split into the six Kuhn tetrahedra sharing the main diagonal
(these are the macro elements, the base mesh of §2.1), refined ``r`` times.
Refinement ``r`` gives ``N = 2**r`` intervals per sub-cube edge and a grid of
``(sx*N+1) x (sy*N+1) x (sz*N+1)`` nodes; the fine tetrahedra are the Kuhn
simplices of every grid cell (the Freudenthal triangulation).  Arrays are
stored z-major / x-fastest with one layer of zero padding on every side, so a
node (x, y, z) sits at ``a[1+z, 1+y, 1+x]``.

The operator is assembled element by element (P1 stiffness
``k_T |T| grad(lambda_i).grad(lambda_j)``, §2.1 Eq. (2)) into a
sparse-diagonal (DIA) form: one padded array per neighbour offset.  A
per-element COO assembly into scipy CSR exists for tiny meshes and is used by
the tests to check the DIA form.

Parity status
-------------
Every function below is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py`` (closed forms, dense direct solves, Galerkin
identities, textbook convergence bands, the paper's Fig. 2 / Tab. 1 bands).
``kappa`` matching the paper's Tab. 1 entries exactly is not claimed: the
paper's "hybrid" Gauss-Seidel ordering is not specified, so the oracle's
cycle counts are only pinned to the paper's qualitative band.
"""

from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "PERMS", "FREUDENTHAL", "Level", "Mesh", "Problem",
    "element_stiffness", "assemble_coo", "dia_to_csr", "apply_A",
    "gs_step", "residual", "restrict", "prolong", "cg", "vcycle",
    "resnorm", "inject_fault", "solve", "kappa", "grad_coeff",
    "interior", "pad", "node_coords", "macro_maps", "NONE", "LR", "DD", "DN", "local_residual", "dn_recover",
]

# Lexicographic permutations of the axes (x=0, y=1, z=2).  Kuhn tetrahedron
# number p of a sub-cube has vertices 0, e_pi0, e_pi0 + e_pi1, (1,1,1).
PERMS = list(itertools.permutations((0, 1, 2)))
# Edge directions of the Freudenthal triangulation: all non-zero 0/1 vectors,
# written (dx, dy, dz).
FREUDENTHAL = [d for d in itertools.product((0, 1), repeat=3) if any(d)]

NONE, LR, DD, DN = 0, 1, 2, 3


def _e(a):
    v = [0, 0, 0]
    v[a] = 1
    return tuple(v)


def _kuhn_offsets(sigma):
    """Vertex offsets (dx, dy, dz) of the Kuhn simplex with axis order sigma."""
    o1 = _e(sigma[0])
    o2 = tuple(a + b for a, b in zip(o1, _e(sigma[1])))
    return [(0, 0, 0), o1, o2, (1, 1, 1)]


def interior(a):
    """View of a padded array without its one-node padding layer."""
    return a[1:-1, 1:-1, 1:-1]


def pad(a):
    """Copy of a grid array with one layer of zero padding."""
    out = np.zeros(tuple(s + 2 for s in a.shape))
    out[1:-1, 1:-1, 1:-1] = a
    return out


def element_stiffness(X):
    """P1 element stiffness of one tetrahedron, unit coefficient (§2.1).

    ``X`` holds the four vertex positions (rows).  With E the matrix whose
    columns are the edge vectors X_a - X_0, the gradients of the barycentric
    coordinates lambda_1..3 are the rows of E^-1 and grad(lambda_0) is minus
    their sum; K_ab = |T| grad(lambda_a) . grad(lambda_b), |T| = |det E| / 6.
    """
    X = np.asarray(X, dtype=np.float64)
    E = (X[1:] - X[0]).T
    Einv = np.linalg.inv(E)
    D = np.vstack([-Einv.sum(axis=0), Einv])
    vol = abs(np.linalg.det(E)) / 6.0
    return vol * (D @ D.T)


def macro_maps(sub, affine=None, vertex_pos=None):
    """Affine map of every macro-tetrahedron from sub-cube units to physical
    space (§2.1: the base mesh is a tetrahedral mesh of a polyhedral domain and
    every refinement is uniform inside a macro, so each macro's fine nodes are
    the image of its reference lattice under that macro's affine map).

    Macro t = 6 * sub-cube + Kuhn type has integer corner coordinates
    V_0..V_3 (0, e_pi0, e_pi0 + e_pi1, (1,1,1) shifted to its sub-cube).
    ``vertex_pos`` (shape (sz+1, sy+1, sx+1, 3), or None) gives the physical
    position of every sub-cube corner; without it the corners sit at
    G (V / sub), G = ``affine`` (identity if None).  Returns (V0, P0, M) with
    x(s) = P0[t] + M[t] (s - V0[t]) for a point s in sub-cube units.
    """
    sx, sy, sz = (int(q) for q in sub)
    G = np.eye(3) if affine is None else np.asarray(affine, dtype=np.float64)[:3, :3]
    n = 6 * sx * sy * sz
    V0 = np.zeros((n, 3))
    P0 = np.zeros((n, 3))
    M = np.zeros((n, 3, 3))
    scale = np.array([sx, sy, sz], dtype=np.float64)
    for c in range(sz):
        for b in range(sy):
            for a in range(sx):
                for p, sigma in enumerate(PERMS):
                    t = ((c * sy + b) * sx + a) * 6 + p
                    corners = [np.array((a, b, c)) + np.array(o) for o in _kuhn_offsets(sigma)]
                    if vertex_pos is None:
                        P = [G @ (v / scale) for v in corners]
                    else:
                        P = [np.asarray(vertex_pos[v[2], v[1], v[0]], dtype=np.float64) for v in corners]
                    EV = np.stack([corners[q] - corners[0] for q in (1, 2, 3)], axis=1).astype(np.float64)
                    EP = np.stack([P[q] - P[0] for q in (1, 2, 3)], axis=1)
                    V0[t], P0[t] = corners[0], P[0]
                    M[t] = EP @ np.linalg.inv(EV)
    return V0, P0, M


class Level:
    """One refinement level of the cube macro mesh (§2.1, uniform refinement).

    Attributes: ``A`` (dict offset -> padded coefficient array), ``boundary``,
    ``colour`` ((x+y+z) mod 4), ``emacro`` (macro id of every fine tetrahedron,
    per Kuhn type), ``Kel`` (unit-coefficient element stiffness per Kuhn type:
    one 4x4 matrix when the mesh is an affine image of the uniform grid, else
    an array (n_macro, 4, 4), one per macro, from ``vertex_pos``).
    """

    def __init__(self, sub, r, coeff, affine=None, vertex_pos=None):
        sx, sy, sz = (int(s) for s in sub)
        self.sub = (sx, sy, sz)
        self.n_macro = 6 * sx * sy * sz
        self.r = int(r)
        N = 1 << self.r
        self.N = N
        self.n = (sx * N, sy * N, sz * N)
        nx, ny, nz = self.n
        self.shape = (nz + 1, ny + 1, nx + 1)
        self.pshape = (nz + 3, ny + 3, nx + 3)
        self.Px, self.Py = nx + 3, ny + 3
        G = np.eye(3) if affine is None else np.asarray(affine, dtype=np.float64)[:, :3]
        self.G = G

        # Macro id of each fine tetrahedron.  The fine simplex (cell c, type
        # sigma) has centroid c + (3 e_s0 + 2 e_s1 + e_s2)/4; inside its
        # sub-cube it lies in the Kuhn macro whose axis order sorts that
        # centroid's local coordinates in decreasing order.
        lz, ly, lx = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
        lut = np.zeros(27, dtype=np.int64)
        for i, p in enumerate(PERMS):
            lut[p[0] * 9 + p[1] * 3 + p[2]] = i
        cz, cy, cx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        slin = ((cz // N) * sy + (cy // N)) * sx + (cx // N)
        self.emacro = []
        for sigma in PERMS:
            pos = [sigma.index(a) for a in range(3)]
            keys = np.stack([4 * lx + 3 - pos[0], 4 * ly + 3 - pos[1], 4 * lz + 3 - pos[2]], axis=-1)
            order = np.argsort(-keys, axis=-1, kind="stable")
            pidx = lut[order[..., 0] * 9 + order[..., 1] * 3 + order[..., 2]]
            self.emacro.append((slin * 6 + np.tile(pidx, (sz, sy, sx))).astype(np.int32))
        del lz, ly, lx, cz, cy, cx, slin

        # Unit-coefficient element stiffness of the six Kuhn types: for an
        # affine image of the uniform grid it does not depend on the cell; with
        # moved macro vertices it depends on the macro (its affine map).
        h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
        self.vertex_pos = vertex_pos
        self.Kel = []
        if vertex_pos is None:
            for sigma in PERMS:
                X = np.array([G @ (np.array(o) * h) for o in _kuhn_offsets(sigma)])
                self.Kel.append(element_stiffness(X))
        else:
            self.maps = macro_maps(self.sub, None, vertex_pos)
            M = self.maps[2]
            for sigma in PERMS:
                offs = [np.array(o, dtype=np.float64) / N for o in _kuhn_offsets(sigma)]
                self.Kel.append(np.stack([element_stiffness(np.array([M[t] @ o for o in offs]))
                                          for t in range(self.n_macro)]))

        self.A = self._assemble_dia(np.asarray(coeff, dtype=np.float64))
        self.off = {d: d[2] * self.Py * self.Px + d[1] * self.Px + d[0] for d in self.A}

        z, y, x = np.indices(self.shape)
        self.boundary = (x == 0) | (x == nx) | (y == 0) | (y == ny) | (z == 0) | (z == nz)
        self.colour = (x + y + z) % 4
        self.xyz = (x, y, z)

    def _cell_slice(self, o):
        nx, ny, nz = self.n
        return (slice(1 + o[2], 1 + o[2] + nz), slice(1 + o[1], 1 + o[1] + ny),
                slice(1 + o[0], 1 + o[0] + nx))

    def _assemble_dia(self, coeff):
        """Element-by-element assembly of A_l (§2.1 Eq. (2)) into DIA form."""
        A = {}
        for s, sigma in enumerate(PERMS):
            offs = _kuhn_offsets(sigma)
            K = self.Kel[s]
            kmap = coeff[self.emacro[s]]
            for a in range(4):
                sl = self._cell_slice(offs[a])
                for b in range(4):
                    d = tuple(ob - oa for ob, oa in zip(offs[b], offs[a]))
                    arr = A.get(d)
                    if arr is None:
                        arr = A[d] = np.zeros(self.pshape)
                    kab = K[a, b] if K.ndim == 2 else K[:, a, b][self.emacro[s]]
                    arr[sl] += kmap * kab
        # drop offsets whose coefficients are all exactly zero
        return {d: a for d, a in A.items() if d == (0, 0, 0) or np.any(a != 0.0)}

    def incident_counts(self, faulty_macros=None):
        """Per node: number of incident fine tetrahedra, and how many of them
        belong to the given macro set."""
        cnt = np.zeros(self.pshape)
        cntf = np.zeros(self.pshape)
        fm = None
        if faulty_macros is not None:
            fm = np.zeros(self.n_macro, dtype=bool)
            fm[np.asarray(list(faulty_macros), dtype=np.int64)] = True
        for s, sigma in enumerate(PERMS):
            flag = fm[self.emacro[s]] if fm is not None else None
            for o in _kuhn_offsets(sigma):
                sl = self._cell_slice(o)
                cnt[sl] += 1.0
                if flag is not None:
                    cntf[sl] += flag
        return interior(cnt), interior(cntf)


def _node_macro(lv, x, y, z):
    """A macro containing each grid node (x, y, z): the Kuhn simplex of its
    sub-cube whose axis order sorts the node's sub-cube-local coordinates in
    decreasing order (on shared faces any containing macro gives the same
    position, as neighbouring macro maps agree there)."""
    N = lv.N
    sx, sy, sz = lv.sub
    sc = [np.minimum(q // N, s - 1) for q, s in ((x, sx), (y, sy), (z, sz))]
    loc = np.stack([x - sc[0] * N, y - sc[1] * N, z - sc[2] * N], axis=-1)
    order = np.argsort(-loc, axis=-1, kind="stable")
    lut = np.zeros(27, dtype=np.int64)
    for i, p in enumerate(PERMS):
        lut[p[0] * 9 + p[1] * 3 + p[2]] = i
    pidx = lut[order[..., 0] * 9 + order[..., 1] * 3 + order[..., 2]]
    return ((sc[2] * sy + sc[1]) * sx + sc[0]) * 6 + pidx


def node_coords(lv):
    """Physical coordinates (x, y, z) of every node of a level."""
    x, y, z = lv.xyz
    nx, ny, nz = lv.n
    if lv.vertex_pos is None:
        p = np.stack([x / nx, y / ny, z / nz], axis=0)
        X = np.tensordot(lv.G, p, axes=(1, 0))
        return X[0], X[1], X[2]
    V0, P0, M = lv.maps
    t = _node_macro(lv, x, y, z)
    s = np.stack([x, y, z], axis=-1) / lv.N - V0[t]
    X = P0[t] + np.einsum("...ab,...b->...a", M[t], s)
    return X[..., 0], X[..., 1], X[..., 2]


def assemble_coo(lv, coeff):
    """Literal per-element assembly of A_l into scipy CSR (tiny meshes only).

    Rows / columns are grid nodes in x-fastest order.  One Python iteration per
    fine tetrahedron: the plain definition of the FE stiffness matrix (§2.1).
    """
    import scipy.sparse as sp
    nx, ny, nz = lv.n
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    rows, cols, vals = [], [], []
    coeff = np.asarray(coeff, dtype=np.float64)

    def gid(p):
        return (p[2] * (ny + 1) + p[1]) * (nx + 1) + p[0]

    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                for s, sigma in enumerate(PERMS):
                    verts = [(cx + o[0], cy + o[1], cz + o[2]) for o in _kuhn_offsets(sigma)]
                    t = lv.emacro[s][cz, cy, cx]
                    if lv.vertex_pos is None:
                        X = np.array([lv.G @ (np.array(v) * h) for v in verts])
                    else:
                        V0, P0, M = lv.maps
                        X = np.array([P0[t] + M[t] @ (np.array(v) / lv.N - V0[t]) for v in verts])
                    K = element_stiffness(X) * coeff[t]
                    ids = [gid(v) for v in verts]
                    for a in range(4):
                        for b in range(4):
                            rows.append(ids[a]); cols.append(ids[b]); vals.append(K[a, b])
    n = (nx + 1) * (ny + 1) * (nz + 1)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def dia_to_csr(lv):
    """The DIA operator of a level as a scipy CSR matrix (x-fastest node ids)."""
    import scipy.sparse as sp
    nz1, ny1, nx1 = lv.shape
    idx = np.arange(nz1 * ny1 * nx1).reshape(lv.shape)
    rows, cols, vals = [], [], []
    for d, a in lv.A.items():
        coef = interior(a)
        z0, z1 = max(0, -d[2]), nz1 - max(0, d[2])
        y0, y1 = max(0, -d[1]), ny1 - max(0, d[1])
        x0, x1 = max(0, -d[0]), nx1 - max(0, d[0])
        r = idx[z0:z1, y0:y1, x0:x1]
        c = idx[z0 + d[2]:z1 + d[2], y0 + d[1]:y1 + d[1], x0 + d[0]:x1 + d[0]]
        v = coef[z0:z1, y0:y1, x0:x1]
        rows.append(r.ravel()); cols.append(c.ravel()); vals.append(v.ravel())
    n = idx.size
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    M.eliminate_zeros()
    return M


def _shift(u, d, lv):
    nx, ny, nz = lv.n
    return u[1 + d[2]:2 + d[2] + nz, 1 + d[1]:2 + d[1] + ny, 1 + d[0]:2 + d[0] + nx]


def apply_A(lv, u):
    """Matrix-free product (A_l u) at every grid node (u padded, zero pad)."""
    y = np.zeros(lv.shape)
    for d, a in lv.A.items():
        y += interior(a) * _shift(u, d, lv)
    return y


class Problem:
    """Which nodes of each level are unknowns (free).

    The global problem frees every interior node; recovery problems free the
    nodes of an open sub-domain (the faulty part for LR/DD step a, the healthy
    part for DD step b, §4.2 Algorithm 1).  Everything else is frozen and acts
    as Dirichlet data on the finest level and as homogeneous Dirichlet data for
    the coarse-level corrections.
    """

    def __init__(self, mesh, free_masks):
        self.free = list(free_masks)
        self.lists = []
        for lv, m in zip(mesh.levels, self.free):
            per = []
            for c in range(4):
                zz, yy, xx = np.nonzero(m & (lv.colour == c))
                per.append(((zz + 1) * lv.Py + (yy + 1)) * lv.Px + (xx + 1))
            self.lists.append(per)


class Mesh:
    """The level hierarchy r0..R of the cube macro mesh (§2.1); with
    ``vertex_pos`` the sub-cube corners sit at the given physical positions
    (general macro shapes, a polyhedral domain of the same connectivity)."""

    def __init__(self, sub, R, r0=2, coeff=None, affine=None, vertex_pos=None):
        self.sub = tuple(int(s) for s in sub)
        self.n_macro = 6 * self.sub[0] * self.sub[1] * self.sub[2]
        if R <= r0:
            raise ValueError("need at least two levels (R > r0)")
        if coeff is None:
            coeff = np.ones(self.n_macro)
        self.coeff = np.asarray(coeff, dtype=np.float64)
        self.affine = affine
        self.vertex_pos = None if vertex_pos is None else np.asarray(vertex_pos, dtype=np.float64)
        if self.vertex_pos is not None and self.vertex_pos.shape != (self.sub[2] + 1, self.sub[1] + 1,
                                                                     self.sub[0] + 1, 3):
            raise ValueError("vertex_pos must have shape (sz+1, sy+1, sx+1, 3)")
        self.R, self.r0 = int(R), int(r0)
        self.levels = [Level(self.sub, r, self.coeff, affine, self.vertex_pos) for r in range(self.r0, self.R + 1)]
        self.global_problem = Problem(self, [~lv.boundary for lv in self.levels])

    @property
    def fine(self):
        return self.levels[-1]

    def fault_masks(self, ids):
        """Per level: (open faulty sub-domain, closed faulty sub-domain).

        A node is inside the open union of the faulty macro-tetrahedra when
        every fine tetrahedron touching it is faulty, and in its closure when
        at least one is (§2.2: Omega_F open, Gamma = its boundary with
        Omega_I).  Nodes on the domain boundary are never inside Omega_F.
        """
        out = []
        for lv in self.levels:
            cnt, cntf = lv.incident_counts(ids)
            open_f = (cntf == cnt) & (cnt > 0) & ~lv.boundary
            closed_f = cntf > 0
            out.append((open_f, closed_f))
        return out

    def local_problem(self, ids):
        """Dirichlet problem on the faulty sub-domain (Algorithm 1, step a)."""
        return Problem(self, [o for o, _ in self.fault_masks(ids)])

    def healthy_problem(self, ids):
        """Dirichlet problem on the healthy sub-domain with the interface frozen
        (Algorithm 1, step b)."""
        return Problem(self, [(~lv.boundary) & ~c for lv, (_, c) in zip(self.levels, self.fault_masks(ids))])


def healthy_mesh(mesh, ids):
    """The level hierarchy of A_I: the operator assembled from the healthy
    macros' elements only (coefficients of the faulty macros set to zero),
    which is the sum of the healthy sub-stencils at interface nodes (§3.2)."""
    coeff = mesh.coeff.copy()
    coeff[np.asarray(list(ids), dtype=np.int64)] = 0.0
    return Mesh(mesh.sub, mesh.R, mesh.r0, coeff=coeff, affine=mesh.affine, vertex_pos=mesh.vertex_pos)


def dn_recover(mesh, u, f, ids, n_global, eta, pre=3, post=3, cg_rtol=1e-12, cg_maxit=1000, hmesh=None):
    """Dirichlet-Neumann recovery, Algorithm 2 (§4.3), after the fault.

    Reading used for the sign of the flux: the healthy sub-domain keeps, on
    the interface nodes G, the flux its own elements produce at the time of
    the fault, b_G = (A_I u)_G (A_I: operator of the healthy macros' elements),
    i.e. the Neumann data -lambda of Eq. (5) with lambda = -(A_I u)_G of
    Algorithm 2 step 4.  Omega_I then iterates on A_I restricted to
    Omega_I and G with right-hand side f on Omega_I and b_G on G; Omega_F
    iterates on its Dirichlet problem with the interface values of the last
    finished Omega_I cycle (one-way I -> F update): block j of Omega_F cycles
    (ceil(j eta) - ceil((j - 1) eta) of them) uses the values after Omega_I
    cycle j - 1.  Returns the number of Omega_F cycles run.
    """
    hm = hmesh or healthy_mesh(mesh, ids)
    fine = mesh.fine
    masks = mesh.fault_masks(ids)
    open_f, closed_f = masks[-1]
    gamma = closed_f & ~open_f & ~fine.boundary
    # Omega_I Neumann problem: free = interior nodes outside the open faulty set
    hp = Problem(hm, [(~lv.boundary) & ~o for lv, (o, _) in zip(mesh.levels, masks)])
    lp = mesh.local_problem(ids)
    top = len(mesh.levels) - 1
    fI = f.copy()
    interior(fI)[gamma] = apply_A(hm.fine, u)[gamma]
    snap = interior(u)[gamma].copy()
    n_F = 0
    for j in range(1, n_global + 1):
        cyc = int(math.ceil(j * eta)) - int(math.ceil((j - 1) * eta))
        uf = u.copy()
        interior(uf)[gamma] = snap
        for _ in range(cyc):
            vcycle(mesh, lp, top, uf, f, pre, post, cg_rtol, cg_maxit)
        n_F += cyc
        interior(u)[open_f] = interior(uf)[open_f]
        vcycle(hm, hp, top, u, fI, pre, post, cg_rtol, cg_maxit)
        snap = interior(u)[gamma].copy()
    return n_F


def gs_step(lv, u, f, lists):
    """One multicolour Gauss-Seidel step (§2.1 smoother): colours 0,1,2,3 in turn,
    u_i <- (f_i - sum_{j != i} a_ij u_j) / a_ii on the free nodes of each colour.
    Nodes of one colour are never coupled, so each colour is one vector update."""
    uf = u.reshape(-1)
    ff = f.reshape(-1)
    diag = lv.A[(0, 0, 0)].reshape(-1)
    for c in range(4):
        idx = lists[c]
        if idx.size == 0:
            continue
        s = np.zeros(idx.size)
        for d, a in lv.A.items():
            if d == (0, 0, 0):
                continue
            s += a.reshape(-1)[idx] * uf[idx + lv.off[d]]
        uf[idx] = (ff[idx] - s) / diag[idx]


def residual(lv, u, f, free):
    """r = f - A u on the free nodes, 0 elsewhere (grid-shaped)."""
    r = interior(f) - apply_A(lv, u)
    r[~free] = 0.0
    return r


def _fine_slices(d, nc):
    """Fine-grid slices of the nodes 2q + d, q in [0, nc - d] (per axis z,y,x)."""
    return tuple(slice(dd, 2 * (n - dd) + dd + 1, 2) for dd, n in zip(d, nc))


def prolong(ec):
    """Linear interpolation P (§2.1): coarse nodes are injected, the midpoint of
    each coarse edge 2q + d gets the mean of its two end points q and q + d."""
    nc = tuple(s - 1 for s in ec.shape)                  # (nz, ny, nx) coarse intervals
    ef = np.zeros(tuple(2 * n + 1 for n in nc))
    ef[::2, ::2, ::2] = ec
    for dx, dy, dz in FREUDENTHAL:
        d = (dz, dy, dx)
        lo = ec[:nc[0] + 1 - dz, :nc[1] + 1 - dy, :nc[2] + 1 - dx]
        hi = ec[dz:, dy:, dx:]
        ef[_fine_slices(d, nc)] = 0.5 * (lo + hi)
    return ef


def restrict(rf):
    """The adjoint of linear interpolation, R = P^T (§2.1)."""
    nc = tuple((s - 1) // 2 for s in rf.shape)
    rc = rf[::2, ::2, ::2].copy()
    for dx, dy, dz in FREUDENTHAL:
        d = (dz, dy, dx)
        t = 0.5 * rf[_fine_slices(d, nc)]
        rc[:nc[0] + 1 - dz, :nc[1] + 1 - dy, :nc[2] + 1 - dx] += t
        rc[dz:, dy:, dx:] += t
    return rc


def cg(lv, b, free, rtol=1e-12, maxit=1000):
    """Conjugate gradients for A_FF x = b_F from x = 0 (§2.1 coarse solver).

    Stops when ||r|| <= rtol ||b_F|| or after maxit iterations.  Returns the
    padded solution (zero off the free set) and the iteration count.
    """
    x = np.zeros(lv.pshape)
    r = np.zeros(lv.pshape)
    interior(r)[free] = interior(b)[free]
    p = r.copy()
    rr = float(np.sum(r * r))
    bnorm = math.sqrt(rr)
    it = 0
    if bnorm == 0.0:
        return x, 0
    while math.sqrt(rr) > rtol * bnorm and it < maxit:
        Ap = np.zeros(lv.pshape)
        interior(Ap)[free] = apply_A(lv, p)[free]
        alpha = rr / float(np.sum(p * Ap))
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(np.sum(r * r))
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        it += 1
    return x, it


def vcycle(mesh, prob, lvl, u, f, pre=3, post=3, cg_rtol=1e-12, cg_maxit=1000):
    """One multigrid V(pre, post) cycle, correction scheme (§2.1), on level
    index ``lvl`` (0 = coarsest).  ``u`` and ``f`` are padded arrays; ``u`` is
    updated in place on the problem's free nodes."""
    lv = mesh.levels[lvl]
    free = prob.free[lvl]
    if lvl == 0:
        x, _ = cg(lv, f, free, cg_rtol, cg_maxit)
        interior(u)[free] = interior(x)[free]
        return
    for _ in range(pre):
        gs_step(lv, u, f, prob.lists[lvl])
    r = residual(lv, u, f, free)
    fc = pad(restrict(r))
    ec = np.zeros(mesh.levels[lvl - 1].pshape)
    vcycle(mesh, prob, lvl - 1, ec, fc, pre, post, cg_rtol, cg_maxit)
    corr = prolong(interior(ec))
    interior(u)[free] += corr[free]
    for _ in range(post):
        gs_step(lv, u, f, prob.lists[lvl])


def resnorm(mesh, u, f, prob=None):
    """Euclidean norm of the algebraic residual on the free fine nodes."""
    prob = prob or mesh.global_problem
    r = residual(mesh.fine, u, f, prob.free[-1])
    return float(np.sqrt(np.sum(r * r)))


def inject_fault(mesh, u, ids):
    """Fault model of §2.2: the unknowns inside the faulty macro-tetrahedra are
    lost and re-initialised with zero; interface values survive (their copies
    exist in neighbouring ghost layers, §3.1)."""
    open_f, _ = mesh.fault_masks(ids)[-1]
    interior(u)[open_f] = 0.0


def solve(mesh, u, f, rtol=1e-8, max_cycles=50, pre=3, post=3, fault_cycle=-1,
          fault_ids=(), recovery=NONE, n_local=0, n_global=0, eta=1.0,
          cg_rtol=1e-12, cg_maxit=1000, record=False, faults=()):
    """V-cycle iteration to a relative residual ``rtol`` with an optional fault.

    The fault strikes after global cycle ``fault_cycle`` (§2.2).  Recovery:
    NONE = do-nothing (zero re-initialisation only), LR = ``n_F`` local
    Dirichlet cycles on Omega_F while Omega_I idles (§4.4), DD = Algorithm 1:
    ``n_F`` local cycles on Omega_F and ``n_I`` cycles on Omega_I with the
    interface frozen, then the global iteration resumes.  ``n_F`` is
    ``n_local`` if positive, else ceil(eta * n_I) (§4.4).  DN = Algorithm 2
    (see ``dn_recover``).

    ``faults`` lists further faults as (cycle, macro ids) pairs, handled the
    same way in cycle order (§5: a second fault at another location after
    the first recovery has finished).

    History: ``hist[0] = 1``, one entry per global cycle, and for a faulty run
    one extra entry right after each fault (and recovery).  ``k_faulty``
    counts global cycles plus n_I for DD and DN per fault (§4.4).
    """
    events = ([(int(fault_cycle), list(fault_ids))] if fault_cycle > 0 else [])
    events += [(int(c), list(ids)) for c, ids in faults]
    prob = mesh.global_problem
    top = len(mesh.levels) - 1
    r0 = resnorm(mesh, u, f)
    hist = [1.0]
    iterates = [u.copy()] if record else None
    k = 0
    extra = 0
    n_F = 0
    while k < max_cycles:
        vcycle(mesh, prob, top, u, f, pre, post, cg_rtol, cg_maxit)
        k += 1
        rel = resnorm(mesh, u, f) / r0
        hist.append(rel)
        if record:
            iterates.append(u.copy())
        for fc, ids in events:
            if k != fc:
                continue
            inject_fault(mesh, u, ids)
            if recovery == DN:
                n_F = dn_recover(mesh, u, f, ids, n_global, eta, pre, post, cg_rtol, cg_maxit)
                extra += n_global
            elif recovery in (LR, DD):
                n_F = n_local if n_local > 0 else int(math.ceil(eta * n_global))
                lp = mesh.local_problem(ids)
                for _ in range(n_F):
                    vcycle(mesh, lp, top, u, f, pre, post, cg_rtol, cg_maxit)
                if recovery == DD:
                    hp = mesh.healthy_problem(ids)
                    for _ in range(n_global):
                        vcycle(mesh, hp, top, u, f, pre, post, cg_rtol, cg_maxit)
                    extra += n_global
            rel = resnorm(mesh, u, f) / r0
            hist.append(rel)
            if record:
                iterates.append(u.copy())
        if rel <= rtol:
            break
    return {"u": u, "hist": np.array(hist), "cycles": k, "k_faulty": k + extra,
            "n_F": n_F, "r0": r0, "iterates": iterates}


def kappa(k_faulty, k_free, k_fault):
    """Cycle advantage, Eq. (3)."""
    return (k_faulty - k_free) / k_fault


def grad_coeff(mesh, u, lam):
    """dL/dk_T = -sum over fine tetrahedra e of macro T of lam_e^T K_e u_e.

    With A = sum_T k_T A_T (§2.1 Eq. (2), coefficient constant per macro) and
    lam the adjoint solution (zero at frozen nodes), differentiating
    A_FF u_F = f_F - A_FD g gives dL/dk_T = -lam^T (A_T u).
    """
    lv = mesh.fine
    g = np.zeros(mesh.n_macro)
    for s, sigma in enumerate(PERMS):
        offs = _kuhn_offsets(sigma)
        K = lv.Kel[s]
        acc = np.zeros(lv.emacro[s].shape)
        for a in range(4):
            la = lam[lv._cell_slice(offs[a])]
            for b in range(4):
                kab = K[a, b] if K.ndim == 2 else K[:, a, b][lv.emacro[s]]
                acc += kab * la * u[lv._cell_slice(offs[b])]
        g += np.bincount(lv.emacro[s].ravel(), weights=acc.ravel(), minlength=mesh.n_macro)
    return -g


def local_residual(sub, R, coeff, affine, u, f, nodes):
    """f_p - (A u)_p at selected nodes p of the finest grid, each row assembled
    on the spot from the fine tetrahedra around p (§2.1 Eq. (2)); for checks on
    meshes too large for a full assembly.  ``u`` and ``f`` are grid arrays
    (unpadded), ``nodes`` an (n, 3) array of (x, y, z) interior node indices."""
    sx, sy, sz = sub
    N = 1 << R
    nx, ny, nz = sx * N, sy * N, sz * N
    # (affine images of the uniform grid only)
    G = np.eye(3) if affine is None else np.asarray(affine, dtype=np.float64)[:, :3]
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    Kel = [element_stiffness(np.array([G @ (np.array(o) * h) for o in _kuhn_offsets(s)])) for s in PERMS]
    coeff = np.asarray(coeff, dtype=np.float64)
    out = np.zeros(len(nodes))
    for q, (x, y, z) in enumerate(np.asarray(nodes, dtype=np.int64)):
        acc = 0.0
        for s, sigma in enumerate(PERMS):
            offs = _kuhn_offsets(sigma)
            for a, oa in enumerate(offs):
                c = (x - oa[0], y - oa[1], z - oa[2])
                if not (0 <= c[0] < nx and 0 <= c[1] < ny and 0 <= c[2] < nz):
                    continue
                # macro of this fine tetrahedron: sort the centroid's sub-cube-local coordinates
                cen = [c[i] + (3 - sigma.index(i)) / 4.0 for i in range(3)]
                sc = [int(cen[i] // N) for i in range(3)]
                loc = [cen[i] - sc[i] * N for i in range(3)]
                pi = tuple(sorted(range(3), key=lambda i: -loc[i]))
                mid = ((sc[2] * sy + sc[1]) * sx + sc[0]) * 6 + PERMS.index(pi)
                for b, ob in enumerate(offs):
                    acc += coeff[mid] * Kel[s][a, b] * u[c[2] + ob[2], c[1] + ob[1], c[0] + ob[0]]
        out[q] = f[z, y, x] - acc
    return out
