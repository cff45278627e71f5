"""Plain FP64 CPU multigrid on a general tetrahedral macro mesh (test
infrastructure only; the same import rule as the rest of ``oracle/``).

Reference: Huber, Gmeiner, Ruede, Wohlmuth, "Resilience for Multigrid Software
at the Extreme Scale", §2.1: a polyhedral domain triangulated by an
unstructured base mesh of tetrahedra, refined uniformly (Bey) into the level
hierarchy, P1 finite elements, V-cycles with linear interpolation and its
adjoint, Gauss-Seidel smoothing and a CG coarse solver.

Representation
--------------
``verts`` (nv, 3) physical vertex positions and ``tets`` (nt, 4) vertex ids
of the macro-tetrahedra.  Inside macro t with vertices g0..g3 the level with
N intervals per macro edge has the lattice nodes (i, j, k), i, j, k >= 0,
i + j + k <= N, at barycentric weights (N - i - j - k, i, j, k) / N.  A node
is identified across macros by the pairs (vertex id, weight) of its positive
weights, so the nodes of shared vertices, edges and faces exist once.  Node
ids are sorted by primitive dimension (vertex, edge, face, volume nodes) and
then by that key.  The fine tetrahedra of a macro are the Kuhn simplices of
its lattice in chain coordinates (a, b, c) = (i + j + k, j + k, k), which is
Bey's uniform refinement; on a shared face every macro induces the same
uniform triangle refinement, so the fine mesh is conforming.

Smoother (the reading for meshes of general connectivity, where the local
colourings of neighbouring macros need not agree on their shared nodes): one
Gauss-Seidel step visits
  * the volume nodes of every macro by their macro's local colour
    (i + 2j + 3k) mod 4, colours 0..3 in turn (a proper colouring of a macro's
    lattice; volume nodes of different macros are never coupled), then
  * the free interface nodes (vertex, edge and face nodes) in the classes of a
    greedy colouring of their coupling graph, taken in node-id order (each
    node gets the smallest class not used by an already coloured coupled
    interface node), classes in increasing order.
Within a class no two nodes are coupled, so each class is one vector update.

Faults (§2.2) and their recovery (LR / DD of Algorithm 1, DN of Algorithm 2)
follow the structured oracle's readings on these meshes.

Parity status: every function is pinned by ``tests/test_oracle_unstructured.py``
(the cube family given as a general mesh reproduces the structured oracle's
operator, transfers, boundary and fault sets; node counts of the macro mesh's
primitives; linear-function kernel and energy = volume; Galerkin identity;
proper smoother classes; V-cycles and recovery sub-problems = direct solves;
second-order error; recovery beats do-nothing).
"""

from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

__all__ = ["UMesh", "ULevel", "gs_step", "vcycle", "solve", "resnorm", "cg", "element_stiffness",
           "inject_fault", "dn_recover", "NONE", "LR", "DD", "DN"]

NONE, LR, DD, DN = 0, 1, 2, 3

PERMS = list(itertools.permutations((0, 1, 2)))


def element_stiffness(X):
    """P1 stiffness of tetrahedra with unit coefficient (§2.1 Eq. (2)):
    K_ab = |T| grad(lambda_a) . grad(lambda_b), the barycentric gradients being
    the rows of E^-1 (E = edge vectors as columns) and minus their sum.
    ``X``: (4, 3) vertex positions, or (m, 4, 3) for m tetrahedra."""
    X = np.asarray(X, dtype=np.float64)
    E = np.swapaxes(X[..., 1:, :] - X[..., :1, :], -1, -2)
    Einv = np.linalg.inv(E)
    D = np.concatenate([-Einv.sum(axis=-2, keepdims=True), Einv], axis=-2)
    vol = np.abs(np.linalg.det(E)) / 6.0
    return vol[..., None, None] * (D @ np.swapaxes(D, -1, -2))


def lattice(N):
    """All lattice points (i, j, k) of a macro at refinement N, as an (n, 3) array."""
    pts = [(i, j, k) for k in range(N + 1) for j in range(N + 1 - k) for i in range(N + 1 - j - k)]
    return np.array(pts, dtype=np.int64)


def _fine_tets(N):
    """The fine tetrahedra of one macro as (m, 4, 3) arrays of lattice points:
    the Kuhn simplices of the chain lattice that lie in N >= a >= b >= c >= 0."""
    out = []
    for a in range(N):
        for b in range(a + 1):
            for c in range(b + 1):
                for p in PERMS:
                    v = [np.array((a, b, c))]
                    cur = np.array((a, b, c))
                    for ax in p:
                        cur = cur.copy()
                        cur[ax] += 1
                        v.append(cur)
                    ok = all(N >= q[0] >= q[1] >= q[2] >= 0 for q in v)
                    if ok:
                        out.append([(q[0] - q[1], q[1] - q[2], q[2]) for q in v])
    return np.array(out, dtype=np.int64)


class ULevel:
    """One level: node keys, positions, the assembled operator ``A`` (CSR),
    the Dirichlet mask ``boundary``, each macro's lattice-to-node map
    ``l2g[t]`` and the smoother classes ``classes`` (lists of node ids)."""

    def __init__(self, mesh, r):
        self.r = int(r)
        N = 1 << self.r
        self.N = N
        verts, tets = mesh.verts, mesh.tets
        self.pts = lattice(N)
        w = np.stack([N - self.pts.sum(axis=1), self.pts[:, 0], self.pts[:, 1], self.pts[:, 2]], axis=1)
        # canonical key of every (macro, lattice point): the (vertex, weight)
        # pairs sorted by vertex id, weight 0 where the vertex is not involved
        keys = []
        for t in range(mesh.nt):
            g = np.broadcast_to(tets[t], w.shape)
            order = np.argsort(g, axis=1, kind="stable")
            gs = np.take_along_axis(g, order, axis=1)
            ws = np.take_along_axis(w, order, axis=1)
            gs = np.where(ws > 0, gs, -1)
            dim = (ws > 0).sum(axis=1)[:, None]
            keys.append(np.concatenate([dim, np.sort(np.where(ws > 0, gs * (N + 1) + ws, -1), axis=1)], axis=1))
        allk = np.concatenate(keys, axis=0)
        uniq, inv = np.unique(allk, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        self.keys = uniq
        self.n = len(uniq)
        self.l2g = [inv[t * len(self.pts):(t + 1) * len(self.pts)] for t in range(mesh.nt)]
        self.dim = uniq[:, 0]                             # 1 vertex, 2 edge, 3 face, 4 volume
        # positions
        X = np.zeros((self.n, 3))
        for t in range(mesh.nt):
            X[self.l2g[t]] = (w / N) @ verts[tets[t]]
        self.X = X
        # Dirichlet nodes: on a face of exactly one macro
        face_count = {}
        for t in range(mesh.nt):
            for f in itertools.combinations(sorted(tets[t]), 3):
                face_count[f] = face_count.get(f, 0) + 1
        bfaces = {f for f, c in face_count.items() if c == 1}
        bnd = np.zeros(self.n, dtype=bool)
        for t in range(mesh.nt):
            for loc in itertools.combinations(range(4), 3):
                if tuple(sorted(tets[t][list(loc)])) in bfaces:
                    on = np.all(w[:, [q for q in range(4) if q not in loc]] == 0, axis=1)
                    bnd[self.l2g[t][on]] = True
        self.boundary = bnd
        # operator, element by element
        ft = _fine_tets(N)
        idx = {tuple(p): q for q, p in enumerate(self.pts)}
        ft_local = np.array([[idx[tuple(p)] for p in e] for e in ft], dtype=np.int64)
        rows, cols, vals = [], [], []
        for t in range(mesh.nt):
            nodes = self.l2g[t][ft_local]                 # (m, 4) node ids
            K = element_stiffness(self.X[nodes]) * mesh.coeff[t]
            rows.append(np.repeat(nodes, 4, axis=1).ravel())
            cols.append(np.tile(nodes, (1, 4)).ravel())
            vals.append(K.reshape(len(nodes), 16).ravel())
        self.A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(self.n, self.n))
        self.A.sum_duplicates()
        self.diag = self.A.diagonal()
        # smoother classes on the free nodes
        free = ~self.boundary
        vol_col = np.full(self.n, -1)
        colour = (self.pts[:, 0] + 2 * self.pts[:, 1] + 3 * self.pts[:, 2]) % 4
        for t in range(mesh.nt):
            inner = self.dim[self.l2g[t]] == 4
            vol_col[self.l2g[t][inner]] = colour[inner]
        self.classes = [np.nonzero((vol_col == c) & free)[0] for c in range(4)]
        iface = np.nonzero((self.dim < 4) & free)[0]
        icls = np.full(self.n, -1)
        Acoo = self.A.tocsr()
        for v in iface:                                   # node-id order
            nb = Acoo.indices[Acoo.indptr[v]:Acoo.indptr[v + 1]]
            used = {icls[q] for q in nb if q != v and icls[q] >= 0}
            c = 0
            while c in used:
                c += 1
            icls[v] = c
        n_ic = int(icls.max()) + 1 if iface.size else 0
        self.classes += [np.nonzero(icls == c)[0] for c in range(n_ic)]
        self.n_interface_classes = n_ic


class UMesh:
    """Level hierarchy r0..R of a general tetrahedral macro mesh (§2.1)."""

    def __init__(self, verts, tets, R, r0=2, coeff=None):
        self.verts = np.asarray(verts, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        self.nt = len(self.tets)
        if R <= r0:
            raise ValueError("need at least two levels (R > r0)")
        for t in range(self.nt):
            E = self.verts[self.tets[t, 1:]] - self.verts[self.tets[t, 0]]
            if abs(np.linalg.det(E)) < 1e-12:
                raise ValueError(f"macro {t} is degenerate")
        self.coeff = np.ones(self.nt) if coeff is None else np.asarray(coeff, dtype=np.float64)
        self.R, self.r0 = int(R), int(r0)
        self.levels = [ULevel(self, r) for r in range(self.r0, self.R + 1)]
        self.P = [self._prolongation(l) for l in range(1, len(self.levels))]

    def fault_masks(self, ids):
        """Per level: (open faulty set, closed faulty set) of nodes (§2.2): a
        node is inside the open union of the faulty macros when every macro
        containing it is faulty (and it is not a Dirichlet node), in its
        closure when at least one is."""
        faulty = np.zeros(self.nt, dtype=bool)
        faulty[np.asarray(list(ids), dtype=np.int64)] = True
        out = []
        for lv in self.levels:
            cnt = np.zeros(lv.n, dtype=np.int64)
            cntf = np.zeros(lv.n, dtype=np.int64)
            for t in range(self.nt):
                cnt[lv.l2g[t]] += 1
                if faulty[t]:
                    cntf[lv.l2g[t]] += 1
            out.append(((cntf == cnt) & ~lv.boundary, cntf > 0))
        return out

    def global_masks(self):
        return [~lv.boundary for lv in self.levels]

    def local_masks(self, ids):
        """Free nodes of the Dirichlet problem on Omega_F (Algorithm 1, step a)."""
        return [o for o, _ in self.fault_masks(ids)]

    def healthy_masks(self, ids):
        """Free nodes of Omega_I with the interface frozen (Algorithm 1, step b)."""
        return [~lv.boundary & ~c for lv, (_, c) in zip(self.levels, self.fault_masks(ids))]

    def healthy(self, ids):
        """The hierarchy of A_I: only the healthy macros' elements (faulty
        coefficients zero), the sum of healthy sub-stencils at the interface."""
        coeff = self.coeff.copy()
        coeff[np.asarray(list(ids), dtype=np.int64)] = 0.0
        return UMesh(self.verts, self.tets, self.R, self.r0, coeff)

    def _prolongation(self, l):
        """Linear interpolation from level l - 1 to level l (§2.1): a fine
        lattice point p (chain coordinates) lies on the coarse edge from
        floor(p / 2) to ceil(p / 2) (a 0/1 chain step, i.e. a Freudenthal
        edge) and takes the mean of its end points; even points are coarse
        nodes."""
        fine, coarse = self.levels[l], self.levels[l - 1]
        cidx = {tuple(p): q for q, p in enumerate(coarse.pts)}
        rows, cols, vals = [], [], []
        seen = np.zeros(fine.n, dtype=bool)
        chain = np.stack([fine.pts.sum(axis=1), fine.pts[:, 1] + fine.pts[:, 2], fine.pts[:, 2]], axis=1)
        lo, hi = chain // 2, (chain + 1) // 2
        to_ijk = lambda c: (c[0] - c[1], c[1] - c[2], c[2])
        for t in range(self.nt):
            for q in range(len(fine.pts)):
                v = fine.l2g[t][q]
                if seen[v]:
                    continue
                seen[v] = True
                a = coarse.l2g[t][cidx[to_ijk(lo[q])]]
                b = coarse.l2g[t][cidx[to_ijk(hi[q])]]
                if a == b:
                    rows.append(v); cols.append(a); vals.append(1.0)
                else:
                    rows += [v, v]; cols += [a, b]; vals += [0.5, 0.5]
        return sp.csr_matrix((vals, (rows, cols)), shape=(fine.n, coarse.n))


def gs_step(lv, u, f, free):
    """One Gauss-Seidel step in the class order described in the module
    docstring; only free nodes change."""
    for cls in lv.classes:
        idx = cls[free[cls]]
        if idx.size == 0:
            continue
        r = f[idx] - lv.A[idx] @ u
        u[idx] += r / lv.diag[idx]


def residual(lv, u, f, free):
    r = f - lv.A @ u
    r[~free] = 0.0
    return r


def resnorm(mesh, u, f):
    lv = mesh.levels[-1]
    return float(np.linalg.norm(residual(lv, u, f, ~lv.boundary)))


def cg(lv, b, free, rtol=1e-12, maxit=1000):
    """CG for A_FF x = b_F from x = 0 (coarse solver)."""
    A = lv.A[free][:, free]
    bf = b[free]
    x = np.zeros(bf.size)
    r = bf.copy()
    p = r.copy()
    rr = r @ r
    stop = rtol * np.sqrt(rr)
    it = 0
    while it < maxit and np.sqrt(rr) > stop and rr > 0:
        Ap = A @ p
        alpha = rr / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    out = np.zeros(lv.n)
    out[free] = x
    return out, it


def vcycle(mesh, lvl, u, f, free_masks, pre=3, post=3, cg_rtol=1e-12, cg_maxit=1000):
    """V(pre, post) correction-scheme cycle on level ``lvl`` (§2.1)."""
    lv = mesh.levels[lvl]
    free = free_masks[lvl]
    if lvl == 0:
        x, _ = cg(lv, residual(lv, u, f, free), free, cg_rtol, cg_maxit)
        u += x
        return
    for _ in range(pre):
        gs_step(lv, u, f, free)
    rc = mesh.P[lvl - 1].T @ residual(lv, u, f, free)
    cfree = free_masks[lvl - 1]
    rc[~cfree] = 0.0
    ec = np.zeros(mesh.levels[lvl - 1].n)
    vcycle(mesh, lvl - 1, ec, rc, free_masks, pre, post, cg_rtol, cg_maxit)
    e = mesh.P[lvl - 1] @ ec
    u[free] += e[free]
    for _ in range(post):
        gs_step(lv, u, f, free)


def inject_fault(mesh, u, ids):
    """Fault model of §2.2: the unknowns strictly inside the faulty macros
    are lost and re-initialised with zero; the interface values survive."""
    u[mesh.local_masks(ids)[-1]] = 0.0


def dn_recover(mesh, u, f, ids, n_global, eta, pre=3, post=3):
    """Dirichlet-Neumann recovery, Algorithm 2 (§4.3), with the same reading
    as the structured oracle: Omega_I and the interface G iterate on A_I with
    right-hand side f on Omega_I and b_G = (A_I u)_G at the fault on G; block
    j of ceil(j eta) - ceil((j - 1) eta) Omega_F Dirichlet cycles uses the G
    values after Omega_I cycle j - 1.  Returns the Omega_F cycles run."""
    import math
    hm = mesh.healthy(ids)
    masks = mesh.fault_masks(ids)
    lv = mesh.levels[-1]
    open_f, closed_f = masks[-1]
    gamma = closed_f & ~open_f & ~lv.boundary
    i_masks = [~l.boundary & ~o for l, (o, _) in zip(mesh.levels, masks)]
    f_masks = [o for o, _ in masks]
    top = len(mesh.levels) - 1
    fI = f.copy()
    fI[gamma] = (hm.levels[-1].A @ u)[gamma]
    snap = u[gamma].copy()
    n_F = 0
    for j in range(1, n_global + 1):
        cyc = int(math.ceil(j * eta)) - int(math.ceil((j - 1) * eta))
        uf = u.copy()
        uf[gamma] = snap
        for _ in range(cyc):
            vcycle(mesh, top, uf, f, f_masks, pre, post)
        n_F += cyc
        u[open_f] = uf[open_f]
        vcycle(hm, top, u, fI, i_masks, pre, post)
        snap = u[gamma].copy()
    return n_F


def solve(mesh, u, f, rtol=1e-8, max_cycles=50, pre=3, post=3, fault_cycle=-1, fault_ids=(),
          recovery=NONE, n_local=0, n_global=0, eta=1.0):
    """V-cycles until ||f - A u|| <= rtol ||f - A u_0|| (free nodes), with an
    optional fault after global cycle ``fault_cycle`` and its recovery (NONE,
    LR, DD as Algorithm 1, DN as Algorithm 2; n_F = n_local if positive, else
    ceil(eta n_I)).  Returns the relative residual history: 1, one entry per
    global cycle, and one extra entry right after the fault and recovery."""
    import math
    top = len(mesh.levels) - 1
    masks = mesh.global_masks()
    r0 = resnorm(mesh, u, f)
    hist = [1.0]
    k = 0
    while k < max_cycles and hist[-1] > rtol:
        vcycle(mesh, top, u, f, masks, pre, post)
        k += 1
        hist.append(resnorm(mesh, u, f) / r0)
        if k == fault_cycle:
            inject_fault(mesh, u, fault_ids)
            if recovery == DN:
                dn_recover(mesh, u, f, fault_ids, n_global, eta, pre, post)
            elif recovery in (LR, DD):
                n_F = n_local if n_local > 0 else int(math.ceil(eta * n_global))
                lm = mesh.local_masks(fault_ids)
                for _ in range(n_F):
                    vcycle(mesh, top, u, f, lm, pre, post)
                if recovery == DD:
                    hm = mesh.healthy_masks(fault_ids)
                    for _ in range(n_global):
                        vcycle(mesh, top, u, f, hm, pre, post)
            hist.append(resnorm(mesh, u, f) / r0)
    return np.array(hist)
