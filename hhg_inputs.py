"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and bench.py.

This module holds no arithmetic of the multigrid method: it only draws the
problem data (right-hand sides, boundary values, coefficients, target fields,
fault sets) that both the CUDA path and the CPU oracle receive as inputs.
Vectors are laid out over the global node grid of the cube family, x fastest:
node (x, y, z) of a grid with nx, ny, nz intervals has flat index
(z * (ny + 1) + y) * (nx + 1) + x.
"""

from __future__ import annotations

import numpy as np


def grid_dims(sub, r):
    """Intervals per axis (nx, ny, nz) of refinement r of ``sub`` sub-cubes."""
    N = 1 << int(r)
    return (int(sub[0]) * N, int(sub[1]) * N, int(sub[2]) * N)


def n_nodes(sub, r):
    nx, ny, nz = grid_dims(sub, r)
    return (nx + 1) * (ny + 1) * (nz + 1)


def grid_coords(sub, r):
    """Physical coordinates of every node of the unit cube, each of shape
    (nz+1, ny+1, nx+1)."""
    nx, ny, nz = grid_dims(sub, r)
    z, y, x = np.meshgrid(np.arange(nz + 1) / nz, np.arange(ny + 1) / ny,
                          np.arange(nx + 1) / nx, indexing="ij")
    return x, y, z


def boundary_mask(sub, r):
    nx, ny, nz = grid_dims(sub, r)
    z, y, x = np.indices((nz + 1, ny + 1, nx + 1))
    return (x == 0) | (x == nx) | (y == 0) | (y == ny) | (z == 0) | (z == nz)


def random_load(sub, r, seed=0):
    """Load vector with i.i.d. uniform[-1, 1] entries per fine node (Philox
    stream keyed by ``seed``), zero on the Dirichlet boundary."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    f = rng.uniform(-1.0, 1.0, size=n_nodes(sub, r))
    nx, ny, nz = grid_dims(sub, r)
    f = f.reshape(nz + 1, ny + 1, nx + 1)
    f[boundary_mask(sub, r)] = 0.0
    return f


def harmonic_boundary(sub, r):
    """u*(x, y, z) = exp(pi x) sin(pi y) on every node (harmonic in 3-D); the
    solver uses its boundary values as Dirichlet data."""
    x, y, _ = grid_coords(sub, r)
    return np.exp(np.pi * x) * np.sin(np.pi * y)


def initial_guess(sub, r, g=None):
    """Zero in the interior, Dirichlet values g (or zero) on the boundary."""
    nx, ny, nz = grid_dims(sub, r)
    u = np.zeros((nz + 1, ny + 1, nx + 1))
    if g is not None:
        b = boundary_mask(sub, r)
        u[b] = g[b]
    return u


def lognormal_coeff(n_macro, seed=1):
    """Per-macro diffusion coefficient k_T = exp(N(0, 1))."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    return np.exp(rng.standard_normal(int(n_macro)))


def smooth_target(sub, r):
    """u_target = sin(pi x) sin(pi y) sin(pi z) at the nodes."""
    x, y, z = grid_coords(sub, r)
    return np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)


def subcube_macros(sub, a=0, b=0, c=0):
    """Ids of the six macro-tetrahedra of sub-cube (a, b, c) (x fastest, six
    Kuhn tetrahedra per sub-cube in lexicographic axis order)."""
    s = (int(c) * int(sub[1]) + int(b)) * int(sub[0]) + int(a)
    return list(range(6 * s, 6 * s + 6))


def random_directions(n_macro, count, seed=2):
    """``count`` random unit directions in coefficient space."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    d = rng.standard_normal((int(count), int(n_macro)))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def macro_vertices(sub):
    """Integer sub-cube coordinates of the 4 vertices of every macro (Kuhn
    tetrahedron p of sub-cube (a, b, c): 0, e_pi0, e_pi0 + e_pi1, (1,1,1))."""
    import itertools
    perms = list(itertools.permutations((0, 1, 2)))
    out = []
    for c in range(sub[2]):
        for b in range(sub[1]):
            for a in range(sub[0]):
                for p in perms:
                    v0 = (a, b, c)
                    v1 = list(v0)
                    v1[p[0]] += 1
                    v2 = list(v1)
                    v2[p[1]] += 1
                    out.append([v0, tuple(v1), tuple(v2), (a + 1, b + 1, c + 1)])
    return out


def jittered_vertices(sub, seed=4, amp=0.12, move_boundary=True):
    """Physical positions of the sub-cube corners, shape (sz+1, sy+1, sx+1, 3):
    the unit cube's corner grid with every corner moved by a seeded uniform
    offset of up to ``amp`` sub-cube edges per axis (Philox).  With
    ``move_boundary`` false the corners on the cube's boundary stay put, so the
    domain remains the unit cube; otherwise it becomes a general polyhedron.
    The macro-tetrahedra then have general shapes (not congruent Kuhn
    simplices)."""
    sx, sy, sz = (int(s) for s in sub)
    rng = np.random.Generator(np.random.Philox(int(seed)))
    k, j, i = np.meshgrid(np.arange(sz + 1), np.arange(sy + 1), np.arange(sx + 1), indexing="ij")
    base = np.stack([i / sx, j / sy, k / sz], axis=-1)
    step = np.array([1.0 / sx, 1.0 / sy, 1.0 / sz])
    off = rng.uniform(-amp, amp, size=base.shape) * step
    if not move_boundary:
        bnd = (i == 0) | (i == sx) | (j == 0) | (j == sy) | (k == 0) | (k == sz)
        off[bnd] = 0.0
    return base + off


def corner_grid(sub):
    """Unit-cube positions of the sub-cube corners, (n_corner, 3), corner
    (a, b, c) at index (c (sy+1) + b)(sx+1) + a."""
    sx, sy, sz = (int(s) for s in sub)
    k, j, i = np.meshgrid(np.arange(sz + 1), np.arange(sy + 1), np.arange(sx + 1), indexing="ij")
    return np.stack([i / sx, j / sy, k / sz], axis=-1).reshape(-1, 3)


def _corner_id(sub, v):
    return (int(v[2]) * (int(sub[1]) + 1) + int(v[1])) * (int(sub[0]) + 1) + int(v[0])


def kuhn_macro_mesh(sub):
    """The cube family's macro mesh as a general one: (verts, tets), the six
    Kuhn tetrahedra of every sub-cube with their vertices in the order 0,
    e_pi0, e_pi0 + e_pi1, (1,1,1) (macro ids as in ``macro_vertices``)."""
    tets = [[_corner_id(sub, v) for v in m] for m in macro_vertices(sub)]
    return corner_grid(sub), np.array(tets, dtype=np.int64)


def five_tet_macro_mesh(sub, seed=None, amp=0.0):
    """A macro mesh of another connectivity: every sub-cube split into five
    tetrahedra (a central one and four corner ones), the split mirrored on
    alternate sub-cubes so that neighbouring splits share their face
    diagonals.  Vertices ordered for a positive orientation.  With ``seed``
    the interior corners move by seeded uniform offsets of up to ``amp``
    sub-cube edges per axis."""
    sx, sy, sz = (int(s) for s in sub)
    verts = corner_grid(sub)
    if seed is not None:
        rng = np.random.Generator(np.random.Philox(int(seed)))
        off = rng.uniform(-amp, amp, size=verts.shape) * np.array([1.0 / sx, 1.0 / sy, 1.0 / sz])
        b = (np.isclose(verts, 0.0) | np.isclose(verts, 1.0)).any(axis=1)
        off[b] = 0.0
        verts = verts + off
    tets = []
    for c in range(sz):
        for b in range(sy):
            for a in range(sx):
                cid = lambda d: _corner_id(sub, (a + d[0], b + d[1], c + d[2]))
                even = [(0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
                odd = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]
                inner, apex = (even, odd) if (a + b + c) % 2 == 0 else (odd, even)
                parts = [[cid(d) for d in inner]]
                # each remaining corner with its three axis neighbours (the
                # central tetrahedron's vertices)
                for d in apex:
                    nb = [tuple(d[q] ^ (q == ax) for q in range(3)) for ax in range(3)]
                    parts.append([cid(d)] + [cid(n) for n in nb])
                for tet in parts:
                    X = verts[tet]
                    if np.linalg.det((X[1:] - X[0]).T) < 0:
                        tet = [tet[0], tet[2], tet[1], tet[3]]
                    tets.append(tet)
    return verts, np.array(tets, dtype=np.int64)


def grow_fault_set(sub, size, seed):
    """A connected set of ``size`` macros grown breadth-first (through shared
    faces) from a random seed macro, with a random visiting order."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    verts = [frozenset(v) for v in macro_vertices(sub)]
    n = len(verts)
    size = int(min(size, n))
    start = int(rng.integers(n))
    chosen, frontier = [start], [start]
    seen = {start}
    while frontier and len(chosen) < size:
        cur = frontier.pop(0)
        nbrs = [t for t in range(n) if t not in seen and len(verts[cur] & verts[t]) == 3]
        rng.shuffle(nbrs)
        for t in nbrs:
            if len(chosen) >= size:
                break
            seen.add(t)
            chosen.append(t)
            frontier.append(t)
    return sorted(chosen)


def batch_problems(count, seed=3, max_size=27, levels=(5, 6, 7)):
    """Recovery problems of uneven size: (sub-cubes, refinement, fault macros)
    with sizes ~ U{1..max_size} and refinements drawn from ``levels``; each
    problem lives on the smallest cube of sub-cubes that holds its macros."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    out = []
    for q in range(int(count)):
        size = int(rng.integers(1, max_size + 1))
        r = int(levels[int(rng.integers(len(levels)))])
        for sub in [(1, 1, 1), (2, 1, 1), (2, 2, 1), (2, 2, 2), (3, 2, 2), (3, 3, 2), (3, 3, 3)]:
            if 6 * sub[0] * sub[1] * sub[2] >= size:
                break
        out.append((sub, r, grow_fault_set(sub, size, seed * 1000 + q)))
    return out


def boundary_contact(sub, macro):
    """(faces, edges) of a macro-tetrahedron that lie on the boundary of the
    unit cube (pure geometry of the macro mesh)."""
    import itertools
    V = macro_vertices(sub)[int(macro)]
    ext = [int(s) for s in sub]

    def on_bnd(pts):
        for a in range(3):
            if all(p[a] == 0 for p in pts) or all(p[a] == ext[a] for p in pts):
                return True
        return False
    faces = sum(on_bnd(c) for c in itertools.combinations(V, 3))
    edges = sum(on_bnd(c) for c in itertools.combinations(V, 2))
    return faces, edges


def kappa_scenarios():
    """The three fault scenarios of the cycle-advantage study (§4.4): (name,
    sub-cubes, faulty macro ids).  I: 1x1x1 cube, a tetrahedron with two faces
    on the boundary; II: 2x2x2, the first tetrahedron touching the boundary
    along an edge only; III: 3x3x3, a tetrahedron of the centre sub-cube (no
    boundary contact)."""
    out = [("I", (1, 1, 1), [0])]
    sub = (2, 2, 2)
    for t in range(6 * 8):
        f, e = boundary_contact(sub, t)
        if f == 0 and e > 0:
            out.append(("II", sub, [t]))
            break
    out.append(("III", (3, 3, 3), subcube_macros((3, 3, 3), 1, 1, 1)[:1]))
    return out
