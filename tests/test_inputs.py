"""The seeded input generators (hhg_inputs.py) draw what the workloads state:
the load vector's distribution and boundary zeros, a harmonic Dirichlet
field, Kuhn macro-tetrahedra that tile each sub-cube, connected fault sets of
the requested sizes, the batch mix, and the boundary contact of the three
fault scenarios of §4.4."""

import itertools

import numpy as np

import hhg_inputs as I


def test_random_load_is_seeded_uniform_and_zero_on_the_boundary():
    sub, r = (2, 2, 2), 4
    f = I.random_load(sub, r, seed=0)
    assert f.shape == (33, 33, 33)
    assert np.array_equal(f, I.random_load(sub, r, seed=0))
    assert not np.array_equal(f, I.random_load(sub, r, seed=1))
    b = I.boundary_mask(sub, r)
    assert np.all(f[b] == 0.0)
    inner = f[~b]
    assert inner.size == 31 ** 3
    assert inner.min() >= -1.0 and inner.max() <= 1.0
    # uniform[-1, 1]: mean 0, variance 1/3 (29,791 samples)
    assert abs(inner.mean()) < 0.02
    assert abs(inner.var() - 1.0 / 3.0) < 0.01


def test_harmonic_boundary_field_is_harmonic():
    # exp(pi x) sin(pi y): the 7-point difference Laplacian vanishes to O(h^2)
    errs = []
    for r in (4, 5):
        u = I.harmonic_boundary((1, 1, 1), r)
        h = 1.0 / (1 << r)
        lap = (u[1:-1, 1:-1, 2:] + u[1:-1, 1:-1, :-2] + u[1:-1, 2:, 1:-1] + u[1:-1, :-2, 1:-1]
               + u[2:, 1:-1, 1:-1] + u[:-2, 1:-1, 1:-1] - 6 * u[1:-1, 1:-1, 1:-1]) / h ** 2
        errs.append(np.abs(lap).max() / np.abs(u).max())
    assert errs[1] < errs[0] / 3.4       # second order (ratio -> 4)
    assert errs[1] < 0.02


def test_initial_guess_and_target():
    sub, r = (1, 1, 2), 3
    g = I.harmonic_boundary(sub, r)
    u = I.initial_guess(sub, r, g)
    b = I.boundary_mask(sub, r)
    assert np.array_equal(u[b], g[b]) and np.all(u[~b] == 0.0)
    t = I.smooth_target(sub, r)
    assert np.abs(t[b]).max() < 1e-12 and t[~b].min() > 0.0


def _volume(v):
    a, b, c, d = (np.array(p, dtype=float) for p in v)
    return np.linalg.det(np.stack([b - a, c - a, d - a])) / 6.0


def test_macro_tetrahedra_tile_every_sub_cube():
    sub = (2, 3, 1)
    V = I.macro_vertices(sub)
    assert len(V) == 6 * 2 * 3 * 1
    for s in range(len(V) // 6):
        tets = V[6 * s:6 * s + 6]
        vols = [abs(_volume(v)) for v in tets]
        assert np.allclose(vols, 1.0 / 6.0)           # six Kuhn tetrahedra, volume 1/6 each
        assert len({(v[0], v[3]) for v in tets}) == 1  # all share the main diagonal
        # their interiors are disjoint: the centroid of each tetrahedron lies
        # inside that tetrahedron only
        for p, v in enumerate(tets):
            x = np.mean(np.array(v, dtype=float), axis=0)
            inside = []
            for w in tets:
                T = np.stack([np.array(w[q], dtype=float) - np.array(w[0], dtype=float) for q in (1, 2, 3)], 1)
                lam = np.linalg.solve(T, x - np.array(w[0], dtype=float))
                inside.append(lam.min() > 1e-12 and lam.sum() < 1 - 1e-12)
            assert inside == [q == p for q in range(6)]
    assert I.subcube_macros(sub, 1, 2, 0) == list(range(6 * 5, 6 * 6))


def _connected(sub, ids):
    verts = [frozenset(v) for v in I.macro_vertices(sub)]
    ids = list(ids)
    seen, stack = {ids[0]}, [ids[0]]
    while stack:
        a = stack.pop()
        for b in ids:
            if b not in seen and len(verts[a] & verts[b]) == 3:
                seen.add(b)
                stack.append(b)
    return len(seen) == len(ids)


def test_fault_sets_are_connected_and_seeded():
    for sub, size, seed in [((1, 1, 1), 6, 0), ((2, 2, 2), 13, 5), ((3, 3, 3), 27, 9), ((2, 1, 1), 40, 1)]:
        ids = I.grow_fault_set(sub, size, seed)
        n = 6 * sub[0] * sub[1] * sub[2]
        assert len(ids) == min(size, n)
        assert ids == sorted(set(ids)) and 0 <= ids[0] and ids[-1] < n
        assert _connected(sub, ids)
        assert ids == I.grow_fault_set(sub, size, seed)


def test_batch_mix_of_sizes_and_levels():
    probs = I.batch_problems(64, seed=3)
    assert len(probs) == 64
    subs = [(1, 1, 1), (2, 1, 1), (2, 2, 1), (2, 2, 2), (3, 2, 2), (3, 3, 2), (3, 3, 3)]
    sizes = []
    for sub, r, ids in probs:
        assert r in (5, 6, 7)
        assert 1 <= len(ids) <= 27
        # the smallest cube of the list that holds the set
        k = subs.index(tuple(sub))
        assert 6 * np.prod(sub) >= len(ids) and (k == 0 or 6 * np.prod(subs[k - 1]) < len(ids))
        assert _connected(sub, ids)
        sizes.append(len(ids))
    assert len(set(sizes)) > 10 and len({r for _, r, _ in probs}) == 3


def test_fault_scenarios_touch_the_boundary_as_in_section_4_4():
    (n1, s1, i1), (n2, s2, i2), (n3, s3, i3) = I.kappa_scenarios()
    assert (n1, n2, n3) == ("I", "II", "III")
    assert I.boundary_contact(s1, i1[0])[0] == 2          # two faces on the boundary
    f2, e2 = I.boundary_contact(s2, i2[0])
    assert f2 == 0 and e2 >= 1                             # an edge, no face
    assert I.boundary_contact(s3, i3[0]) == (0, 0)
    ext = np.array(s3)
    for p in I.macro_vertices(s3)[i3[0]]:                  # not even a vertex
        assert np.all(np.array(p) > 0) and np.all(np.array(p) < ext)
    # boundary contact by brute force on scenario II's mesh: a face lies on the
    # boundary iff its three vertices share a coordinate plane of the cube
    for t, v in enumerate(I.macro_vertices(s2)):
        faces = 0
        for tri in itertools.combinations(v, 3):
            P = np.array(tri)
            faces += any(np.all(P[:, a] == 0) or np.all(P[:, a] == s2[a]) for a in range(3))
        assert faces == I.boundary_contact(s2, t)[0]


def test_five_tetrahedra_meshes_are_conforming_and_oriented():
    for sub, seed in [((2, 2, 2), None), ((3, 2, 1), 3)]:
        v, t = I.five_tet_macro_mesh(sub, seed=seed, amp=0.12)
        assert len(t) == 5 * int(np.prod(sub))
        dets = [np.linalg.det((v[tt[1:]] - v[tt[0]]).T) for tt in t]
        assert min(dets) > 0.0                                    # positive orientation
        faces = {}
        for tt in t:
            for f in itertools.combinations(sorted(tt), 3):
                faces[f] = faces.get(f, 0) + 1
        assert max(faces.values()) == 2                           # a face joins at most two
        for f, c in faces.items():                                # outer faces on the cube
            P = v[list(f)]
            on = any(np.allclose(P[:, a], 0.0) or np.allclose(P[:, a], 1.0) for a in range(3))
            assert on == (c == 1)
        assert abs(sum(abs(d) for d in dets) / 6.0 - 1.0) < 1e-12
    # the cube family as a general mesh: six Kuhn tetrahedra per sub-cube
    v, t = I.kuhn_macro_mesh((2, 1, 1))
    assert len(t) == 12 and np.allclose(v[t[0]], np.array(I.macro_vertices((2, 1, 1))[0]) / [2, 1, 1])
