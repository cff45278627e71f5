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
