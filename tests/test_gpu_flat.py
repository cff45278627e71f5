"""The flat kernels (hhg_set_flat_gs) against the oracle and the tile kernels.

The flat Gauss-Seidel, residual and prolongation kernels give every thread one
16-byte vector of same-colour nodes, and the flat restriction one slot of four
coarse nodes, looked up in per-level item tables, instead of walking row-pair
tiles; their
per-item arithmetic is the tile kernels', and a colour's nodes read only
other colours, so the iterate must equal the tile kernels' bit for bit (the
residual norms only up to the order of their partial sums).  Each
test runs a mesh with the flat kernel on every smoothed level next to a twin
on the tile kernel and compares:
  * the iterates with the oracle node by node (parity.assert_close) and the
    residual histories with the oracle's,
  * the flat and the tile iterates bit for bit,
for FP64 V-cycles, a Dirichlet-Dirichlet and a Dirichlet-Neumann recovery
(the sub-problems of Algorithms 1 and 2 use the kernel too) and FP32 cycles
inside FP64 refinement.  Meshes without the 7-point structure ignore the
setting; meshes of general connectivity refuse it.
(§2.1 smoother and V-cycle; §4.2 Algorithm 1; §4.3 Algorithm 2.)
"""

import numpy as np
import pytest

import hhg_inputs as I
import oracle as O
from parity import assert_close

pytestmark = pytest.mark.gpu

ATOL_HIST = 1e-12
SHEAR = np.array([[1.0, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.1]])


@pytest.fixture(scope="module")
def hhg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1506_06185_gb300 import build
    from paper_1506_06185_gb300 import hhg as H
    build()
    return H


def _twins(hhg, sub, R, f, u0, **mesh_kw):
    """A mesh on the flat kernel and a twin on the tile kernel, same problem."""
    F = hhg.Mesh(sub, R, **mesh_kw)
    T = hhg.Mesh(sub, R, **mesh_kw)
    hhg.hhg_set_flat_gs(F.h, True)
    for M in (F, T):
        M.set_problem(f, u0)
    return F, T


@pytest.mark.parametrize("sub,R", [((2, 2, 2), 5), ((3, 2, 2), 6)])
def test_flat_vcycles(hhg, sub, R):
    f = I.random_load(sub, R, seed=11)
    u0 = I.initial_guess(sub, R, I.harmonic_boundary(sub, R))
    F, T = _twins(hhg, sub, R, f, u0)
    m = O.Mesh(sub, R)
    uo, fo = O.pad(u0.copy()), O.pad(f)
    r0 = O.resnorm(m, uo, fo)
    top = len(m.levels) - 1
    for k in range(4):
        rf = F.vcycle()
        rt = T.vcycle()
        O.vcycle(m, m.global_problem, top, uo, fo)
        uf, ut = F.get_solution(), T.get_solution()
        assert_close(uf, O.interior(uo), what=f"cycle {k}")
        assert np.array_equal(uf, ut), f"cycle {k}: flat and tile kernels differ"
        ro = O.resnorm(m, uo, fo)
        # the norms' partial sums follow each kernel's grid: equal up to rounding
        assert abs(rf - ro) <= ATOL_HIST * r0 and abs(rf - rt) <= 1e-14 * r0, k
    F.close()
    T.close()


def _solve_both(hhg, sub, R, f, u0, kw, mesh_kw=None):
    mesh_kw = mesh_kw or {}
    F, T = _twins(hhg, sub, R, f, u0, **mesh_kw)
    hf, cf, _ = F.solve(**kw)
    ht, ct, _ = T.solve(**kw)
    m = O.Mesh(sub, R, **mesh_kw)
    uo = O.pad(u0.copy())
    okw = dict(rtol=kw["rtol"], max_cycles=kw["max_cycles"], fault_cycle=kw.get("fault_cycle", -1),
               fault_ids=kw.get("fault_ids", ()), recovery=kw.get("recovery", 0), n_local=kw.get("n_local", 0),
               n_global=kw.get("n_global", 0), eta=kw.get("eta", 1.0))
    ref = O.solve(m, uo, O.pad(f), **okw)
    assert cf == ct == ref["cycles"]
    assert np.abs(hf - ref["hist"]).max() <= ATOL_HIST
    uf, ut = F.get_solution(), T.get_solution()
    assert_close(uf, O.interior(uo), what="solve")
    assert np.array_equal(uf, ut), "flat and tile kernels differ"
    F.close()
    T.close()


def test_flat_dirichlet_dirichlet(hhg):
    """DD (Algorithm 1) on a sub-cube: Omega_F and Omega_I cycles on the flat kernel."""
    sub, R = (2, 2, 2), 6
    f = I.random_load(sub, R, seed=12)
    _solve_both(hhg, sub, R, f, I.initial_guess(sub, R),
                dict(rtol=1e-9, max_cycles=40, fault_cycle=3, fault_ids=I.subcube_macros(sub, 1, 0, 1), recovery=2,
                     n_global=2, eta=3.0))


def test_flat_dirichlet_neumann(hhg):
    """DN (Algorithm 2): the Neumann side reaches Gamma through its own copy lists."""
    sub, R = (3, 2, 2), 5
    f = I.random_load(sub, R, seed=13)
    _solve_both(hhg, sub, R, f, I.initial_guess(sub, R),
                dict(rtol=1e-9, max_cycles=40, fault_cycle=3, fault_ids=[13, 14, 30, 31], recovery=3, n_global=2,
                     eta=2.0))


def test_flat_mixed_precision(hhg):
    """FP32 cycles inside FP64 refinement on the flat kernel (FP32 item tables)."""
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=14)
    u0 = I.initial_guess(sub, R)
    kw = dict(rtol=1e-10, max_cycles=40, fault_cycle=4, fault_ids=I.subcube_macros(sub), recovery=2, n_global=2,
              eta=4.0, mixed_precision=True)
    F, T = _twins(hhg, sub, R, f, u0, precision=32)
    hf, cf, _ = F.solve(**kw)
    ht, ct, _ = T.solve(**kw)
    assert cf == ct and np.abs(hf - ht).max() <= 1e-14 and hf[-1] <= 1e-10
    assert np.array_equal(F.get_solution(), T.get_solution())
    F.close()
    T.close()


def test_flat_switch_off_and_fifteen_point(hhg):
    """Switching the kernel off restores the tile kernel (same bits); a sheared
    15-point mesh ignores the setting."""
    sub, R = (2, 1, 2), 5
    f = I.random_load(sub, R, seed=15)
    u0 = I.initial_guess(sub, R)
    F, T = _twins(hhg, sub, R, f, u0)
    F.vcycle()
    hhg.hhg_set_flat_gs(F.h, False)
    F.vcycle()
    T.vcycle()
    T.vcycle()
    assert np.array_equal(F.get_solution(), T.get_solution())
    F.close()
    T.close()
    coeff = np.exp(np.random.default_rng(16).standard_normal(6 * 4))
    F, T = _twins(hhg, sub, R, f, u0, affine=SHEAR, coeff=coeff)
    for _ in range(2):
        F.vcycle()
        T.vcycle()
    assert np.array_equal(F.get_solution(), T.get_solution())
    F.close()
    T.close()


def test_flat_refused_on_general_meshes(hhg):
    verts, macros = I.five_tet_macro_mesh((1, 1, 1))
    G = hhg.Mesh.general(verts, macros, 3)
    with pytest.raises(hhg.HHGError) as e:
        hhg.hhg_set_flat_gs(G.h, True)
    assert e.value.code == hhg.HHG_ERR_STATE
    G.close()
