"""Mixed precision: FP32 smoothing, transfers and recovery cycles inside FP64
iterative refinement (FP64 fine residual, update and coarse CG).  Parity is on
the final residual (the same stopping test as FP64); the solution's error
against the FP64 oracle is bounded and printed."""

import numpy as np
import pytest

import hhg_inputs as I
import oracle as O
from parity import assert_close, errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hhg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1506_06185_gb300 import build
    from paper_1506_06185_gb300 import hhg as H
    build()
    return H


def _check(hhg, sub, R, f, u0, coeff=None, **kw):
    M = hhg.Mesh(sub, R, precision=32, coeff=coeff)
    M.set_problem(f, u0)
    hist, cyc, _ = M.solve(mixed_precision=True, **kw)
    ug = M.get_solution()
    m = O.Mesh(sub, R, coeff=coeff)
    uo = O.pad(u0.copy())
    okw = {k: v for k, v in kw.items() if k in ("rtol", "max_cycles", "fault_cycle", "fault_ids", "recovery",
                                                  "n_local", "n_global", "eta")}
    ref = O.solve(m, uo, O.pad(f), **okw)
    err, err_max = errors(ug, O.interior(uo))
    print(f"mixed: {cyc} cycles (FP64 oracle {ref['cycles']}), final rel. residual {hist[-1]:.2e}, "
          f"|u - u_oracle| / |u_oracle| = {err:.2e}, max-norm {err_max:.2e}")
    assert hist[-1] <= kw["rtol"]
    assert abs(cyc - ref["cycles"]) <= 1
    # both solutions satisfy the same stopping test ||r|| <= rtol ||r_0||, so
    # each is within cond(A) rtol (relative) of the discrete solution; on
    # meshes refined 4-5 times cond(A) ~ 4^R <= 1e3, which bounds the two
    # solutions' difference node by node
    assert_close(ug, O.interior(uo), 1e3 * kw["rtol"], what="mixed vs FP64 oracle")
    M.close()
    return err


def test_mixed_config1_fault_lr(hhg):
    sub, R = (2, 2, 2), 4
    g = I.harmonic_boundary(sub, R)
    _check(hhg, sub, R, np.zeros(g.shape), I.initial_guess(sub, R, g), rtol=1e-10, max_cycles=40,
           fault_cycle=5, fault_ids=[0], recovery=1, n_local=2)


def test_mixed_dd_subcube_random_load(hhg):
    sub, R = (2, 2, 2), 5
    f = I.random_load(sub, R, seed=0)
    _check(hhg, sub, R, f, I.initial_guess(sub, R), rtol=1e-10, max_cycles=40, fault_cycle=5,
           fault_ids=I.subcube_macros(sub), recovery=2, n_global=2, eta=4.0)


def test_mixed_coefficients_fault_free(hhg):
    sub, R = (3, 2, 2), 5
    coeff = np.exp(np.random.default_rng(4).standard_normal(72))
    f = I.random_load(sub, R, seed=1)
    _check(hhg, sub, R, f, I.initial_guess(sub, R), coeff=coeff, rtol=1e-10, max_cycles=40)


def test_mixed_needs_precision32_mesh(hhg):
    M = hhg.Mesh((1, 1, 1), 3)
    with pytest.raises(hhg.HHGError) as e:
        M.solve(rtol=1e-6, max_cycles=5, mixed_precision=True)
    assert e.value.code == hhg.HHG_ERR_STATE
    M.close()


@pytest.mark.slow
def test_mixed_full_size_refined_9_levels_with_fault():
    """2x2x2x6 macros refined 9 levels (1.07e9 unknowns): FP32 cycles inside
    FP64 iterative refinement, fault after cycle 4 on sub-cube (0,0,0), DD
    recovery (eta = 4, n_I = 3), to 1e-8.  The FP64 GPU solve of the same
    problem is the comparison; the oracle's residual assembled row by row at
    sampled nodes checks the mixed solution (a wrong stencil anywhere sampled
    would leave O(1) residuals)."""
    import torch
    assert torch.cuda.is_available()
    from paper_1506_06185_gb300 import build
    from paper_1506_06185_gb300 import hhg
    build()
    sub, R = (2, 2, 2), 9
    f = I.random_load(sub, R, seed=0)
    fd = torch.from_numpy(f).cuda()
    u0 = torch.zeros_like(fd)
    M = hhg.Mesh(sub, R, precision=32)
    kw = dict(rtol=1e-8, max_cycles=40, fault_cycle=4, fault_ids=I.subcube_macros(sub), recovery=2, n_global=3,
              eta=4.0)
    M.set_problem(fd, u0)
    h64, c64, _ = M.solve(**kw)
    u64 = torch.zeros_like(fd)
    M.get_solution(u64)
    M.set_problem(None, u0)
    h32, c32, _ = M.solve(mixed_precision=True, **kw)
    u32 = torch.zeros_like(fd)
    M.get_solution(u32)
    M.close()
    del fd
    diff = float((u32 - u64).norm() / u64.norm())
    print(f"r=9: FP64 {c64} cycles, mixed {c32} cycles, |u_mixed - u_fp64| / |u_fp64| = {diff:.2e}")
    assert h64[-1] <= 1e-8 and h32[-1] <= 1e-8 and abs(c32 - c64) <= 1
    assert diff <= 1e-6
    u = u32.cpu().numpy()
    del u32, u64
    r0 = np.linalg.norm(f[~I.boundary_mask(sub, R)])
    rng = np.random.default_rng(12)
    n = 1 << R
    nodes = rng.integers(1, 2 * n, size=(200, 3))
    nodes[:30] = np.maximum((nodes[:30] // 4) * 4, 4)
    nodes[30:50, 1] = n
    r = O.local_residual(sub, R, np.ones(48), None, u, f, nodes)
    # the stopping test bounds the global residual norm by 1e-8 r0
    assert np.abs(r).max() <= 1e-8 * r0, np.abs(r).max() / r0
