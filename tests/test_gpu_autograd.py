"""Differentiation through the solve: the adjoint gradients of
L = 1/2 ||u - u_target||^2 with respect to the load vector f and the per-macro
coefficients k, against the oracle's adjoint (direct solves) and against
central finite differences of GPU solves."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import hhg_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1506_06185_gb300 import build
    build()
    from paper_1506_06185_gb300 import autograd as AG
    from paper_1506_06185_gb300 import hhg as H
    return torch, H, AG


def _direct(lv, rhs, free):
    A = O.dia_to_csr(lv)
    fr = free.ravel()
    x = np.zeros(fr.size)
    x[fr] = spla.spsolve(A[fr][:, fr].tocsc(), rhs.ravel()[fr])
    return x.reshape(lv.shape)


def _loss(torch, u, ut, mask):
    return 0.5 * ((u - ut)[~mask] ** 2).sum()


def test_adjoint_gradients_match_oracle(mods):
    torch, H, AG = mods
    sub, R = (2, 2, 2), 4
    k0 = I.lognormal_coeff(48, seed=1)
    f = I.random_load(sub, R, seed=3)
    ut = I.smooth_target(sub, R)
    mask = I.boundary_mask(sub, R)
    M = H.Mesh(sub, R, coeff=k0)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    kt = torch.from_numpy(k0.copy()).cuda().requires_grad_(True)
    u = AG.solve(M, ft, kt, rtol=1e-13, max_cycles=80)
    loss = _loss(torch, u, torch.from_numpy(ut).cuda(), torch.from_numpy(mask).cuda())
    loss.backward()
    # oracle: forward and adjoint by sparse direct solves, gradient by element sums
    lv = O.Level(sub, R, k0)
    free = ~lv.boundary
    uo = _direct(lv, f, free)
    lam = _direct(lv, np.where(free, uo - ut, 0.0), free)
    m = O.Mesh(sub, R, coeff=k0)
    gk = O.grad_coeff(m, O.pad(uo), O.pad(lam))
    assert np.abs(u.detach().cpu().numpy() - uo).max() <= 1e-10 * np.abs(uo).max()
    gf = ft.grad.cpu().numpy()
    assert np.abs(gf - lam).max() <= 1e-9 * np.abs(lam).max()
    gk_gpu = kt.grad.cpu().numpy()
    assert np.abs(gk_gpu - gk).max() <= 1e-8 * np.abs(gk).max(), (gk_gpu[:4], gk[:4])
    M.close()


def test_coefficient_gradient_central_differences(mods):
    torch, H, AG = mods
    sub, R = (2, 1, 2), 4
    n = 24
    k0 = I.lognormal_coeff(n, seed=5)
    f = torch.from_numpy(I.random_load(sub, R, seed=6)).cuda()
    ut = torch.from_numpy(I.smooth_target(sub, R)).cuda()
    mask = torch.from_numpy(I.boundary_mask(sub, R)).cuda()
    M = H.Mesh(sub, R, coeff=k0)
    opts = dict(rtol=1e-13, max_cycles=80)

    def L(k):
        with torch.no_grad():
            return float(_loss(torch, AG.solve(M, f, torch.from_numpy(k).cuda(), **opts), ut, mask))

    kt = torch.from_numpy(k0.copy()).cuda().requires_grad_(True)
    loss = _loss(torch, AG.solve(M, f, kt, **opts), ut, mask)
    loss.backward()
    g = kt.grad.cpu().numpy()
    h = 1e-6
    for d in I.random_directions(n, 4, seed=2):
        fd = (L(k0 + h * d) - L(k0 - h * d)) / (2 * h)
        assert abs(fd - g @ d) <= 1e-5 * max(abs(fd), 1e-12) + 1e-9, (fd, g @ d)
    M.close()


def test_coefficient_gradient_sixteen_directions_384_macros(mods):
    """The differentiation workload's shape at a size the test affords: 4x4x4
    sub-cubes x 6 = 384 macros (refined 4 times), k ~ lognormal(0, 1) (seed
    1), loss 1/2 ||u - u_target||^2 with the smooth target; the adjoint
    gradient against central differences (h = 1e-6) on 16 random coefficient
    directions (seed 2)."""
    torch, H, AG = mods
    sub, R = (4, 4, 4), 4
    n = 384
    k0 = I.lognormal_coeff(n, seed=1)
    f = torch.from_numpy(I.random_load(sub, R, seed=0)).cuda()
    ut = torch.from_numpy(I.smooth_target(sub, R)).cuda()
    mask = torch.from_numpy(I.boundary_mask(sub, R)).cuda()
    M = H.Mesh(sub, R, coeff=k0)
    opts = dict(rtol=1e-13, max_cycles=100)

    def L(k):
        with torch.no_grad():
            return float(_loss(torch, AG.solve(M, f, torch.from_numpy(k).cuda(), **opts), ut, mask))

    kt = torch.from_numpy(k0.copy()).cuda().requires_grad_(True)
    loss = _loss(torch, AG.solve(M, f, kt, **opts), ut, mask)
    loss.backward()
    g = kt.grad.cpu().numpy()
    h = 1e-6
    worst = 0.0
    for d in I.random_directions(n, 16, seed=2):
        fd = (L(k0 + h * d) - L(k0 - h * d)) / (2 * h)
        err = abs(fd - g @ d) / max(abs(fd), 1e-12)
        worst = max(worst, err)
        assert abs(fd - g @ d) <= 1e-5 * max(abs(fd), 1e-12) + 1e-9, (fd, g @ d)
    print(f"384 macros, 16 directions: largest relative gap to central differences {worst:.2e}")
    M.close()
