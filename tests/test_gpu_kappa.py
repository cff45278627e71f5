"""Cycle advantage of the recovery strategies (§4.4, Eq. (3), Tab. 1): the GPU
solve and the oracle must take the same number of global cycles for every
strategy, superman factor and n_I on Scenario I (one cube of six macros, the
fault in a tetrahedron with two faces on the boundary), refined 5 times."""

import math

import numpy as np
import pytest

import hhg_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hhg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1506_06185_gb300 import build
    from paper_1506_06185_gb300 import hhg as H
    build()
    return H


def _kw(rec, eta, n_I, k_F, ids):
    n_F = int(math.ceil(eta * n_I))
    if rec == O.LR:
        return dict(fault_cycle=k_F, fault_ids=ids, recovery=rec, n_local=n_F)
    return dict(fault_cycle=k_F, fault_ids=ids, recovery=rec, n_global=n_I, eta=eta)


def test_kappa_matches_oracle_scenario_I(hhg):
    name, sub, ids = I.kappa_scenarios()[0]
    R, k_F, rtol = 5, 5, 1e-10
    f = I.random_load(sub, R, seed=0)
    u0 = I.initial_guess(sub, R)
    M = hhg.Mesh(sub, R)
    m = O.Mesh(sub, R)
    M.set_problem(f, u0)
    _, free_gpu, _ = M.solve(rtol=rtol, max_cycles=60)
    free = O.solve(m, O.pad(u0.copy()), O.pad(f), rtol=rtol, max_cycles=60)["cycles"]
    assert free_gpu == free
    for rec in (O.LR, O.DD, O.DN):
        for eta in (2.0, 5.0):
            for n_I in (0, 1, 2, 3):
                kw = _kw(rec, eta, n_I, k_F, ids)
                M.set_problem(None, u0)
                hist, cyc, _ = M.solve(rtol=rtol, max_cycles=60, **kw)
                ref = O.solve(m, O.pad(u0.copy()), O.pad(f), rtol=rtol, max_cycles=60, **kw)
                assert cyc == ref["cycles"], (rec, eta, n_I, cyc, ref["cycles"])
                assert np.abs(hist - ref["hist"]).max() <= 1e-12
                # k_faulty = global cycles + n_I for every strategy (§4.4)
                kappa = O.kappa(cyc + n_I, free, k_F)
                assert 0.0 <= kappa <= 1.0 + n_I / k_F
    M.close()
