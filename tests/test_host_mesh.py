"""Host logic of the CUDA path on the CPU: the mesh builder's per-macro
stencils, interface copies, restriction gathers and coarse CG matrices
(paper_1506_06185_gb300/csrc/mesh.cpp, compiled with the check program in
tests/host/) against the oracle's element-by-element assembly (§2.1, §3.2
Fig. 4), on the cube, on a sheared cube with per-macro coefficients and on
meshes with moved sub-cube corners (general macro shapes), for the global
problem and the three recovery problem kinds."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import hhg_inputs as I
import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHEAR = np.array([[1.0, 0.3, -0.2], [0.1, 0.9, 0.25], [-0.15, 0.2, 1.1]])


@pytest.fixture(scope="module")
def check_prog(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    cuda_inc = "/usr/local/cuda/include"
    if not cxx or not os.path.isdir(cuda_inc):
        pytest.skip("needs a C++ compiler and the CUDA headers")
    out = tmp_path_factory.mktemp("meshcheck") / "mesh_check"
    subprocess.check_call([cxx, "-O1", "-std=c++17", "-I" + cuda_inc, "-o", str(out),
                           os.path.join(ROOT, "tests", "host", "mesh_check.cpp"),
                           os.path.join(ROOT, "paper_1506_06185_gb300", "csrc", "mesh.cpp")])
    return str(out)


def _problems(m, faulty):
    probs = [m.global_problem]
    if faulty:
        masks = m.fault_masks(faulty)
        probs += [m.local_problem(faulty), m.healthy_problem(faulty),
                  O.Problem(m, [(~lv.boundary) & ~o for lv, (o, _) in zip(m.levels, masks)])]
    return probs


@pytest.mark.parametrize("sub,R,geometry,faulty", [
    ((2, 2, 2), 4, 0, [13]),
    ((2, 1, 2), 4, 1, [0, 1, 2, 3, 4, 5]),
    ((3, 2, 2), 4, 1, [13, 14, 30]),
    ((2, 2, 1), 4, 2, [6, 7, 8, 9, 10, 11]),
    ((2, 2, 2), 3, 2, [13, 20]),
])
def test_mesh_builder_matches_oracle(check_prog, tmp_path, sub, R, geometry, faulty):
    n_macro = 6 * sub[0] * sub[1] * sub[2]
    coeff = np.exp(np.random.default_rng(3).standard_normal(n_macro))
    coeff.tofile(tmp_path / "coeff.bin")
    aff = SHEAR if geometry == 1 else None
    vp = I.jittered_vertices(sub, seed=4) if geometry == 2 else None
    if vp is not None:
        vp.tofile(tmp_path / "vpos.bin")
    m = O.Mesh(sub, R, coeff=coeff, affine=aff, vertex_pos=vp)
    rng = np.random.default_rng(0)
    ins = []
    for l, lv in enumerate(m.levels):
        g = rng.standard_normal(lv.shape)
        g.tofile(tmp_path / f"in_{l}.bin")
        ins.append(g)
    probs = _problems(m, faulty)
    for kind, pr in enumerate(probs):
        for l in range(1, len(m.levels)):
            r = rng.standard_normal(m.levels[l].shape)
            r[~pr.free[l]] = 0.0
            r.tofile(tmp_path / f"r_{kind}_{l}.bin")
    subprocess.check_call([check_prog, *map(str, sub), str(R), str(geometry), str(tmp_path), str(len(faulty)),
                           *map(str, faulty)])
    # stencils: A g through blocks and copy lists = the assembled operator
    for l, lv in enumerate(m.levels):
        Ag = np.fromfile(tmp_path / f"Ag_{l}.bin").reshape(lv.shape)
        ref = O.apply_A(lv, O.pad(ins[l]))
        inner = ~lv.boundary
        assert np.abs(Ag[inner] - ref[inner]).max() <= 1e-13 * np.abs(ref).max()
    hm = O.hhg_oracle.healthy_mesh(m, faulty)
    for kind, pr in enumerate(probs):
        # restriction gathers = full weighting R = P^T at the free coarse interface nodes
        for l in range(len(m.levels) - 1):
            r = np.fromfile(tmp_path / f"r_{kind}_{l + 1}.bin").reshape(m.levels[l + 1].shape)
            rc = O.restrict(r)
            d = np.fromfile(tmp_path / f"rc_{kind}_{l}.bin").reshape(-1, 2)
            g = d[:, 0].astype(np.int64)
            if len(g):
                assert np.abs(rc.ravel()[g] - d[:, 1]).max() <= 1e-12 * max(1.0, np.abs(rc).max())
        # coarse CG matrix = the level-0 operator (A_I for the Neumann side) on the free nodes
        dump = np.fromfile(tmp_path / f"csr_{kind}.bin")
        n, pos = int(dump[0]), 1
        A = O.dia_to_csr((hm if kind == 3 else m).levels[0]).tocsr()
        free = pr.free[0].ravel()
        rows = []
        for _ in range(n):
            gid, nnz = int(dump[pos]), int(dump[pos + 1])
            pos += 2
            rows.append(gid)
            ref = A.getrow(gid).toarray().ravel()
            ref[~free] = 0.0
            mine = np.zeros_like(ref)
            for _ in range(nnz):
                mine[int(dump[pos])] += dump[pos + 1]
                pos += 2
            assert np.abs(mine - ref).max() <= 1e-13 * np.abs(ref).max()
        assert sorted(rows) == sorted(np.nonzero(free)[0].tolist())
        # interface stencil tables (summed weights per distinct neighbour) =
        # the level's operator (A_I for the Neumann side) at the free
        # interface nodes; every level above the coarsest has them
        opm = hm if kind == 3 else m
        for l in range(1, len(m.levels)):
            fn = tmp_path / f"At_{kind}_{l}.bin"
            assert fn.exists(), fn
            d = np.fromfile(fn).reshape(-1, 2)
            ref = O.apply_A(opm.levels[l], O.pad(ins[l])).ravel()
            g = d[:, 0].astype(np.int64)
            assert len(g) == len(np.unique(g))
            assert np.abs(ref[g] - d[:, 1]).max(initial=0.0) <= 1e-13 * np.abs(ref).max()
