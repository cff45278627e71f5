"""Host logic of the general-connectivity mesh builder on the CPU
(paper_1506_06185_gb300/csrc/mesh.cpp, build_general_mesh and
build_general_problem, compiled with the check program in tests/host/)
against the general-mesh oracle (oracle/unstructured.py): node keys, the
operator applied through macro blocks and copy lists, the interface smoother
classes, and for the global problem and the three recovery problem kinds
(§4.2 Algorithm 1, §4.3 Algorithm 2) the restriction gathers and the coarse
CG matrix (§2.1, §3.1, §3.2 Fig. 4), on meshes of another connectivity than
the cube family; and a host model of the device V-cycle (those tables driven
with the kernels' per-node arithmetic and order, tests/host/general_vcycle.cpp)
against the oracle's V-cycle iterates and, with a fault, its LR / DD / DN
recovery (§2.2, §4.2 Algorithm 1, §4.3 Algorithm 2)."""

import os
import shutil
import subprocess

import numpy as np
import pytest

import hhg_inputs as I
from oracle import unstructured as U

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def check_prog(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    cuda_inc = "/usr/local/cuda/include"
    if not cxx or not os.path.isdir(cuda_inc):
        pytest.skip("needs a C++ compiler and the CUDA headers")
    out = tmp_path_factory.mktemp("generalcheck") / "general_check"
    subprocess.check_call([cxx, "-O1", "-std=c++17", "-I" + cuda_inc, "-o", str(out),
                           os.path.join(ROOT, "tests", "host", "general_check.cpp"),
                           os.path.join(ROOT, "paper_1506_06185_gb300", "csrc", "mesh.cpp")])
    return str(out)


def _perm(path, lv):
    """Library node order -> oracle node id, matched by node keys."""
    keys = np.fromfile(path, dtype=np.int64).reshape(-1, 5)
    assert len(keys) == lv.n
    okeys = {tuple(k): q for q, k in enumerate(lv.keys.tolist())}
    return np.array([okeys[tuple(k)] for k in keys.tolist()])


@pytest.mark.parametrize("mesh,R,faulty", [("five", 4, [0, 1, 2, 3, 4]), ("five-moved", 4, [7, 12]),
                                           ("kuhn", 3, [3, 4, 5])])
def test_general_builder_matches_oracle(check_prog, tmp_path, mesh, R, faulty):
    if mesh == "kuhn":
        v, t = I.kuhn_macro_mesh((2, 1, 2))
    else:
        v, t = I.five_tet_macro_mesh((2, 2, 1), seed=3 if mesh == "five-moved" else None, amp=0.12)
    coeff = np.exp(np.random.default_rng(6).standard_normal(len(t)))
    np.ascontiguousarray(v, dtype=np.float64).tofile(tmp_path / "verts.bin")
    np.ascontiguousarray(t, dtype=np.int32).tofile(tmp_path / "tets.bin")
    coeff.tofile(tmp_path / "coeff.bin")
    subprocess.check_call([check_prog, str(len(v)), str(len(t)), str(R), str(tmp_path), str(len(faulty)),
                           *map(str, faulty)])
    om = U.UMesh(v, t, R, coeff=coeff)
    perms = []
    for l, lv in enumerate(om.levels):
        perm = _perm(tmp_path / f"keys_{l}.bin", lv)
        assert np.array_equal(np.sort(perm), np.arange(lv.n))       # a bijection
        perms.append(perm)
        # A g through blocks and copy lists = the oracle's assembled operator
        g = np.fromfile(tmp_path / f"g_{l}.bin")
        Ag = np.fromfile(tmp_path / f"Ag_{l}.bin")
        go = np.zeros(lv.n)
        go[perm] = g
        ref = (lv.A @ go)[perm]
        assert np.abs(Ag - ref).max() <= 1e-13 * np.abs(ref).max()
        # interface classes = the oracle's, Dirichlet nodes marked
        cls = np.fromfile(tmp_path / f"cls_{l}.bin", dtype=np.int32)
        n_if = len(cls)
        ocls = np.full(lv.n, -1)
        for c, members in enumerate(lv.classes[4:]):
            ocls[members] = c
        assert np.array_equal(cls, ocls[perm[:n_if]])
        assert np.all(lv.dim[perm[:n_if]] < 4) and np.all(lv.dim[perm[n_if:]] == 4)
    if mesh != "kuhn":
        # the five-tetrahedra meshes have coarse nodes with more than 15 fine
        # neighbours: the variable-length gathers are exercised
        cols = np.diff(om.P[0].tocsc().indptr)
        assert cols[(om.levels[0].dim < 4) & ~om.levels[0].boundary].max() > 15
    # per problem kind: restriction gathers = P^T on the free coarse interface
    # nodes, coarse CG matrix = the level-0 operator (A_I for kind 3) on the
    # free nodes
    hm = om.healthy(faulty)
    fmasks = om.fault_masks(faulty)
    kinds = [om.global_masks(), om.local_masks(faulty), om.healthy_masks(faulty),
             [~lv.boundary & ~o for lv, (o, _) in zip(om.levels, fmasks)]]
    for kind, free in enumerate(kinds):
        for l in range(len(om.levels) - 1):
            r = np.fromfile(tmp_path / f"r_{kind}_{l + 1}.bin")
            ro = np.zeros(om.levels[l + 1].n)
            ro[perms[l + 1]] = r
            ro[~free[l + 1]] = 0.0
            rc = om.P[l].T @ ro
            d = np.fromfile(tmp_path / f"rc_{kind}_{l}.bin").reshape(-1, 2)
            ids = perms[l][d[:, 0].astype(np.int64)]
            want = np.nonzero(free[l] & (om.levels[l].dim < 4))[0]
            assert sorted(ids.tolist()) == want.tolist()
            assert np.abs(rc[ids] - d[:, 1]).max(initial=0.0) <= 1e-13 * max(1.0, np.abs(rc).max())
        lv0 = (hm if kind == 3 else om).levels[0]
        dump = np.fromfile(tmp_path / f"csr_{kind}.bin")
        n, pos = int(dump[0]), 1
        A = lv0.A.tocsr()
        rows = []
        for _ in range(n):
            gid, nnz = int(dump[pos]), int(dump[pos + 1])
            pos += 2
            o = perms[0][gid]
            rows.append(o)
            refr = A.getrow(o).toarray().ravel()
            refr[~free[0]] = 0.0
            mine = np.zeros_like(refr)
            for _ in range(nnz):
                mine[perms[0][int(dump[pos])]] += dump[pos + 1]
                pos += 2
            assert np.abs(mine - refr).max() <= 1e-13 * max(np.abs(refr).max(), 1e-300)
        assert sorted(rows) == np.nonzero(free[0])[0].tolist()


def _lib_to_oracle(om, tets):
    """Library node order -> oracle node id: the interface nodes in the same
    key order, then the volume nodes macro by macro, local order k, j, i."""
    lv = om.levels[-1]
    N = lv.N
    n_if = int((lv.dim < 4).sum())
    okeys = {tuple(k): q for q, k in enumerate(lv.keys.tolist())}
    perm = list(range(n_if))
    for t in tets:
        for k in range(1, N):
            for j in range(1, N - k):
                for i in range(1, N - j - k):
                    w = [N - i - j - k, i, j, k]
                    perm.append(okeys[(4, *sorted(int(g) * (N + 1) + ww for g, ww in zip(t, w)))])
    return np.array(perm)


@pytest.fixture(scope="module")
def vcycle_prog(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    cuda_inc = "/usr/local/cuda/include"
    if not cxx or not os.path.isdir(cuda_inc):
        pytest.skip("needs a C++ compiler and the CUDA headers")
    out = tmp_path_factory.mktemp("generalvcycle") / "general_vcycle"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I" + cuda_inc, "-o", str(out),
                           os.path.join(ROOT, "tests", "host", "general_vcycle.cpp"),
                           os.path.join(ROOT, "paper_1506_06185_gb300", "csrc", "mesh.cpp")])
    return str(out)


@pytest.mark.parametrize("moved", [False, True])
def test_host_model_of_the_device_vcycle_matches_oracle(vcycle_prog, tmp_path, moved):
    """The library's tables driven with its kernels' per-node arithmetic and
    order (a host model of the device V-cycle) give the oracle's iterates."""
    v, t = I.five_tet_macro_mesh((2, 2, 1), seed=3 if moved else None, amp=0.12)
    R = 4
    coeff = np.exp(np.random.default_rng(9).standard_normal(len(t)))
    om = U.UMesh(v, t, R, coeff=coeff)
    lv = om.levels[-1]
    perm = _lib_to_oracle(om, t)
    assert np.array_equal(np.sort(perm), np.arange(lv.n))
    rng = np.random.default_rng(4)
    fo = np.where(lv.boundary, 0.0, rng.uniform(-1, 1, lv.n))
    uo = np.where(lv.boundary, np.exp(np.pi * lv.X[:, 0]) * np.sin(np.pi * lv.X[:, 1]), 0.0)
    np.ascontiguousarray(v, dtype=np.float64).tofile(tmp_path / "verts.bin")
    np.ascontiguousarray(t, dtype=np.int32).tofile(tmp_path / "tets.bin")
    coeff.tofile(tmp_path / "coeff.bin")
    fo[perm].tofile(tmp_path / "f.bin")
    uo[perm].tofile(tmp_path / "u0.bin")
    cycles = 4
    subprocess.check_call([vcycle_prog, str(len(v)), str(len(t)), str(R), str(cycles), str(tmp_path)])
    masks = om.global_masks()
    for c in range(cycles):
        U.vcycle(om, len(om.levels) - 1, uo, fo, masks)
        ul = np.fromfile(tmp_path / f"u_{c}.bin")
        assert np.linalg.norm(ul - uo[perm]) <= 1e-11 * np.linalg.norm(uo), c


@pytest.mark.parametrize("recovery", ["LR", "DD", "DN"])
def test_host_model_of_the_device_fault_recovery_matches_oracle(vcycle_prog, tmp_path, recovery):
    """Fault after cycle 2 on one sub-cube's five macros and its LR / DD / DN
    recovery through the library's tables and the kernels' arithmetic (DN in
    the device's block schedule): the residual history and the iterates
    equal the oracle's."""
    v, t = I.five_tet_macro_mesh((2, 2, 1), seed=3, amp=0.12)
    R = 4
    om = U.UMesh(v, t, R)
    lv = om.levels[-1]
    perm = _lib_to_oracle(om, t)
    fo = np.where(lv.boundary, 0.0, np.random.default_rng(8).uniform(-1, 1, lv.n))
    uo = np.zeros(lv.n)
    np.ascontiguousarray(v, dtype=np.float64).tofile(tmp_path / "verts.bin")
    np.ascontiguousarray(t, dtype=np.int32).tofile(tmp_path / "tets.bin")
    np.ones(len(t)).tofile(tmp_path / "coeff.bin")
    fo[perm].tofile(tmp_path / "f.bin")
    uo[perm].tofile(tmp_path / "u0.bin")
    ids = [5, 6, 7, 8, 9]
    cycles, n_local, n_global = 5, 3, 2
    rec = {"LR": 1, "DD": 2, "DN": 3}[recovery]
    eta = 2.5
    subprocess.check_call([vcycle_prog, str(len(v)), str(len(t)), str(R), str(cycles), str(tmp_path), "2", str(rec),
                           str(n_local), str(n_global), str(len(ids)), *map(str, ids), str(eta)])
    kw = {"LR": dict(recovery=U.LR, n_local=n_local),
          "DD": dict(recovery=U.DD, n_local=n_local, n_global=n_global),
          "DN": dict(recovery=U.DN, n_global=n_global, eta=eta)}[recovery]
    hist_o = U.solve(om, uo, fo, rtol=0.0, max_cycles=cycles, fault_cycle=2, fault_ids=ids, **kw)
    hist = np.fromfile(tmp_path / "hist.bin")
    assert len(hist) == len(hist_o) == cycles + 2
    assert np.abs(hist - hist_o).max() <= 1e-11
    ul = np.fromfile(tmp_path / f"u_{cycles - 1}.bin")
    assert np.linalg.norm(ul - uo[perm]) <= 1e-11 * np.linalg.norm(uo)
