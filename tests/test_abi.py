"""The C ABI library builds, loads and exports every entry point that
include/hhg.h declares (no GPU needed: no compute call is made)."""

import os
import re

import pytest


def _declared(root):
    with open(os.path.join(root, "include", "hhg.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^int\s+(hhg_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary(root):
    names = _declared(root)
    for n in ["hhg_mesh_create", "hhg_vcycle", "hhg_inject_fault", "hhg_recover_local", "hhg_solve"]:
        assert n in names


def test_library_exports_every_declared_symbol(root):
    from paper_1506_06185_gb300 import build
    from paper_1506_06185_gb300 import hhg
    build()
    lib = hhg.load_library()
    for n in _declared(root):
        assert hasattr(lib, n), n
    assert sorted(hhg.EXPORTS) == sorted(n for n in _declared(root) if n in hhg.EXPORTS)
    assert set(_declared(root)) <= set(hhg.EXPORTS)


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1506_06185_gb300 import hhg
    with pytest.raises(hhg.HHGError) as e:
        hhg.Mesh((1, 1, 1), 3)
    assert e.value.code == hhg.HHG_ERR_CUDA


def test_invalid_arguments_are_rejected_before_device_use():
    from paper_1506_06185_gb300 import hhg
    for kw in ({"subcubes": (0, 1, 1), "levels": 3}, {"subcubes": (1, 1, 1), "levels": 2},
               {"subcubes": (1, 1, 1), "levels": 3, "precision": 16}):
        with pytest.raises(hhg.HHGError) as e:
            hhg.hhg_mesh_create(**kw)
        assert e.value.code == hhg.HHG_ERR_ARG


def test_null_handles_are_rejected_without_device_use():
    # every entry point called with NULL handles / pointers and zero sizes:
    # HHG_ERR_ARG with a message, destroying NULL is a no-op (no GPU needed)
    import ctypes as C
    from paper_1506_06185_gb300 import hhg
    lib = hhg.lib()
    buf = C.create_string_buffer(256)
    for name in hhg.EXPORTS:
        if name == "hhg_last_error":
            continue
        fn = getattr(lib, name)
        args = [0.0 if t is C.c_double else 0 if t in (C.c_int, C.c_size_t, C.c_int64) else None
                for t in fn.argtypes]
        rc = fn(*args)
        if name.endswith("_destroy"):
            assert rc == hhg.HHG_OK, name
            continue
        assert rc == hhg.HHG_ERR_ARG, (name, rc)
        assert lib.hhg_last_error(buf, 256) == hhg.HHG_ERR_ARG
        assert buf.value, name


def test_moved_corners_are_validated_before_device_use():
    # inverted or degenerate macros, and affine together with vertex_pos, are
    # argument errors found while building the host mesh (no GPU needed)
    import numpy as np
    import torch
    import hhg_inputs as I
    from paper_1506_06185_gb300 import hhg
    sub = (2, 1, 1)
    vp = I.jittered_vertices(sub, seed=4)
    bad = vp.copy()
    bad[0, 0, 1] = bad[1, 1, 1]            # a corner onto another: degenerate macros
    with pytest.raises(hhg.HHGError) as e:
        hhg.hhg_mesh_create(sub, 3, vertex_pos=bad)
    assert e.value.code == hhg.HHG_ERR_ARG and "macro" in str(e.value)
    flipped = vp.copy()
    flipped[..., 0] *= -1.0                # a mirror image: every macro inverted
    with pytest.raises(hhg.HHGError) as e:
        hhg.hhg_mesh_create(sub, 3, vertex_pos=flipped)
    assert e.value.code == hhg.HHG_ERR_ARG
    with pytest.raises(hhg.HHGError) as e:
        hhg.hhg_mesh_create(sub, 3, affine=np.eye(3), vertex_pos=vp)
    assert e.value.code == hhg.HHG_ERR_ARG
    with pytest.raises(ValueError):
        hhg.hhg_mesh_create(sub, 3, vertex_pos=vp[:, :, :2])
    if not torch.cuda.is_available():
        # accepted corners get past the host checks to the device step
        with pytest.raises(hhg.HHGError) as e:
            hhg.hhg_mesh_create(sub, 3, vertex_pos=vp)
        assert e.value.code == hhg.HHG_ERR_CUDA


def test_general_meshes_are_validated_before_device_use():
    import numpy as np
    import torch
    import hhg_inputs as I
    from paper_1506_06185_gb300 import hhg
    v, t = I.five_tet_macro_mesh((2, 1, 1))
    bad = t.copy()
    bad[0, 0] = len(v)                                    # id out of range
    with pytest.raises(hhg.HHGError) as e:
        hhg.hhg_mesh_create_general(v, bad, 3)
    assert e.value.code == hhg.HHG_ERR_ARG
    flat = v.copy()
    flat[:, 2] = 0.0                                      # every macro flattened
    with pytest.raises(hhg.HHGError) as e:
        hhg.hhg_mesh_create_general(flat, t, 3)
    assert e.value.code == hhg.HHG_ERR_ARG and "degenerate" in str(e.value)
    rep = t.copy()
    rep[0, 1] = rep[0, 0]                                 # a repeated vertex
    with pytest.raises(hhg.HHGError) as e:
        hhg.hhg_mesh_create_general(v, rep, 3)
    assert e.value.code == hhg.HHG_ERR_ARG
    tri = np.vstack([t, t[:1]])                           # one face shared by three macros
    with pytest.raises(hhg.HHGError) as e:
        hhg.hhg_mesh_create_general(v, tri, 3)
    assert e.value.code == hhg.HHG_ERR_ARG
    with pytest.raises(ValueError):
        hhg.hhg_mesh_create_general(v, t[:, :3], 3)
    if not torch.cuda.is_available():
        with pytest.raises(hhg.HHGError) as e:
            hhg.hhg_mesh_create_general(v, t, 3)
        assert e.value.code == hhg.HHG_ERR_CUDA
