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
