"""Index arithmetic of the CUDA path on the CPU (tests/host/layout_check.cpp):
the blocked colour-split layout gives every lattice node its own slot inside
its colour's array, rows start on 16-byte boundaries and the neighbour-row
offsets the vector kernels use hold; the slot-prefix closed form equals its
definition; the row-pair tiles of the volume kernels (default and autotuner
candidates) cover every interior row of every slice exactly once, within the
kernels' per-tile table sizes, largest first.  Refinements 2..130, 256, 512.
The streaming Gauss-Seidel units (refinements 64..512, FP64 and FP32 bands):
staged ranges fit the shared-memory slots, every neighbour read of every
updated node lands on the right lattice node inside its staged range, and
every interior node of every colour is updated exactly once.  The flat
Gauss-Seidel item tables (FP64 and FP32 vectors) cover every interior node of
every colour exactly once, each item holding at least one node, and the flat
restriction's slot items cover every interior node exactly once.  The walk order
of the large stencil launches (interface chunks spread among the volume
units) visits every chunk and unit exactly once, each kind in its own order,
with at most n_vol / n_if volume units between two chunks."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def check_prog(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    cuda_inc = "/usr/local/cuda/include"
    if not cxx or not os.path.isdir(cuda_inc):
        pytest.skip("needs a C++ compiler and the CUDA headers")
    out = tmp_path_factory.mktemp("layoutcheck") / "layout_check"
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-I" + cuda_inc, "-o", str(out),
                           os.path.join(ROOT, "tests", "host", "layout_check.cpp"),
                           os.path.join(ROOT, "paper_1506_06185_gb300", "csrc", "mesh.cpp")])
    return str(out)


def test_layout_and_tiles(check_prog):
    r = subprocess.run([check_prog, "130"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok")
