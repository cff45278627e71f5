"""Parity checks shared by the GPU tests.

An FP64 iterate of the CUDA path matches the oracle's when both
  * the relative Euclidean error ||u - u_ref|| / ||u_ref|| and
  * the largest error of any single node, max |u - u_ref| / max |u_ref|
are at most the tolerance (1e-12 for the FP64 path).  The second bound is the
per-element one: a global norm alone would let one wrong node out of 10^5 be
off by several hundred times the tolerance.
"""

import numpy as np

RTOL_U = 1e-12


def errors(u, ref):
    """(relative l2 error, relative max-norm error) of u against ref."""
    u = np.asarray(u, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = u - ref
    l2 = np.linalg.norm(d) / max(np.linalg.norm(ref), 1e-300)
    mx = np.abs(d).max() / max(np.abs(ref).max(), 1e-300) if d.size else 0.0
    return float(l2), float(mx)


def assert_close(u, ref, rtol=RTOL_U, what=""):
    """Both the global and the per-element error of u against ref within rtol."""
    l2, mx = errors(u, ref)
    assert l2 <= rtol and mx <= rtol, f"{what}: relative l2 error {l2:.3e}, max-norm error {mx:.3e} (bound {rtol:.1e})"
    return l2, mx
