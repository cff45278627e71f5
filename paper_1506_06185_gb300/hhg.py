"""ctypes binding of the HHG C ABI (include/hhg.h).

Argument marshalling only: every step of the multigrid path runs in the CUDA
library.  The module-level functions carry the C names (``hhg_mesh_create``,
``hhg_vcycle``, ...) and take the same arguments; :class:`Mesh` is a thin
object wrapper over them.  Vectors may be torch tensors (CUDA or CPU) or
numpy arrays of float64 in the global x-fastest node order.  If the shared
library is missing the import of this module fails loudly: there is no CPU
fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HHG_LIB may point at another build of the same library (e.g. a debug build)
LIB_PATH = os.environ.get("HHG_LIB") or os.path.join(_HERE, "_lib", "libhhg.so")

HHG_OK, HHG_ERR_ARG, HHG_ERR_CUDA, HHG_ERR_OOM, HHG_ERR_TIMEOUT, HHG_ERR_NOT_CONVERGED, HHG_ERR_STATE = range(7)
HHG_RECOVERY_NONE, HHG_RECOVERY_LR, HHG_RECOVERY_DD, HHG_RECOVERY_DN = 0, 1, 2, 3

EXPORTS = ["hhg_mesh_create", "hhg_mesh_destroy", "hhg_mesh_info", "hhg_mesh_bytes", "hhg_set_problem",
           "hhg_get_solution", "hhg_vcycle", "hhg_residual_norm", "hhg_inject_fault", "hhg_recover_local",
           "hhg_solve", "hhg_last_error", "hhg_profile_enable", "hhg_profile_read", "hhg_profile_info",
           "hhg_launch_count", "hhg_vcycle_noalloc", "hhg_set_coefficients", "hhg_grad_coeff",
           "hhg_autotune", "hhg_batch_create", "hhg_batch_launch", "hhg_batch_destroy",
           "hhg_batch_launch_persistent", "hhg_batch_info", "hhg_batch_set_priority", "hhg_recover_dn",
           "hhg_mesh_create_general", "hhg_set_launch_limit", "hhg_walk_counts", "hhg_set_streaming",
           "hhg_set_wait_limit", "hhg_measure_fp64_peak", "hhg_profile_breakdown", "hhg_set_flat_gs"]


class hhg_mesh_desc(C.Structure):
    _fields_ = [("subcubes", C.c_int * 3), ("levels", C.c_int), ("coarsest", C.c_int), ("precision", C.c_int),
                ("coeff", C.POINTER(C.c_double)), ("affine", C.POINTER(C.c_double)),
                ("vertex_pos", C.POINTER(C.c_double))]


class hhg_general_desc(C.Structure):
    _fields_ = [("n_vertices", C.c_int), ("vertices", C.POINTER(C.c_double)), ("n_macros", C.c_int),
                ("macros", C.POINTER(C.c_int)), ("levels", C.c_int), ("coarsest", C.c_int),
                ("precision", C.c_int), ("coeff", C.POINTER(C.c_double))]


class hhg_fault(C.Structure):
    _fields_ = [("cycle", C.c_int), ("macro_ids", C.POINTER(C.c_int)), ("n_ids", C.c_int)]


class hhg_solve_opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_cycles", C.c_int), ("pre", C.c_int), ("post", C.c_int),
                ("fault_cycle", C.c_int), ("fault_ids", C.POINTER(C.c_int)), ("n_fault_ids", C.c_int),
                ("recovery", C.c_int), ("n_local", C.c_int), ("n_global", C.c_int), ("eta", C.c_double),
                ("mixed_precision", C.c_int), ("coarse_rtol", C.c_double), ("coarse_maxit", C.c_int),
                ("faults", C.POINTER(hhg_fault)), ("n_faults", C.c_int)]


class HHGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"HHG error {code}: {msg}")
        self.code = code


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -m paper_1506_06185_gb300.build)")
    lib = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "hhg_mesh_create": ([C.POINTER(hhg_mesh_desc), C.POINTER(P)], C.c_int),
        "hhg_mesh_destroy": ([P], C.c_int),
        "hhg_mesh_create_general": ([C.POINTER(hhg_general_desc), C.POINTER(P)], C.c_int),
        "hhg_mesh_info": ([P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int)], C.c_int),
        "hhg_mesh_bytes": ([P, C.POINTER(C.c_int64)], C.c_int),
        "hhg_set_problem": ([P, P, P, P], C.c_int),
        "hhg_get_solution": ([P, P, P], C.c_int),
        "hhg_vcycle": ([P, C.c_int, C.c_int, C.POINTER(C.c_double), P], C.c_int),
        "hhg_residual_norm": ([P, C.POINTER(C.c_double), P], C.c_int),
        "hhg_inject_fault": ([P, C.POINTER(C.c_int), C.c_int, P], C.c_int),
        "hhg_recover_local": ([P, C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                               C.POINTER(C.c_double), P], C.c_int),
        "hhg_recover_dn": ([P, C.POINTER(C.c_int), C.c_int, C.c_int, C.c_double, C.POINTER(C.c_int),
                            C.POINTER(C.c_double), C.POINTER(C.c_double), P], C.c_int),
        "hhg_solve": ([P, C.POINTER(hhg_solve_opts), C.POINTER(C.c_double), C.POINTER(C.c_int),
                       C.POINTER(C.c_int), P], C.c_int),
        "hhg_last_error": ([C.c_char_p, C.c_size_t], C.c_int),
        "hhg_profile_enable": ([P, C.c_int], C.c_int),
        "hhg_profile_read": ([P, C.POINTER(C.c_int64), C.POINTER(C.c_double)], C.c_int),
        "hhg_profile_info": ([P, C.POINTER(C.c_int64), C.POINTER(C.c_int)], C.c_int),
        "hhg_launch_count": ([C.POINTER(C.c_int64)], C.c_int),
        "hhg_set_launch_limit": ([P, C.c_int], C.c_int),
        "hhg_walk_counts": ([P, C.POINTER(C.c_int64)], C.c_int),
        "hhg_set_streaming": ([P, C.c_int], C.c_int),
        "hhg_set_wait_limit": ([P, C.c_int], C.c_int),
        "hhg_set_flat_gs": ([P, C.c_int], C.c_int),
        "hhg_measure_fp64_peak": ([C.POINTER(C.c_double)], C.c_int),
        "hhg_profile_breakdown": ([P, C.POINTER(C.c_double), C.c_int], C.c_int),
        "hhg_vcycle_noalloc": ([P, C.c_int, C.c_int, P], C.c_int),
        "hhg_set_coefficients": ([P, C.POINTER(C.c_double), P], C.c_int),
        "hhg_grad_coeff": ([P, P, P, C.POINTER(C.c_double), P], C.c_int),
        "hhg_autotune": ([P, C.c_int, C.POINTER(C.c_int), P], C.c_int),
        "hhg_batch_create": ([P, C.c_int, C.POINTER(P), C.POINTER(C.POINTER(C.c_int)), C.POINTER(C.c_int),
                              C.POINTER(C.c_int), C.c_int, C.c_int, C.POINTER(P)], C.c_int),
        "hhg_batch_launch": ([P, C.POINTER(C.c_double), P], C.c_int),
        "hhg_batch_destroy": ([P], C.c_int),
        "hhg_batch_launch_persistent": ([P, C.POINTER(C.c_double), P], C.c_int),
        "hhg_batch_info": ([P, C.POINTER(C.c_int64)], C.c_int),
        "hhg_batch_set_priority": ([P, C.POINTER(C.c_int)], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _check(rc, allow=()):
    if rc != HHG_OK and rc not in allow:
        buf = C.create_string_buffer(1024)
        lib().hhg_last_error(buf, 1024)
        raise HHGError(rc, buf.value.decode(errors="replace"))
    return rc


def _ptr(x):
    """Raw address of a torch tensor or numpy array (must be contiguous float64)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if str(x.dtype) != "torch.float64":
            raise ValueError("tensor must be float64")
        return C.c_void_p(x.data_ptr())
    a = np.asarray(x)
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous float64")
    return C.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ids(ids):
    a = (C.c_int * len(ids))(*[int(i) for i in ids])
    return a, len(ids)


# --- C-named wrappers -------------------------------------------------------

def hhg_mesh_create(subcubes, levels, coarsest=2, precision=64, coeff=None, affine=None, vertex_pos=None):
    d = hhg_mesh_desc()
    d.subcubes[:] = [int(s) for s in subcubes]
    d.levels, d.coarsest, d.precision = int(levels), int(coarsest), int(precision)
    keep = []
    if coeff is not None:
        c = np.ascontiguousarray(coeff, dtype=np.float64)
        keep.append(c)
        d.coeff = c.ctypes.data_as(C.POINTER(C.c_double))
    if affine is not None:
        a = np.ascontiguousarray(np.asarray(affine, dtype=np.float64)[:3, :3])
        keep.append(a)
        d.affine = a.ctypes.data_as(C.POINTER(C.c_double))
    if vertex_pos is not None:
        sx, sy, sz = (int(s) for s in subcubes)
        v = np.ascontiguousarray(vertex_pos, dtype=np.float64)
        if v.shape != (sz + 1, sy + 1, sx + 1, 3):
            raise ValueError("vertex_pos must have shape (sz+1, sy+1, sx+1, 3)")
        keep.append(v)
        d.vertex_pos = v.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_void_p()
    _check(lib().hhg_mesh_create(C.byref(d), C.byref(h)))
    return h


def hhg_mesh_create_general(vertices, macros, levels, coarsest=2, precision=64, coeff=None):
    v = np.ascontiguousarray(vertices, dtype=np.float64)
    t = np.ascontiguousarray(macros, dtype=np.int32)
    if v.ndim != 2 or v.shape[1] != 3 or t.ndim != 2 or t.shape[1] != 4:
        raise ValueError("vertices must be (nv, 3) and macros (nt, 4)")
    d = hhg_general_desc()
    d.n_vertices, d.n_macros = v.shape[0], t.shape[0]
    d.vertices = v.ctypes.data_as(C.POINTER(C.c_double))
    d.macros = t.ctypes.data_as(C.POINTER(C.c_int))
    d.levels, d.coarsest, d.precision = int(levels), int(coarsest), int(precision)
    keep = [v, t]
    if coeff is not None:
        c = np.ascontiguousarray(coeff, dtype=np.float64)
        keep.append(c)
        d.coeff = c.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_void_p()
    _check(lib().hhg_mesh_create_general(C.byref(d), C.byref(h)))
    return h


def hhg_mesh_destroy(h):
    return _check(lib().hhg_mesh_destroy(h))


def hhg_mesh_info(h):
    a, b, c = C.c_int64(), C.c_int64(), C.c_int()
    _check(lib().hhg_mesh_info(h, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def hhg_mesh_bytes(h):
    a = C.c_int64()
    _check(lib().hhg_mesh_bytes(h, C.byref(a)))
    return a.value


def hhg_set_problem(h, f=None, u0=None, stream=None):
    return _check(lib().hhg_set_problem(h, _ptr(f), _ptr(u0), _stream(stream)))


def hhg_get_solution(h, u, stream=None):
    return _check(lib().hhg_get_solution(h, _ptr(u), _stream(stream)))


def hhg_vcycle(h, pre=3, post=3, want_residual=True, stream=None):
    r = C.c_double()
    _check(lib().hhg_vcycle(h, int(pre), int(post), C.byref(r) if want_residual else None, _stream(stream)))
    return r.value if want_residual else None


def hhg_vcycle_noalloc(h, pre=3, post=3, stream=None):
    """One global V-cycle whose coarse CG uses the library's static device
    scratch instead of allocated memory (see include/hhg.h)."""
    return _check(lib().hhg_vcycle_noalloc(h, int(pre), int(post), _stream(stream)))


def hhg_residual_norm(h, stream=None):
    r = C.c_double()
    _check(lib().hhg_residual_norm(h, C.byref(r), _stream(stream)))
    return r.value


def hhg_inject_fault(h, ids, stream=None):
    a, n = _ids(ids)
    return _check(lib().hhg_inject_fault(h, a, n, _stream(stream)))


def hhg_recover_local(h, ids, n_local, n_global=0, timed=False, stream=None):
    a, n = _ids(ids)
    tl, tg = C.c_double(), C.c_double()
    _check(lib().hhg_recover_local(h, a, n, int(n_local), int(n_global), C.byref(tl) if timed else None,
                                   C.byref(tg) if timed else None, _stream(stream)))
    return (tl.value, tg.value) if timed else None


def hhg_recover_dn(h, ids, n_global, eta, timed=False, stream=None):
    """Returns the Omega_F cycles run, and with ``timed`` also the device
    seconds of the two sides."""
    a, n = _ids(ids)
    nf = C.c_int()
    tl, tg = C.c_double(), C.c_double()
    _check(lib().hhg_recover_dn(h, a, n, int(n_global), float(eta), C.byref(nf), C.byref(tl) if timed else None,
                                C.byref(tg) if timed else None, _stream(stream)))
    return (nf.value, tl.value, tg.value) if timed else nf.value


def hhg_solve(h, rtol=1e-8, max_cycles=50, pre=3, post=3, fault_cycle=0, fault_ids=(), recovery=0, n_local=0,
              n_global=0, eta=1.0, mixed_precision=False, coarse_rtol=0.0, coarse_maxit=0, stream=None,
              allow_not_converged=False, faults=()):
    """``faults``: further (cycle, macro ids) faults, recovered like the first."""
    o = hhg_solve_opts()
    o.rtol, o.max_cycles, o.pre, o.post = float(rtol), int(max_cycles), int(pre), int(post)
    ids, n = _ids(fault_ids) if len(fault_ids) else (None, 0)
    o.fault_cycle = int(fault_cycle)
    o.fault_ids = ids
    o.n_fault_ids = n
    o.recovery, o.n_local, o.n_global, o.eta = int(recovery), int(n_local), int(n_global), float(eta)
    o.mixed_precision = 1 if mixed_precision else 0
    o.coarse_rtol, o.coarse_maxit = float(coarse_rtol), int(coarse_maxit)
    keep = []
    if len(faults):
        arr = (hhg_fault * len(faults))()
        for q, (cyc_q, ids_q) in enumerate(faults):
            a, n_q = _ids(ids_q)
            keep.append(a)
            arr[q].cycle, arr[q].macro_ids, arr[q].n_ids = int(cyc_q), a, n_q
        o.faults, o.n_faults = arr, len(faults)
    hist = (C.c_double * (int(max_cycles) + 2 + len(faults)))()
    nh, cyc = C.c_int(), C.c_int()
    rc = lib().hhg_solve(h, C.byref(o), hist, C.byref(nh), C.byref(cyc), _stream(stream))
    _check(rc, allow=(HHG_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return np.array(hist[:nh.value]), cyc.value, rc


def hhg_set_coefficients(h, coeff, stream=None):
    c = np.ascontiguousarray(np.asarray(coeff, dtype=np.float64))
    return _check(lib().hhg_set_coefficients(h, c.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)))


def hhg_grad_coeff(h, u, lam, n_macro, stream=None):
    g = np.zeros(int(n_macro))
    _check(lib().hhg_grad_coeff(h, _ptr(u), _ptr(lam), g.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)))
    return g


def hhg_autotune(h, n_levels, reps=3, stream=None):
    ch = (C.c_int * int(n_levels))()
    _check(lib().hhg_autotune(h, int(reps), ch, _stream(stream)))
    return list(ch)


class Batch:
    """Recovery tasks (and an optional global solve) captured into one CUDA
    graph; ``launch()`` runs them all with one graph launch."""

    def __init__(self, tasks, global_mesh=None, global_cycles=0, mixed=False):
        # tasks: list of (Mesh, fault ids, local cycles)
        self._keep = []
        n = len(tasks)
        meshes = (C.c_void_p * max(n, 1))(*[t[0].h for t in tasks])
        idarrs = [(C.c_int * len(t[1]))(*[int(i) for i in t[1]]) for t in tasks]
        self._keep += [meshes, idarrs]
        ids = (C.POINTER(C.c_int) * max(n, 1))(*[C.cast(a, C.POINTER(C.c_int)) for a in idarrs])
        nids = (C.c_int * max(n, 1))(*[len(t[1]) for t in tasks])
        cyc = (C.c_int * max(n, 1))(*[int(t[2]) for t in tasks])
        self._keep += [ids, nids, cyc]
        self.n = n + (1 if global_mesh is not None else 0)
        self.h = C.c_void_p()
        _check(lib().hhg_batch_create(global_mesh.h if global_mesh is not None else None, int(global_cycles),
                                      meshes, ids, nids, cyc, n, 1 if mixed else 0, C.byref(self.h)))

    def launch(self, timed=True, stream=None):
        ms = (C.c_double * max(self.n, 1))()
        _check(lib().hhg_batch_launch(self.h, ms if timed else None, _stream(stream)))
        return list(ms)[:self.n] if timed else None

    def launch_persistent(self, timed=True, stream=None):
        """The same work as one launch of the persistent scheduler kernel."""
        ms = (C.c_double * max(self.n, 1))()
        _check(lib().hhg_batch_launch_persistent(self.h, ms if timed else None, _stream(stream)))
        return list(ms)[:self.n] if timed else None

    def set_priority(self, prio=None):
        """Priority per task (the global task last) for the persistent
        launch; None: all equal."""
        if prio is None:
            _check(lib().hhg_batch_set_priority(self.h, None))
            return
        arr = (C.c_int * self.n)(*[int(x) for x in prio])
        _check(lib().hhg_batch_set_priority(self.h, arr))

    def info(self):
        """(tasks, recorded operations, work units, kernels in the graph)."""
        v = (C.c_int64 * 4)()
        _check(lib().hhg_batch_info(self.h, v))
        return tuple(int(x) for x in v)

    def close(self):
        if self.h is not None and self.h.value is not None:
            lib().hhg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hhg_profile_enable(h, enable=True):
    """enable: True/1 times the dominant kernel's launches, 2 records the
    phase breakdown, 3 both; False/0 stops."""
    return _check(lib().hhg_profile_enable(h, int(enable)))


BREAKDOWN_PHASES = ["fine_smoothing", "fine_residual", "restriction", "prolongation", "coarse_levels", "coarse_cg",
                    "stopping_test", "host_turnaround", "fault_recovery", "ir_correction"]


def hhg_profile_breakdown(h):
    """Per-phase device time (ms) of the global cycles since profiling bit 1
    was enabled, as a dict keyed by BREAKDOWN_PHASES."""
    ms = (C.c_double * len(BREAKDOWN_PHASES))()
    _check(lib().hhg_profile_breakdown(h, ms, len(BREAKDOWN_PHASES)))
    return dict(zip(BREAKDOWN_PHASES, list(ms)))


def hhg_profile_read(h):
    n, t = C.c_int64(), C.c_double()
    _check(lib().hhg_profile_read(h, C.byref(n), C.byref(t)))
    return n.value, t.value


def hhg_profile_info(h):
    n, s = C.c_int64(), C.c_int()
    _check(lib().hhg_profile_info(h, C.byref(n), C.byref(s)))
    return n.value, bool(s.value)


def hhg_set_launch_limit(h, max_ctas):
    return _check(lib().hhg_set_launch_limit(h, int(max_ctas)))


def hhg_set_streaming(h, enable=True):
    return _check(lib().hhg_set_streaming(h, 1 if enable else 0))


def hhg_set_flat_gs(h, enable=True):
    _check(lib().hhg_set_flat_gs(h, 1 if enable else 0))


def hhg_set_wait_limit(h, tries):
    """tries >= 0: at most that many tries per bounded device wait (0: every
    wait runs out at once); tries < 0: the default."""
    return _check(lib().hhg_set_wait_limit(h, int(tries)))


def hhg_walk_counts(h):
    """Dynamic-walk launches completed by the global, faulty, healthy
    (Gamma frozen) and DN Neumann problems."""
    c = (C.c_int64 * 4)()
    _check(lib().hhg_walk_counts(h, c))
    return list(c)


def hhg_measure_fp64_peak():
    """FP64 FMA throughput of the current device, TFLOP/s."""
    t = C.c_double()
    _check(lib().hhg_measure_fp64_peak(C.byref(t)))
    return t.value


def hhg_launch_count():
    n = C.c_int64()
    _check(lib().hhg_launch_count(C.byref(n)))
    return n.value


class Mesh:
    """Owning wrapper of an ``hhg_mesh`` handle."""

    def __init__(self, subcubes, levels, coarsest=2, precision=64, coeff=None, affine=None, vertex_pos=None):
        self.subcubes = tuple(int(s) for s in subcubes)
        self.levels = int(levels)
        self.h = hhg_mesh_create(subcubes, levels, coarsest, precision, coeff, affine, vertex_pos)
        self.n_nodes, self.n_dof, self.n_macro = hhg_mesh_info(self.h)
        N = 1 << self.levels
        self.shape = (self.subcubes[2] * N + 1, self.subcubes[1] * N + 1, self.subcubes[0] * N + 1)

    @classmethod
    def general(cls, vertices, macros, levels, coarsest=2, precision=64, coeff=None):
        """A macro mesh of general connectivity (vertex positions and the four
        vertex ids of every macro); vectors are flat, in the library's node
        order (see ``hhg_mesh_create_general`` in include/hhg.h)."""
        self = cls.__new__(cls)
        self.h = None
        self.subcubes = None
        self.levels = int(levels)
        self.h = hhg_mesh_create_general(vertices, macros, levels, coarsest, precision, coeff)
        self.n_nodes, self.n_dof, self.n_macro = hhg_mesh_info(self.h)
        self.shape = (self.n_nodes,)
        return self

    def close(self):
        if self.h is not None:
            hhg_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bytes(self):
        return hhg_mesh_bytes(self.h)

    def set_problem(self, f=None, u0=None, stream=None):
        hhg_set_problem(self.h, f, u0, stream)

    def get_solution(self, out=None, stream=None):
        if out is None:
            out = np.zeros(self.shape)
        hhg_get_solution(self.h, out, stream)
        return out

    def vcycle(self, pre=3, post=3, stream=None):
        return hhg_vcycle(self.h, pre, post, True, stream)

    def residual_norm(self, stream=None):
        return hhg_residual_norm(self.h, stream)

    def inject_fault(self, ids, stream=None):
        hhg_inject_fault(self.h, ids, stream)

    def recover_local(self, ids, n_local, n_global=0, timed=False, stream=None):
        return hhg_recover_local(self.h, ids, n_local, n_global, timed, stream)

    def recover_dn(self, ids, n_global, eta, timed=False, stream=None):
        return hhg_recover_dn(self.h, ids, n_global, eta, timed, stream)

    def solve(self, **kw):
        return hhg_solve(self.h, **kw)

    def set_coefficients(self, coeff, stream=None):
        hhg_set_coefficients(self.h, coeff, stream)

    def grad_coeff(self, u, lam, stream=None):
        return hhg_grad_coeff(self.h, u, lam, self.n_macro, stream)
