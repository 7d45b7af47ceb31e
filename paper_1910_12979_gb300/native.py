"""ctypes binding of libmgproj.so (include/mg.h): argument marshalling only.

Every function here has the name and the argument order of the C entry point
it wraps.  No arithmetic of the solve happens in Python: the library's CUDA
kernels do all of it.  Loading fails loudly when the library cannot be built
or found; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

MG_OK, MG_ERR_INVALID_ARG, MG_ERR_OOM, MG_ERR_CUDA, MG_ERR_NOT_CONVERGED, MG_ERR_DIVERGED, \
    MG_ERR_INCOMPATIBLE_RHS, MG_ERR_TIMEOUT, MG_ERR_BUSY, MG_ERR_UNSUPPORTED = range(10)
MG_BC_PERIODIC, MG_BC_NEUMANN, MG_BC_DIRICHLET = 0, 1, 2
MG_LOC_CELL, MG_LOC_NODAL = 0, 1
MG_PREC_FP64, MG_PREC_MIXED = 0, 1
MG_FLAG_NO_FUSED = 1
MG_FLAG_NO_GRAPH = 2
MG_FLAG_SWEEP_PIPE = 4
MG_FLAG_AUTOTUNE = 8
MG_FLAG_ZERO_GUESS = 16
MG_FLAG_SWEEP_TMA = 32
MG_FLAG_CELL_PIPE = 64
MG_FLAG_BATCH_BRANCHES = 128

BC = {"periodic": MG_BC_PERIODIC, "neumann": MG_BC_NEUMANN, "dirichlet": MG_BC_DIRICHLET}

_dp = ctypes.POINTER(ctypes.c_double)


class mg_geometry(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double * 3), ("loc", ctypes.c_int)]


class mg_bc(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int * 3), ("hi", ctypes.c_int * 3)]


class mg_coeff(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_void_p), ("face", ctypes.c_void_p * 3)]


class mg_beta0(ctypes.Structure):
    _fields_ = [("cell", ctypes.c_void_p), ("face", ctypes.c_void_p * 3)]


class mg_options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("coarsest_max", ctypes.c_int), ("interp_order", ctypes.c_int), ("omega", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("flags", ctypes.c_int), ("inner_cycles", ctypes.c_int)]


class mg_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_resid", ctypes.c_double), ("rel_constraint", ctypes.c_double),
                ("rhs_norm", ctypes.c_double), ("src_norm", ctypes.c_double), ("ms", ctypes.c_double),
                ("status", ctypes.c_int), ("vcycles", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# (name, restype, argtypes) of every entry point declared in include/mg.h
SIGNATURES = [
    ("mg_default_options", None, [ctypes.POINTER(mg_options)]),
    ("mg_hierarchy_bytes", ctypes.c_int, [ctypes.POINTER(mg_geometry), ctypes.POINTER(mg_bc),
                                          ctypes.POINTER(mg_options), ctypes.POINTER(ctypes.c_size_t)]),
    ("mg_setup", ctypes.c_int, [ctypes.POINTER(mg_coeff), ctypes.POINTER(mg_geometry), ctypes.POINTER(mg_bc),
                                ctypes.POINTER(mg_options), ctypes.c_void_p, ctypes.c_size_t,
                                ctypes.POINTER(ctypes.c_void_p)]),
    ("mg_update_coeff", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(mg_coeff)]),
    ("mg_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                ctypes.POINTER(mg_stats)]),
    ("mg_project", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p * 3, ctypes.POINTER(mg_beta0), ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(mg_stats)]),
    ("mg_base_state_beta0", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    ("mg_base_state_map", ctypes.c_int, [ctypes.POINTER(mg_geometry), ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p * 3,
                                         ctypes.c_void_p]),
    ("mg_rhs", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p * 3, ctypes.POINTER(mg_beta0), ctypes.c_void_p,
                              ctypes.c_void_p]),
    ("mg_solve_batch", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                      ctypes.POINTER(mg_stats)]),
    ("mg_project_batch", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(mg_beta0), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                        ctypes.POINTER(mg_stats)]),
    ("mg_set_stream", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("mg_apply", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("mg_destroy", None, [ctypes.c_void_p]),
    ("mg_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("mg_last_error", ctypes.c_char_p, []),
    ("mg_mac_constraint_noalloc", ctypes.c_int, [ctypes.POINTER(mg_geometry), ctypes.c_void_p * 3,
                                                 ctypes.POINTER(mg_beta0), ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p]),
    ("mg_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p * 3, ctypes.c_void_p * 3,
                               ctypes.c_void_p * 3, ctypes.POINTER(mg_beta0), ctypes.c_void_p, ctypes.c_double,
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                               ctypes.c_double, ctypes.POINTER(mg_stats)]),
    ("mg_rotation_forces", ctypes.c_int, [ctypes.POINTER(mg_geometry), ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double,
                                          ctypes.c_void_p * 3, ctypes.c_void_p * 3, ctypes.c_void_p]),
    ("mg_convert_f64_to_f32", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("mg_convert_f32_to_f64", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("mg_convert_f64_to_f32_pow2", ctypes.c_int,
     [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]),
    ("mg_reciprocal_f64", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("mg_fp64_fma_probe", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_double)]),
    ("mg_smoother_kind", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("mg_prof_enable", None, [ctypes.c_int]),
    ("mg_launch_count", ctypes.c_longlong, []),
    ("mg_set_batch_groups", ctypes.c_int, [ctypes.c_int]),
    ("mg_prof_query", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
]

MG_PROF_CELL_SMOOTH_FINE, MG_PROF_RESID64, MG_PROF_NODE_SMOOTH_FINE, MG_PROF_CELL_RESTRICT_FINE, \
    MG_PROF_NODE_RESID64, MG_PROF_CELL_PIPE_DOWN, MG_PROF_CELL_PIPE_UP, MG_PROF_BATCH_SMOOTH, \
    MG_PROF_BATCH_RESTRICT, MG_PROF_BATCH_PROLONG, MG_PROF_BATCH_COARSE, MG_PROF_BATCH_RESID64, \
    MG_PROF_BATCH_SMOOTH_COARSE = range(13)
PROF_NAMES = {MG_PROF_CELL_SMOOTH_FINE: "cell_smooth_fine", MG_PROF_RESID64: "cell_resid64",
              MG_PROF_NODE_SMOOTH_FINE: "node_smooth_fine", MG_PROF_CELL_RESTRICT_FINE: "cell_restrict_fine",
              MG_PROF_NODE_RESID64: "node_resid64", MG_PROF_CELL_PIPE_DOWN: "cell_pipe_down",
              MG_PROF_CELL_PIPE_UP: "cell_pipe_up", MG_PROF_BATCH_SMOOTH: "batch_smooth",
              MG_PROF_BATCH_RESTRICT: "batch_restrict", MG_PROF_BATCH_PROLONG: "batch_prolong",
              MG_PROF_BATCH_COARSE: "batch_coarse", MG_PROF_BATCH_RESID64: "batch_resid64",
              MG_PROF_BATCH_SMOOTH_COARSE: "batch_smooth_coarse"}
# kernel classes bound by the FP64 pipe rather than by HBM
PROF_FP64_BOUND = {"cell_resid64", "node_resid64", "batch_resid64"}

_lib = None
_lib_gil = None   # the same library through ctypes.PyDLL: calls keep the GIL


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libmgproj.so (building it first when stale and nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_needed:
        try:
            path = _build.build()
        except Exception as e:  # no nvcc, or a compile error: fail loudly unless a built library exists
            if not os.path.exists(path):
                raise ImportError(f"libmgproj.so is not built and cannot be built: {e}") from e
    if not os.path.exists(path):
        raise ImportError(f"libmgproj.so not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    global _lib_gil
    _lib_gil = ctypes.PyDLL(path)
    _lib_gil.mg_destroy.restype = None
    _lib_gil.mg_destroy.argtypes = [ctypes.c_void_p]
    _lib = lib
    return lib


class MGError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        self.status = status
        msg = lib.mg_strerror(status).decode()
        detail = lib.mg_last_error().decode()
        super().__init__(f"{where}: {msg} ({detail})")


def check(status, where, allow=(MG_OK,)):
    if status not in allow:
        raise MGError(status, where)
    return status


# thin wrappers with the C names ------------------------------------------------

def mg_default_options():
    o = mg_options()
    load().mg_default_options(ctypes.byref(o))
    return o


def mg_hierarchy_bytes(geom, bc, opt):
    n = ctypes.c_size_t(0)
    check(load().mg_hierarchy_bytes(ctypes.byref(geom), ctypes.byref(bc), ctypes.byref(opt), ctypes.byref(n)),
          "mg_hierarchy_bytes")
    return n.value


def mg_setup(coeff, geom, bc, opt, workspace_ptr, workspace_bytes):
    h = ctypes.c_void_p()
    check(load().mg_setup(ctypes.byref(coeff), ctypes.byref(geom), ctypes.byref(bc), ctypes.byref(opt),
                          ctypes.c_void_p(workspace_ptr), ctypes.c_size_t(workspace_bytes), ctypes.byref(h)),
          "mg_setup")
    return h


def mg_update_coeff(h, coeff):
    return check(load().mg_update_coeff(h, ctypes.byref(coeff)), "mg_update_coeff")


def mg_solve(h, rhs_ptr, phi_ptr, tol, allow=(MG_OK,)):
    st = mg_stats()
    rc = load().mg_solve(h, ctypes.c_void_p(rhs_ptr), ctypes.c_void_p(phi_ptr), ctypes.c_double(tol),
                         ctypes.byref(st))
    check(rc, "mg_solve", allow)
    return st


def mg_project(h, U_ptrs, beta0, S_ptr, phi_ptr, tol, allow=(MG_OK,)):
    st = mg_stats()
    arr = (ctypes.c_void_p * 3)(*[ctypes.c_void_p(p) if p else None for p in U_ptrs])
    rc = load().mg_project(h, arr, ctypes.byref(beta0), ctypes.c_void_p(S_ptr),
                           ctypes.c_void_p(phi_ptr) if phi_ptr else None, ctypes.c_double(tol), ctypes.byref(st))
    check(rc, "mg_project", allow)
    return st


def mg_rhs(h, U_ptrs, beta0, S_ptr, f_ptr):
    arr = (ctypes.c_void_p * 3)(*[ctypes.c_void_p(p) if p else None for p in U_ptrs])
    return check(load().mg_rhs(h, arr, ctypes.byref(beta0), ctypes.c_void_p(S_ptr), ctypes.c_void_p(f_ptr)),
                 "mg_rhs")


def mg_solve_batch(handles, rhs_ptrs, phi_ptrs, tols, allow=(MG_OK,)):
    n = len(handles)
    H = (ctypes.c_void_p * n)(*[h.value for h in handles])
    R = (ctypes.c_void_p * n)(*rhs_ptrs)
    P = (ctypes.c_void_p * n)(*phi_ptrs)
    T = (ctypes.c_double * n)(*tols)
    st = (mg_stats * n)()
    rc = load().mg_solve_batch(H, R, P, T, n, st)
    check(rc, "mg_solve_batch", allow)
    return list(st)


def mg_project_batch(handles, U_ptrs, beta0s, S_ptrs, phi_ptrs, tols, allow=(MG_OK,)):
    """U_ptrs: per entry a list of 3 device pointers (None for absent components)."""
    n = len(handles)
    P = ctypes.c_void_p
    hs = (P * n)(*[h.value for h in handles])
    U = (P * (3 * n))(*[u for e in U_ptrs for u in (list(e) + [None] * (3 - len(e)))])
    b0 = (mg_beta0 * n)(*beta0s)
    S = (P * n)(*S_ptrs)
    ph = (P * n)(*phi_ptrs) if phi_ptrs is not None else None
    tl = (ctypes.c_double * n)(*tols)
    st = (mg_stats * n)()
    check(load().mg_project_batch(hs, U, b0, S, ph, tl, n, st), "mg_project_batch", allow)
    return list(st)


def mg_set_stream(h, stream_ptr):
    return check(load().mg_set_stream(h, ctypes.c_void_p(stream_ptr)), "mg_set_stream")


def mg_apply(h, phi_ptr, out_ptr):
    return check(load().mg_apply(h, ctypes.c_void_p(phi_ptr), ctypes.c_void_p(out_ptr)), "mg_apply")


def mg_destroy(h, keep_gil=False):
    """keep_gil: call without releasing the GIL.  Finalizers that run inside a
    garbage collection must not release it: another thread could then start a
    second collection over the same object lists."""
    lib = load()
    (_lib_gil if keep_gil else lib).mg_destroy(h)


def mg_strerror(s):
    return load().mg_strerror(s).decode()


def mg_last_error():
    return load().mg_last_error().decode()


def mg_step(mac, nodal, U_ptrs, Unew_ptrs, Uadv_ptrs, beta0, S_ptr, dt, omega=None, center=None, centrifugal=False,
            tol=1e-10, allow=(MG_OK,)):
    arr = lambda p: (ctypes.c_void_p * 3)(*(list(p) + [None] * (3 - len(p))))
    om = (ctypes.c_double * 3)(*omega) if omega is not None else None
    c = (ctypes.c_double * 3)(*center) if center is not None else None
    st = (mg_stats * 2)()
    check(load().mg_step(mac, nodal, arr(U_ptrs), arr(Unew_ptrs), arr(Uadv_ptrs), ctypes.byref(beta0),
                         ctypes.c_void_p(S_ptr), float(dt), om, c, 1 if centrifugal else 0, float(tol), st),
          "mg_step", allow)
    return st[0], st[1]


def mg_rotation_forces(geom, omega, center, centrifugal, alpha, U_ptrs, F_ptrs, stream=None):
    om = (ctypes.c_double * 3)(*omega)
    c = (ctypes.c_double * 3)(*center) if center is not None else None
    u = (ctypes.c_void_p * 3)(*(list(U_ptrs) + [None] * (3 - len(U_ptrs))))
    f = (ctypes.c_void_p * 3)(*(list(F_ptrs) + [None] * (3 - len(F_ptrs))))
    return check(load().mg_rotation_forces(ctypes.byref(geom), om, c, 1 if centrifugal else 0, float(alpha), u, f,
                                           stream), "mg_rotation_forces")


def mg_convert_f64_to_f32(x_ptr, y_ptr, n, stream=None):
    check(load().mg_convert_f64_to_f32(x_ptr, y_ptr, n, stream), "mg_convert_f64_to_f32")


def mg_convert_f32_to_f64(x_ptr, y_ptr, n, stream=None):
    check(load().mg_convert_f32_to_f64(x_ptr, y_ptr, n, stream), "mg_convert_f32_to_f64")


def mg_convert_f64_to_f32_pow2(x_ptr, y_ptr, n, shift, stream=None):
    check(load().mg_convert_f64_to_f32_pow2(x_ptr, y_ptr, n, shift, stream), "mg_convert_f64_to_f32_pow2")


def mg_reciprocal_f64(x_ptr, y_ptr, n, stream=None):
    check(load().mg_reciprocal_f64(x_ptr, y_ptr, n, stream), "mg_reciprocal_f64")


def mg_fp64_fma_probe(blocks, iters, sink_ptr, stream=None):
    """Launch the FP64 FMA probe; returns its flop count (time it with CUDA events)."""
    fl = ctypes.c_double()
    check(load().mg_fp64_fma_probe(blocks, iters, sink_ptr, stream, ctypes.byref(fl)), "mg_fp64_fma_probe")
    return fl.value


def mg_smoother_kind(h, level):
    return int(load().mg_smoother_kind(h, level))


def mg_launch_count():
    return int(load().mg_launch_count())


def mg_prof_enable(on):
    load().mg_prof_enable(1 if on else 0)


def mg_set_batch_groups(groups):
    """Concurrent batched loops a batch is split into (0: automatic)."""
    return check(load().mg_set_batch_groups(int(groups)), "mg_set_batch_groups")


def mg_prof_query(kernel):
    ms, n, by, fl = ctypes.c_double(), ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    check(load().mg_prof_query(kernel, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(by), ctypes.byref(fl)),
          "mg_prof_query")
    return {"ms": ms.value, "launches": n.value, "bytes": by.value, "flops": fl.value}


def mg_base_state_beta0(p0_ptr, gamma1_ptr, gamma1_const, rho0_base, nr, beta0_ptr, stream_ptr=None):
    return check(load().mg_base_state_beta0(ctypes.c_void_p(p0_ptr), ctypes.c_void_p(gamma1_ptr) if gamma1_ptr else None,
                                            ctypes.c_double(gamma1_const), ctypes.c_double(rho0_base), nr,
                                            ctypes.c_void_p(beta0_ptr), ctypes.c_void_p(stream_ptr)),
                 "mg_base_state_beta0")


def mg_base_state_map(geom, spherical, center, r0, dr, nr, beta0_r_ptr, rho0_r_ptr, sigma_ptr, beta0_cell_ptr,
                      beta0_face_ptrs, stream_ptr=None):
    c = (ctypes.c_double * 3)(*center)
    f = (ctypes.c_void_p * 3)(*[ctypes.c_void_p(p) if p else None for p in beta0_face_ptrs])
    return check(load().mg_base_state_map(ctypes.byref(geom), int(spherical), c, ctypes.c_double(r0),
                                          ctypes.c_double(dr), nr, ctypes.c_void_p(beta0_r_ptr),
                                          ctypes.c_void_p(rho0_r_ptr), ctypes.c_void_p(sigma_ptr),
                                          ctypes.c_void_p(beta0_cell_ptr), f, ctypes.c_void_p(stream_ptr)),
                 "mg_base_state_map")
