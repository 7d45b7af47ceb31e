"""FP64 CPU oracle for the projection solve of Eq. 6 (S2) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It wraps
``mg_oracle.c`` (plain C, compiled with gcc) through ctypes and shares no code
with the CUDA library.  ``all_cores(threads)`` switches the calls inside it to
``mg_oracle_omp.c``, the same source built with colour-ordered smoothers and
OpenMP loops: the benchmark's all-core CPU baseline, never used for parity.

Arrays are numpy float64, C order, always 3-D shaped (nz, ny, nx) with nz = 1
for 2-D problems:

* cells ``(nz, ny, nx)``; x faces ``(nz, ny, nx+1)``; y faces ``(nz, ny+1, nx)``;
  z faces ``(nz+1, ny, nx)`` (absent in 2-D);
* nodes ``(Nz, Ny, Nx)`` with ``N_d = n_d`` on periodic axes and ``n_d + 1``
  otherwise (``Nz = 1`` in 2-D).

Boundary kinds: ``"periodic"``, ``"neumann"`` (wall), ``"dirichlet"`` (phi = 0).

Parity status of each routine (what pins it, in ``tests/test_oracle_*.py``):
every public routine here is pinned by closed forms, invariants or brute force;
none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")

BC_CODES = {"periodic": 0, "neumann": 1, "dirichlet": 2}


_SRC_OMP = os.path.join(_HERE, "mg_oracle_omp.c")
_LIB_OMP = os.path.join(_HERE, "_build", "liborc_omp.so")


def build(force: bool = False) -> str:
    """Compile mg_oracle.c into oracle/_build/liborc.so (plain gcc, no -march)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build_omp(force: bool = False) -> str:
    """Compile the all-core CPU baseline (mg_oracle_omp.c: this oracle with
    colour-ordered smoothers and OpenMP loops) into oracle/_build/liborc_omp.so.
    Timing only: the parity tests never use it."""
    os.makedirs(os.path.dirname(_LIB_OMP), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_OMP))
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < newest:
        tmp = _LIB_OMP + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC_OMP,
                               "-lm"])
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double * 3),
                ("bclo", ctypes.c_int * 3), ("bchi", ctypes.c_int * 3)]


class _Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("relres", ctypes.c_double), ("constraint", ctypes.c_double),
                ("rhs_norm", ctypes.c_double), ("src_norm", ctypes.c_double)]


_lib = None
_lib_omp = None
_use_omp = False


def _L():
    global _lib, _lib_omp
    if _use_omp:
        if _lib_omp is None:
            _lib_omp = _declare(ctypes.CDLL(build_omp()))
        return _lib_omp
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


class all_cores:
    """Context: the oracle calls inside run on the all-core CPU-baseline build
    (colour-ordered smoothers, OpenMP loops) with ``threads`` threads.  Timing
    only; not for parity (another smoother, so other iteration counts)."""

    def __init__(self, threads):
        self.threads = int(threads)

    def __enter__(self):
        global _use_omp
        _use_omp = True
        _L().orc_omp_set_threads(self.threads)
        return self

    def __exit__(self, *exc):
        global _use_omp
        _use_omp = False
        return False


def _declare(lib):
    for name in ("orc_mac_faces", "orc_mac_apply", "orc_mac_div", "orc_mac_rhs", "orc_mac_grad_update",
                 "orc_mac_solve_dense", "orc_mac_solve_mg", "orc_mac_project", "orc_nodal_apply",
                 "orc_nodal_div", "orc_nodal_lump", "orc_nodal_grad", "orc_nodal_rhs",
                 "orc_nodal_solve_dense", "orc_nodal_solve_mg", "orc_nodal_project", "orc_beta0_eq5",
                 "orc_map_radial", "orc_rotation_forces", "orc_face_average", "orc_advect"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


@dataclass(frozen=True)
class Grid:
    """Uniform grid: ``n`` cells per axis, spacing ``h``, boundary kinds per face."""
    dim: int
    n: tuple
    h: tuple
    bclo: tuple
    bchi: tuple

    @staticmethod
    def make(n, bclo, bchi, h=None):
        dim = len(n)
        n3 = tuple(n) + (1,) * (3 - dim)
        h3 = tuple(h) if h is not None else tuple(1.0 / v for v in n)
        h3 = h3 + (1.0,) * (3 - len(h3))
        lo = tuple(bclo) + ("neumann",) * (3 - dim)
        hi = tuple(bchi) + ("neumann",) * (3 - dim)
        for d in range(dim):
            if (lo[d] == "periodic") != (hi[d] == "periodic"):
                raise ValueError("periodic boundaries must be paired")
        return Grid(dim, n3, h3, lo, hi)

    def c(self):
        g = _Grid()
        g.dim = self.dim
        for d in range(3):
            g.n[d] = self.n[d]
            g.h[d] = self.h[d]
            g.bclo[d] = BC_CODES[self.bclo[d]]
            g.bchi[d] = BC_CODES[self.bchi[d]]
        return g

    @property
    def cell_shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def face_shape(self, d):
        m = [self.n[0], self.n[1], self.n[2]]
        m[d] += 1
        return (m[2], m[1], m[0])

    def node_extent(self, d):
        if d >= self.dim:
            return 1
        return self.n[d] if self.bclo[d] == "periodic" else self.n[d] + 1

    @property
    def node_shape(self):
        return (self.node_extent(2), self.node_extent(1), self.node_extent(0))

    @property
    def singular(self):
        return not any("dirichlet" in (self.bclo[d], self.bchi[d]) for d in range(self.dim))

    def dirichlet_node_mask(self):
        """Boolean mask over the node array: True on Dirichlet (non-unknown) nodes."""
        m = np.zeros(self.node_shape, dtype=bool)
        for d in range(self.dim):
            ax = 2 - d
            if self.bclo[d] == "dirichlet":
                idx = [slice(None)] * 3
                idx[ax] = 0
                m[tuple(idx)] = True
            if self.bchi[d] == "dirichlet":
                idx = [slice(None)] * 3
                idx[ax] = self.n[d]
                m[tuple(idx)] = True
        return m


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr3(arrs):
    return [(_p(a) if a is not None else None) for a in (list(arrs) + [None] * (3 - len(arrs)))]


def _arr3(ptrs):
    return (ctypes.POINTER(ctypes.c_double) * 3)(*[p if p is not None else ctypes.POINTER(ctypes.c_double)()
                                                  for p in ptrs])


# ---------------------------------------------------------------- MAC system

def mac_faces(g: Grid, sigma):
    """Face coefficients B (harmonic mean of adjacent sigma), one array per axis."""
    sigma = _f64(sigma)
    B = [np.zeros(g.face_shape(d)) for d in range(g.dim)]
    p = _ptr3(B)
    _L().orc_mac_faces(ctypes.byref(g.c()), _p(sigma), p[0], p[1], p[2])
    return B


def mac_apply(g: Grid, B, phi):
    """(L phi) on cells."""
    B = [_f64(b) for b in B]
    phi = _f64(phi)
    out = np.zeros(g.cell_shape)
    p = _ptr3(B)
    _L().orc_mac_apply(ctypes.byref(g.c()), p[0], p[1], p[2], _p(phi), _p(out))
    return out


def mac_div(g: Grid, V):
    """D(V) on cells for face arrays V."""
    V = [_f64(v) for v in V]
    out = np.zeros(g.cell_shape)
    p = _ptr3(V)
    _L().orc_mac_div(ctypes.byref(g.c()), p[0], p[1], p[2], _p(out))
    return out


def mac_rhs(g: Grid, beta0_cell, beta0_face, U, S):
    """f = D(beta0 U) - beta0 S (no mean removal)."""
    bc, S = _f64(beta0_cell), _f64(S)
    bf = [_f64(b) for b in beta0_face]
    U = [_f64(u) for u in U]
    out = np.zeros(g.cell_shape)
    _L().orc_mac_rhs(ctypes.byref(g.c()), _p(bc), _arr3(_ptr3(bf)), _arr3(_ptr3(U)), _p(S), _p(out))
    return out


def mac_grad_update(g: Grid, B, beta0_face, phi, U):
    """Returns U - (B / beta0_face) G phi (copies)."""
    B = [_f64(b) for b in B]
    bf = [_f64(b) for b in beta0_face]
    U = [np.array(u, dtype=np.float64, copy=True) for u in U]
    phi = _f64(phi)
    _L().orc_mac_grad_update(ctypes.byref(g.c()), _arr3(_ptr3(B)), _arr3(_ptr3(bf)), _p(phi), _arr3(_ptr3(U)))
    return U


def mac_solve_dense(g: Grid, B, f):
    """Exact solution of L phi = f by LU (zero-mean gauge when singular)."""
    B = [_f64(b) for b in B]
    f = _f64(f)
    phi = np.zeros(g.cell_shape)
    p = _ptr3(B)
    rc = _L().orc_mac_solve_dense(ctypes.byref(g.c()), p[0], p[1], p[2], _p(f), _p(phi))
    if rc != 0:
        raise RuntimeError("oracle dense MAC solve failed (singular matrix)")
    return phi


def mac_solve_mg(g: Grid, B, f, tol=1e-14, max_cycles=200, phi0=None, require=1e-9):
    """Multigrid solve to tol or the round-off floor; returns (phi, stats dict).

    Raises when the relative residual stays above ``require`` (e.g. a strongly
    anisotropic grid, where point Gauss-Seidel does not smooth), so that no test
    ever compares against an unconverged oracle."""
    B = [_f64(b) for b in B]
    f = _f64(f)
    phi = np.zeros(g.cell_shape) if phi0 is None else np.array(phi0, dtype=np.float64, copy=True)
    st = _Stats()
    p = _ptr3(B)
    rc = _L().orc_mac_solve_mg(ctypes.byref(g.c()), p[0], p[1], p[2], _p(f), _p(phi), ctypes.c_double(tol),
                               ctypes.c_int(max_cycles), ctypes.byref(st))
    if rc != 0:
        raise RuntimeError("oracle MAC multigrid setup failed")
    if st.relres > max(tol, require):
        raise RuntimeError(f"oracle MAC multigrid did not converge (relres {st.relres:.3e}); use mac_solve_dense")
    return phi, {"iters": st.iters, "relres": st.relres}


def mac_project(g: Grid, sigma, beta0_cell, beta0_face, U, S, tol=1e-14, dense=False):
    """Full MAC projection.  Returns dict(phi, U, iters, relres, constraint, src_norm, rhs_norm)."""
    sigma, bc, S = _f64(sigma), _f64(beta0_cell), _f64(S)
    bf = [_f64(b) for b in beta0_face]
    U = [np.array(u, dtype=np.float64, copy=True) for u in U]
    phi = np.zeros(g.cell_shape)
    st = _Stats()
    rc = _L().orc_mac_project(ctypes.byref(g.c()), _p(sigma), _p(bc), _arr3(_ptr3(bf)), _arr3(_ptr3(U)), _p(S),
                              _p(phi), ctypes.c_double(tol), ctypes.c_int(1 if dense else 0), ctypes.byref(st))
    if rc != 0:
        raise RuntimeError("oracle MAC projection failed")
    if st.relres > max(tol, 1e-9):
        raise RuntimeError(f"oracle MAC projection did not converge (relres {st.relres:.3e})")
    return {"phi": phi, "U": U, "iters": st.iters, "relres": st.relres, "constraint": st.constraint,
            "src_norm": st.src_norm, "rhs_norm": st.rhs_norm}


# -------------------------------------------------------------- nodal system

def nodal_apply(g: Grid, sigma, phi):
    sigma, phi = _f64(sigma), _f64(phi)
    out = np.zeros(g.node_shape)
    _L().orc_nodal_apply(ctypes.byref(g.c()), _p(sigma), _p(phi), _p(out))
    return out


def nodal_div(g: Grid, V):
    """D_N(V) on nodes for cell-centred components V."""
    V = [_f64(v) for v in V]
    out = np.zeros(g.node_shape)
    _L().orc_nodal_div(ctypes.byref(g.c()), _arr3(_ptr3(V)), _p(out))
    return out


def nodal_lump(g: Grid, gc):
    gc = _f64(gc)
    out = np.zeros(g.node_shape)
    _L().orc_nodal_lump(ctypes.byref(g.c()), _p(gc), _p(out))
    return out


def nodal_grad(g: Grid, phi):
    """G_N(phi) on cells, one array per axis."""
    phi = _f64(phi)
    G = [np.zeros(g.cell_shape) for _ in range(g.dim)]
    _L().orc_nodal_grad(ctypes.byref(g.c()), _p(phi), _arr3(_ptr3(G)))
    return G


def nodal_rhs(g: Grid, beta0, U, S):
    beta0, S = _f64(beta0), _f64(S)
    U = [_f64(u) for u in U]
    out = np.zeros(g.node_shape)
    _L().orc_nodal_rhs(ctypes.byref(g.c()), _p(beta0), _arr3(_ptr3(U)), _p(S), _p(out))
    return out


def nodal_solve_dense(g: Grid, sigma, f):
    sigma, f = _f64(sigma), _f64(f)
    phi = np.zeros(g.node_shape)
    rc = _L().orc_nodal_solve_dense(ctypes.byref(g.c()), _p(sigma), _p(f), _p(phi))
    if rc != 0:
        raise RuntimeError("oracle dense nodal solve failed (singular matrix)")
    return phi


def nodal_solve_mg(g: Grid, sigma, f, tol=1e-14, max_cycles=200, phi0=None, require=1e-9):
    sigma, f = _f64(sigma), _f64(f)
    phi = np.zeros(g.node_shape) if phi0 is None else np.array(phi0, dtype=np.float64, copy=True)
    st = _Stats()
    rc = _L().orc_nodal_solve_mg(ctypes.byref(g.c()), _p(sigma), _p(f), _p(phi), ctypes.c_double(tol),
                                 ctypes.c_int(max_cycles), ctypes.byref(st))
    if rc != 0:
        raise RuntimeError("oracle nodal multigrid setup failed")
    if st.relres > max(tol, require):
        raise RuntimeError(f"oracle nodal multigrid did not converge (relres {st.relres:.3e})")
    return phi, {"iters": st.iters, "relres": st.relres}


def nodal_project(g: Grid, sigma, beta0, U, S, tol=1e-14, dense=False):
    """Full nodal projection.  Returns dict(phi, U, iters, relres, constraint, src_norm, rhs_norm)."""
    sigma, beta0, S = _f64(sigma), _f64(beta0), _f64(S)
    U = [np.array(u, dtype=np.float64, copy=True) for u in U]
    phi = np.zeros(g.node_shape)
    st = _Stats()
    rc = _L().orc_nodal_project(ctypes.byref(g.c()), _p(sigma), _p(beta0), _arr3(_ptr3(U)), _p(S), _p(phi),
                                ctypes.c_double(tol), ctypes.c_int(1 if dense else 0), ctypes.byref(st))
    if rc != 0:
        raise RuntimeError("oracle nodal projection failed")
    if st.relres > max(tol, 1e-9):
        raise RuntimeError(f"oracle nodal projection did not converge (relres {st.relres:.3e})")
    return {"phi": phi, "U": U, "iters": st.iters, "relres": st.relres, "constraint": st.constraint,
            "src_norm": st.src_norm, "rhs_norm": st.rhs_norm}


# ------------------------------------------------------------- base state

def beta0_eq5(p0, rho00, gamma1=None, g1=5.0 / 3.0):
    """beta0 of Eq. 5 on a radial grid from tabulated p0 (and optional Gamma1 per point)."""
    p0 = _f64(p0)
    out = np.zeros_like(p0)
    ga = _f64(gamma1) if gamma1 is not None else None
    _L().orc_beta0_eq5(_p(p0), _p(ga) if ga is not None else None, ctypes.c_double(g1), ctypes.c_double(rho00),
                       ctypes.c_int(len(p0)), _p(out))
    return out


def map_radial(g: Grid, spherical, center, r0, dr, beta0_r, rho0_r):
    """(sigma, beta0_cell, beta0_face list) from uniform radial tables."""
    b, rho = _f64(beta0_r), _f64(rho0_r)
    sigma, bc = np.zeros(g.cell_shape), np.zeros(g.cell_shape)
    bf = [np.zeros(g.face_shape(d)) for d in range(g.dim)]
    c = (ctypes.c_double * 3)(*(list(center) + [0.0] * (3 - len(center))))
    _L().orc_map_radial(ctypes.byref(g.c()), ctypes.c_int(1 if spherical else 0), c, ctypes.c_double(r0),
                        ctypes.c_double(dr), ctypes.c_int(len(b)), _p(b), _p(rho), _p(sigma), _p(bc),
                        _arr3(_ptr3(bf)))
    return sigma, bc, bf


def rotation_forces(g: Grid, omega, center, U, F=None, alpha=1.0, centrifugal=True):
    """F += alpha (-2 omega x U - omega x (omega x r)) at cell centres (S5); returns F."""
    U = [_f64(u) for u in U]
    if F is None:
        F = [np.zeros(g.cell_shape) for _ in range(g.dim)]
    else:
        F = [np.array(f, dtype=np.float64, order="C", copy=True) for f in F]
    om = (ctypes.c_double * 3)(*(list(omega) + [0.0] * (3 - len(omega))))
    c = (ctypes.c_double * 3)(*(list(center) + [0.0] * (3 - len(center))))
    _L().orc_rotation_forces(ctypes.byref(g.c()), om, c, ctypes.c_int(1 if centrifugal else 0),
                             ctypes.c_double(alpha), _arr3(_ptr3(U)), _arr3(_ptr3(F)))
    return F


def face_average(g: Grid, U):
    """MAC face velocities from cell-centred U (mean of the two cells; walls 0; outflow: interior value)."""
    U = [_f64(u) for u in U]
    Uf = [np.zeros(g.face_shape(d)) for d in range(g.dim)]
    _L().orc_face_average(ctypes.byref(g.c()), _arr3(_ptr3(U)), _arr3(_ptr3(Uf)))
    return Uf


def advect(g: Grid, Uf, q):
    """Upwind advective derivative (U_adv . grad) q at cell centres."""
    Uf = [_f64(u) for u in Uf]
    q = _f64(q)
    A = np.zeros(g.cell_shape)
    _L().orc_advect(ctypes.byref(g.c()), _arr3(_ptr3(Uf)), _p(q), _p(A))
    return A


def time_step(g: Grid, sigma, beta0_cell, beta0_face, U, S, dt, omega=None, center=None, centrifugal=True,
              tol=1e-14):
    """One step around the two projections (S2-S3), in the order of the method:
    face velocities from U^n, MAC projection of them, advection of U^n by the
    projected face velocities (plus the rotation accelerations when omega is
    given), nodal projection of the result.  Returns the new cell velocities, the
    projected face velocities and the two projections' results."""
    Uf = face_average(g, U)
    mac = mac_project(g, sigma, beta0_cell, beta0_face, Uf, S, tol=tol)
    Uadv = mac["U"]
    Ustar = [np.asarray(U[d], dtype=np.float64) - dt * advect(g, Uadv, U[d]) for d in range(g.dim)]
    if omega is not None:
        Ustar = rotation_forces(g, omega, center, U, F=Ustar, alpha=dt, centrifugal=centrifugal)
    nod = nodal_project(g, sigma, beta0_cell, Ustar, S, tol=tol)
    return {"U": nod["U"], "Uadv": Uadv, "mac": mac, "nodal": nod}
