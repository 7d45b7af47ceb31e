"""Torch-facing wrapper of the C ABI: one resident multigrid hierarchy per object.

PyTorch provides the device memory (the hierarchy workspace comes from the
caching allocator) and the stream; every step of the solve runs in the
library's CUDA kernels.  Tensors are float64, contiguous, on a CUDA device,
in the layouts documented in include/mg.h (shaped (nz, ny, nx) here, nz = 1 in
2-D).
"""
from __future__ import annotations

import torch

from . import native as N


def _ptr(t, name, shape=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


class ProjectionSolver:
    """Resident hierarchy for one grid.

    geom: dict(dim, n, h, bclo, bchi) as produced by ``inputs.geometry``;
    loc: "cell" (MAC projection) or "nodal"; prec: "mixed" or "fp64".
    """

    def __init__(self, geom, sigma, loc="cell", prec="mixed", faces=None, nu1=2, nu2=2, max_iters=100,
                 coarsest_max=8, interp_order=1, omega=0.9, stream=None, flags=0, inner_cycles=0):
        N.load()
        self.dim = int(geom["dim"])
        n = list(geom["n"]) + [1] * (3 - len(geom["n"]))
        h = list(geom["h"]) + [1.0] * (3 - len(geom["h"]))
        self.n = tuple(n)
        self.loc = loc
        self.geo = N.mg_geometry(self.dim, (n[0], n[1], n[2]), (h[0], h[1], h[2]),
                                 N.MG_LOC_CELL if loc == "cell" else N.MG_LOC_NODAL)
        lo = [N.BC[b] for b in geom["bclo"]] + [N.MG_BC_NEUMANN] * (3 - self.dim)
        hi = [N.BC[b] for b in geom["bchi"]] + [N.MG_BC_NEUMANN] * (3 - self.dim)
        self.bc = N.mg_bc((lo[0], lo[1], lo[2]), (hi[0], hi[1], hi[2]))
        self.periodic = [geom["bclo"][d] == "periodic" for d in range(self.dim)]
        opt = N.mg_default_options()
        opt.prec = N.MG_PREC_MIXED if prec == "mixed" else N.MG_PREC_FP64
        opt.nu1, opt.nu2, opt.max_iters = nu1, nu2, max_iters
        opt.coarsest_max, opt.interp_order, opt.omega = coarsest_max, interp_order, omega
        opt.flags = flags
        opt.inner_cycles = inner_cycles
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        opt.stream = self.stream.cuda_stream
        self.opt = opt
        self.device = sigma.device
        nbytes = N.mg_hierarchy_bytes(self.geo, self.bc, opt)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.handle = None
        coeff = self._coeff(sigma, faces)
        self.handle = N.mg_setup(coeff, self.geo, self.bc, opt, aligned, nbytes + 256 - (aligned - base))

    # shapes ------------------------------------------------------------------
    @property
    def cell_shape(self):
        return (self.n[2], self.n[1], self.n[0])

    def face_shape(self, d):
        m = list(self.n)
        m[d] += 1
        return (m[2], m[1], m[0])

    @property
    def node_shape(self):
        ext = [(self.n[d] if self.periodic[d] else self.n[d] + 1) if d < self.dim else 1 for d in range(3)]
        return (ext[2], ext[1], ext[0])

    @property
    def vec_shape(self):
        return self.cell_shape if self.loc == "cell" else self.node_shape

    def _coeff(self, sigma, faces):
        c = N.mg_coeff()
        c.sigma = _ptr(sigma, "sigma", self.cell_shape)
        self._keep = [sigma]
        if faces is not None:
            for d in range(self.dim):
                c.face[d] = _ptr(faces[d], f"faces[{d}]", self.face_shape(d))
            self._keep += list(faces)
        return c

    # API ---------------------------------------------------------------------
    def update_coeff(self, sigma, faces=None):
        N.mg_update_coeff(self.handle, self._coeff(sigma, faces))

    def solve(self, rhs, phi, tol=1e-10, allow_not_converged=False):
        allow = (N.MG_OK, N.MG_ERR_NOT_CONVERGED) if allow_not_converged else (N.MG_OK,)
        st = N.mg_solve(self.handle, _ptr(rhs, "rhs", self.vec_shape), _ptr(phi, "phi", self.vec_shape), tol, allow)
        return st.as_dict()

    def project(self, U, beta0_cell, S, beta0_face=None, phi=None, tol=1e-10, allow_not_converged=False):
        if self.loc == "cell":
            ptrs = [_ptr(U[d], f"U[{d}]", self.face_shape(d)) for d in range(self.dim)]
        else:
            ptrs = [_ptr(U[d], f"U[{d}]", self.cell_shape) for d in range(self.dim)]
        ptrs += [None] * (3 - self.dim)
        b0 = N.mg_beta0()
        b0.cell = _ptr(beta0_cell, "beta0_cell", self.cell_shape)
        if self.loc == "cell":
            if beta0_face is None:
                raise ValueError("the MAC projection needs beta0 at faces")
            for d in range(self.dim):
                b0.face[d] = _ptr(beta0_face[d], f"beta0_face[{d}]", self.face_shape(d))
        allow = (N.MG_OK, N.MG_ERR_NOT_CONVERGED) if allow_not_converged else (N.MG_OK,)
        st = N.mg_project(self.handle, ptrs, b0, _ptr(S, "S", self.cell_shape),
                          _ptr(phi, "phi", self.vec_shape) if phi is not None else None, tol, allow)
        return st.as_dict()

    def _beta0(self, beta0_cell, beta0_face):
        b0 = N.mg_beta0()
        b0.cell = _ptr(beta0_cell, "beta0_cell", self.cell_shape)
        if self.loc == "cell":
            if beta0_face is None:
                raise ValueError("the MAC projection needs beta0 at faces")
            for d in range(self.dim):
                b0.face[d] = _ptr(beta0_face[d], f"beta0_face[{d}]", self.face_shape(d))
        return b0

    def rhs(self, U, beta0_cell, S, beta0_face=None, out=None):
        """f = D(beta0 U) - beta0 S (MAC) or D_N(beta0 U) - S_N (nodal), mean-free if singular."""
        if out is None:
            out = torch.empty(self.vec_shape, dtype=torch.float64, device=self.device)
        shp = (lambda d: self.face_shape(d)) if self.loc == "cell" else (lambda d: self.cell_shape)
        ptrs = [_ptr(U[d], f"U[{d}]", shp(d)) for d in range(self.dim)] + [None] * (3 - self.dim)
        N.mg_rhs(self.handle, ptrs, self._beta0(beta0_cell, beta0_face), _ptr(S, "S", self.cell_shape),
                 _ptr(out, "f", self.vec_shape))
        return out

    def apply(self, phi, out=None):
        if out is None:
            out = torch.empty(self.vec_shape, dtype=torch.float64, device=self.device)
        N.mg_apply(self.handle, _ptr(phi, "phi", self.vec_shape), _ptr(out, "out", self.vec_shape))
        return out

    def close(self, _keep_gil=False):
        if self.handle is not None:
            N.mg_destroy(self.handle, keep_gil=_keep_gil)
            self.handle = None
        self.workspace = None

    def __del__(self):
        try:
            self.close(_keep_gil=True)   # may run inside a garbage collection on any thread
        except Exception:
            pass


def solve_batch(solvers, rhs, phi, tols, allow_not_converged=False):
    """mg_solve_batch over several ProjectionSolver objects."""
    allow = (N.MG_OK, N.MG_ERR_NOT_CONVERGED) if allow_not_converged else (N.MG_OK,)
    st = N.mg_solve_batch([s.handle for s in solvers], [_ptr(r, "rhs") for r in rhs], [_ptr(p, "phi") for p in phi],
                          list(tols), allow)
    return [s.as_dict() for s in st]


def project_batch(solvers, U, beta0_cell, S, beta0_face=None, phi=None, tols=None, allow_not_converged=False):
    """mg_project_batch: one projection per solver (U[i]: its velocity components,
    updated in place; beta0_cell[i], S[i]; beta0_face[i] for MAC solvers; phi[i]
    or None), the solves as one graph launch.  Returns the statistics."""
    n = len(solvers)
    faces = beta0_face if beta0_face is not None else [None] * n
    phis = phi if phi is not None else [None] * n
    tols = tols if tols is not None else [1e-10] * n
    Up, b0s, Sp, pp = [], [], [], []
    for s, u, bc, sv, bf, ph in zip(solvers, U, beta0_cell, S, faces, phis):
        shp = (lambda d: s.face_shape(d)) if s.loc == "cell" else (lambda d: s.cell_shape)
        Up.append([_ptr(u[d], f"U[{d}]", shp(d)) for d in range(s.dim)])
        b0s.append(s._beta0(bc, bf))
        Sp.append(_ptr(sv, "S", s.cell_shape))
        pp.append(_ptr(ph, "phi", s.vec_shape) if ph is not None else None)
    allow = (N.MG_OK, N.MG_ERR_NOT_CONVERGED) if allow_not_converged else (N.MG_OK,)
    st = N.mg_project_batch([s.handle for s in solvers], Up, b0s, Sp, pp, tols, allow)
    return [x.as_dict() for x in st]


def time_step(mac, nodal, U, Unew, Uadv, beta0_cell, beta0_face, S, dt, omega=None, center=None, centrifugal=False,
              tol=1e-10, allow_not_converged=False):
    """mg_step: face velocities, MAC projection, advection (+ rotation), nodal
    projection.  mac / nodal: ProjectionSolver objects of the same grid;
    U: cell components of U^n; Unew: output cell components; Uadv: face arrays
    (scratch; the projected face velocities on return).  Returns the two
    projections' statistics."""
    b0 = N.mg_beta0()
    b0.cell = _ptr(beta0_cell, "beta0_cell", mac.cell_shape)
    for d in range(mac.dim):
        b0.face[d] = _ptr(beta0_face[d], f"beta0_face[{d}]", mac.face_shape(d))
    allow = (N.MG_OK, N.MG_ERR_NOT_CONVERGED) if allow_not_converged else (N.MG_OK,)
    a, b = N.mg_step(mac.handle, nodal.handle, [_ptr(u, "U", mac.cell_shape) for u in U],
                     [_ptr(u, "Unew", mac.cell_shape) for u in Unew],
                     [_ptr(u, "Uadv", mac.face_shape(d)) for d, u in enumerate(Uadv)], b0,
                     _ptr(S, "S", mac.cell_shape), dt, omega, center, centrifugal, tol, allow)
    return a.as_dict(), b.as_dict()
