"""The allocation-free entry point, checked against the regular projection path.

mg_mac_constraint_noalloc exists for callers that cannot allocate device memory
when they need the answer (for example code running inside a captured CUDA
graph, or under a device-memory budget that is already handed out).  It keeps
its reduction scratch in a fixed device array instead of calling cudaMalloc.
This test projects a velocity field with mg_project, then asks the new entry
point for the constraint of the projected field twice in a row: both calls
must agree with the constraint mg_project reported, to the 1e-9 relative
tolerance of the FP64 parity tests.  Grids that do not fill the kernel's blocks
evenly, a 2-D grid, and a grid with more partial sums than the final reduction
has threads are checked against the CPU oracle's own right-hand side.

The file is named to be collected last so that a run stopping at its first
failure has already run every other test when this one fails; nothing in it
depends on the other tests (each case passes in a fresh process too).
"""
import ctypes

import numpy as np
import pytest

import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1910_12979_gb300 import ProjectionSolver  # noqa: E402
from paper_1910_12979_gb300 import native as N  # noqa: E402


def _T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda:0")


@pytest.mark.parametrize("n,prec", [(32, "fp64"), (64, "mixed")])
def test_noalloc_constraint_matches_project(n, prec):
    p = I.stratified(n, seed=12, contrast=1e3, nodal=False)
    s = ProjectionSolver(p["geom"], _T(p["sigma"]), loc="cell", prec=prec)
    U = [_T(u) for u in p["U_mac"]]
    b0c, S = _T(p["beta0"]), _T(p["S"])
    b0f = [_T(b) for b in p["beta0_face"]]
    st = s.project(U, b0c, S, beta0_face=b0f, tol=1e-11)
    torch.cuda.synchronize()

    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda:0")
    beta0 = N.mg_beta0()
    beta0.cell = b0c.data_ptr()
    for d in range(3):
        beta0.face[d] = b0f[d].data_ptr()
    Uptr = (ctypes.c_void_p * 3)(*[u.data_ptr() for u in U])
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):   # two calls in a row share (and overwrite) the fixed scratch
        out.fill_(float("nan"))
        rc = N.load().mg_mac_constraint_noalloc(ctypes.byref(s.geo), Uptr, ctypes.byref(beta0),
                                                ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                                ctypes.c_void_p(stream))
        assert rc == N.MG_OK, N.mg_last_error()
        torch.cuda.synchronize()
        v = out.cpu().numpy()
        rel = np.sqrt(v[2] / v[1])
        assert rel == pytest.approx(st["rel_constraint"], rel=1e-9)
        assert np.sqrt(v[1]) == pytest.approx(st["src_norm"], rel=1e-9)


def test_noalloc_rejects_oversize_grid():
    g = N.mg_geometry(3, (512, 512, 256), (1 / 512, 1 / 512, 1 / 256), N.MG_LOC_CELL)
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    ptr = ctypes.c_void_p(dummy.data_ptr())
    beta0 = N.mg_beta0()
    beta0.cell = dummy.data_ptr()
    for d in range(3):
        beta0.face[d] = dummy.data_ptr()
    U = (ctypes.c_void_p * 3)(ptr, ptr, ptr)
    rc = N.load().mg_mac_constraint_noalloc(ctypes.byref(g), U, ctypes.byref(beta0), ptr, ptr, None)
    assert rc == N.MG_ERR_UNSUPPORTED
    assert "scratch" in N.mg_last_error()


@pytest.mark.parametrize("n", [(63, 47), (97, 96, 96)])
def test_noalloc_ragged_grids_match_oracle(oracle, n):
    """63 x 47 (2-D; 2961 cells, the last block partly filled) and 97 x 96 x 96
    (894,048 cells: 437 partial sums, more than the 256 threads of the final
    reduction, and a partial last block) against sums formed from the oracle's
    D(beta0 U) - beta0 S."""
    O = oracle
    dim = len(n)
    rng = np.random.default_rng(7)
    lo = ("neumann", "periodic", "neumann")[:dim]
    hi = ("dirichlet", "periodic", "dirichlet")[:dim]
    g = O.Grid.make(n, lo, hi)
    U = [rng.normal(scale=1e-2, size=g.face_shape(d)) for d in range(dim)]
    b0f = [np.exp(rng.normal(scale=0.3, size=g.face_shape(d))) for d in range(dim)]
    b0c = np.exp(rng.normal(scale=0.3, size=g.cell_shape))
    S = rng.random(g.cell_shape)
    v = O.mac_rhs(g, b0c, b0f, U, S)
    want = np.array([v.sum(), ((b0c * S) ** 2).sum(), (v ** 2).sum()])

    geo = N.mg_geometry(dim, tuple(n) + (1,) * (3 - dim), tuple(1.0 / m for m in n) + (1.0,) * (3 - dim),
                        N.MG_LOC_CELL)
    Ut = [_T(u) for u in U] + [None] * (3 - dim)
    bft = [_T(b) for b in b0f] + [None] * (3 - dim)
    b0ct, St = _T(b0c), _T(S)
    beta0 = N.mg_beta0()
    beta0.cell = b0ct.data_ptr()
    for d in range(dim):
        beta0.face[d] = bft[d].data_ptr()
    Uptr = (ctypes.c_void_p * 3)(*[(u.data_ptr() if u is not None else None) for u in Ut])
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.fill_(float("nan"))
        rc = N.load().mg_mac_constraint_noalloc(ctypes.byref(geo), Uptr, ctypes.byref(beta0),
                                                ctypes.c_void_p(St.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                                ctypes.c_void_p(stream))
        assert rc == N.MG_OK, N.mg_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - want[0]) <= 1e-9 * np.abs(v).sum()
        np.testing.assert_allclose(got[1:], want[1:], rtol=1e-9)
