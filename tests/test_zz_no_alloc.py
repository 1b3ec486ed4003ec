"""pic_pcg_solve_static: the Poisson solve for callers that cannot allocate
device memory (an application running inside a device arena it manages
itself, or under an allocator budgeted elsewhere, cannot create a context).
The caller supplies the matrix, the right-hand side and the solution buffer;
the solver's work vectors live in the library's fixed static device array.

Checked through the C ABI against the context's own Poisson solve on the same
system, on two calls in a row (charge-free, then with space charge and a warm
start), within the tolerance the other parity tests use, and against a direct
sparse solve (scipy) of the same matrix.  Also: the iteration cap, a call after
a failed one, and inputs the kernel refuses (a non-finite right-hand side, a
column index outside the matrix).  Collected last so that a run stopping at
the first failure has run every other test."""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_1906_08125_gb300 import configs as K
from paper_1906_08125_gb300 import inputs

pytestmark = pytest.mark.gpu


def _system(mesh, E0):
    """P1 stiffness and Neumann load on the free nodes, assembled with numpy."""
    P = mesh.xyz[mesh.tet]
    J = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
    Ji = np.linalg.inv(J)
    g = np.concatenate([-Ji.sum(axis=1, keepdims=True), Ji], axis=1)
    vol = np.linalg.det(J) / 6
    Ke = vol[:, None, None] * np.einsum("tik,tjk->tij", g, g)
    N = mesh.n_nodes
    rows = np.repeat(mesh.tet, 4, axis=1).ravel()
    cols = np.tile(mesh.tet, (1, 4)).ravel()
    M = sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(N, N)).tocsr()
    free = np.nonzero(mesh.dirichlet == 0)[0]
    M = M[free][:, free].tocsr()
    M.sort_indices()
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    tt, kk = np.nonzero(mesh.nbr == -1)
    fn = mesh.tet[tt[:, None], loc[kk]]
    A = 0.5 * np.linalg.norm(np.cross(mesh.xyz[fn[:, 1]] - mesh.xyz[fn[:, 0]],
                                      mesh.xyz[fn[:, 2]] - mesh.xyz[fn[:, 0]]), axis=1)
    fN = np.bincount(fn.ravel(), weights=np.repeat(E0 * A / 3, 3), minlength=N)[free]
    return M, fN, free


def test_static_scratch_solve_matches_poisson_solve(tip_small):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_08125_gb300 import picfem
    L = picfem.load()
    dev = torch.device("cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    mesh = tip_small
    E0, w_sp, S = 1e10, 0.5, 32
    p = K.params(E0=E0, w_sp=w_sp, pcg_rtol=1e-12, capacity=20000, precision=K.PREC_FP64)
    ctx = picfem.Context(p).mesh_load(mesh)
    M, fN, free = _system(mesh, E0)
    n = len(free)
    rowptr = torch.from_numpy(M.indptr.astype(np.int32)).to(dev)
    col = torch.from_numpy(M.indices.astype(np.int32)).to(dev)
    val = torch.from_numpy(M.data.astype(np.float64)).to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)

    def call(b, max_iter=20000, colv=None):
        bt = torch.from_numpy(np.ascontiguousarray(b)).to(dev)
        it, rr = C.c_int32(0), C.c_double(0.0)
        cv = col if colv is None else colv
        rc = L.pic_pcg_solve_static(n, rowptr.data_ptr(), cv.data_ptr(), val.data_ptr(),
                                    bt.data_ptr(), x.data_ptr(), 1e-12, max_iter, C.byref(it),
                                    C.byref(rr), stream)
        return rc, it.value, rr.value

    def solve(b):
        rc, it, rr = call(b)
        assert rc == 0, L.pic_last_error(None)
        assert rr <= 1e-12 and it > 0
        return x.cpu().numpy().copy()

    def rel(a, b):
        return np.abs(a - b).max() / np.abs(b).max()

    # call 1: charge-free, against pic_init_potential and a direct solve
    ctx.init_potential()
    x1 = solve(fN)
    assert rel(x1, ctx.potential()[free]) <= 1e-9
    assert rel(x1, spla.spsolve(M.tocsc(), fN)) <= 1e-9

    # call 2: the space charge of seeded SPs, warm-started from call 1,
    # against deposit + poisson_solve
    r, v, cell, pid = inputs.random_particles(mesh, 4000, seed=21)
    ctx.set_particles(r, v, cell, pid)
    ctx.deposit()
    ctx.poisson_solve()
    W = ctx.charge()
    coef = (K.Q_ELECTRON * w_sp) / K.EPS0
    b2 = coef * (W[free].astype(np.float64) * 2.0 ** -S) + fN
    x2 = solve(b2)
    assert rel(x2, ctx.potential()[free]) <= 1e-9
    assert rel(x2, spla.spsolve(M.tocsc(), b2)) <= 1e-9
    assert rel(x2, x1) > 1e-6   # the space charge changed the answer

    # the iteration cap: PIC_ERR_NOT_CONVERGED after exactly max_iter
    # iterations; the next call on the same array starts from cleared
    # control words and converges to the same solution
    x.zero_()
    rc, it, rr = call(b2, max_iter=2)
    assert rc == -6 and it == 2 and rr > 1e-12
    x3 = solve(b2)
    assert rel(x3, x2) <= 1e-9

    # inputs the kernel refuses before using them: a NaN in b, and a column
    # index outside [0, n) (checked before anything is read through it)
    bad = b2.copy()
    bad[n // 2] = np.nan
    x_before = x.clone()
    rc, it, rr = call(bad)
    assert rc == -1 and it == 0
    assert torch.equal(x, x_before)
    bad_col = col.clone()
    bad_col[len(bad_col) // 3] = n
    rc, it, rr = call(b2, colv=bad_col)
    assert rc == -1 and b"column" in L.pic_last_error(None)
    # and after the refusals a call solves as before
    x4 = solve(b2)
    assert rel(x4, x2) <= 1e-9

    # sizes beyond the static scratch are refused before anything is launched
    rc = L.pic_pcg_solve_static(262145, rowptr.data_ptr(), col.data_ptr(), val.data_ptr(),
                                val.data_ptr(), x.data_ptr(), 1e-12, 10, None, None, stream)
    assert rc == -1
    assert b"262144" in L.pic_last_error(None)
    ctx.close()
