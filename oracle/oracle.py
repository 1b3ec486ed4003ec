"""ctypes front end of the plain FP64 CPU oracle (picfem_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke entry and
by the CPU-baseline leg of the benchmark, never by the CUDA library or its
Python binding.  ``build()`` compiles the C file with gcc (no fused
multiply-add) into ``oracle/_build/liboracle.so`` and, with OpenMP, into
``liboracle_omp.so``: the same source with its independent loops run on all
host cores, bit-identical to the serial build (``Oracle(..., parallel=True)``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "picfem_oracle.c")
LIB = os.path.join(HERE, "_build", "liboracle.so")
LIB_OMP = os.path.join(HERE, "_build", "liboracle_omp.so")

OK, ERR_ARG, ERR_MESH, ERR_CAPACITY, ERR_WALK_LIMIT, ERR_NOT_CONVERGED = 0, -1, -3, -4, -5, -6
FN_MURPHY_GOOD, FN_ELEMENTARY = 0, 1
FATE_ALIVE, FATE_COLLECTED, FATE_ABSORBED = 0, 1, 2


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("E0", C.c_double), ("w_sp", C.c_double),
                ("q", C.c_double), ("q_over_m", C.c_double), ("eps0", C.c_double),
                ("e_charge", C.c_double), ("pcg_rtol", C.c_double),
                ("pcg_max_iter", C.c_int32), ("fn_model", C.c_int32),
                ("seed", C.c_uint64), ("capacity", C.c_int64),
                ("walk_max_steps", C.c_int32), ("quant_bits", C.c_int32),
                ("collisions", C.c_int32), ("pad", C.c_int32), ("coulomb_log", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("injected", C.c_int64), ("collected", C.c_int64), ("absorbed", C.c_int64),
                ("wrapped", C.c_int64), ("crossings", C.c_int64), ("alive", C.c_int64),
                ("max_walk", C.c_int32), ("pcg_iters", C.c_int32), ("pcg_relres", C.c_double),
                ("collected_charge", C.c_double)]


def build(force: bool = False, parallel: bool = False) -> str:
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    out = LIB_OMP if parallel else LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "picfem_oracle.h"))):
        tmp = out + f".{os.getpid()}.tmp"
        omp = ["-fopenmp"] if parallel else []
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-std=c11", *omp, "-o", tmp, SRC, "-lm"])
        os.replace(tmp, out)
    return out


_libs = {False: None, True: None}


def lib(parallel: bool = False):
    if _libs[parallel] is None:
        _libs[parallel] = C.CDLL(build(parallel=parallel))
        L = _libs[parallel]
        P = C.c_void_p
        L.or_create.restype = P
        L.or_create.argtypes = [C.POINTER(Params)]
        L.or_destroy.argtypes = [P]
        L.or_mesh_load.argtypes = [P, C.c_int32, P, C.c_int32, P, P, P, P, C.c_int32, P, P, P]
        L.or_n_free.restype = C.c_int32
        L.or_n_free.argtypes = [P]
        L.or_nnz.restype = C.c_int64
        L.or_nnz.argtypes = [P]
        L.or_geometry.argtypes = [P, P, P, P]
        L.or_matrix.argtypes = [P, P, P, P, P, P]
        L.or_element_stiffness.argtypes = [P, P]
        L.or_fn_current.restype = C.c_double
        L.or_fn_current.argtypes = [C.c_double, C.c_double, C.c_int]
        L.or_uniform.restype = C.c_double
        L.or_uniform.argtypes = [C.c_uint64] * 5
        L.or_splitmix64_next.restype = C.c_uint64
        L.or_splitmix64_next.argtypes = [C.POINTER(C.c_uint64)]
        L.or_init_potential.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
        L.or_get_potential.argtypes = [P, P]
        L.or_set_potential.argtypes = [P, P]
        L.or_get_field.argtypes = [P, P]
        L.or_set_dirichlet.argtypes = [P, P]
        L.or_num_particles.restype = C.c_int64
        L.or_num_particles.argtypes = [P]
        L.or_get_particles.argtypes = [P, P, P, P, P]
        L.or_set_particles.argtypes = [P, C.c_int64, P, P, P, P]
        L.or_get_charge.argtypes = [P, P]
        L.or_step_index.restype = C.c_int64
        L.or_step_index.argtypes = [P]
        L.or_set_step_index.argtypes = [P, C.c_int64]
        L.or_set_work_function.argtypes = [P, P]
        L.or_inject.argtypes = [P, C.c_int64, C.POINTER(C.c_int64)]
        L.or_push_relocate.argtypes = [P, C.c_int64, C.POINTER(Stats)]
        L.or_deposit.argtypes = [P]
        L.or_poisson_solve.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
        L.or_solve.argtypes = [P, P, P, C.c_double, C.c_int32, C.POINTER(C.c_int32),
                               C.POINTER(C.c_double)]
        L.or_step.argtypes = [P, C.c_int64, C.POINTER(Stats)]
        L.or_collide.argtypes = [P, C.c_int64]
        L.or_locate.argtypes = [P, C.c_int64, P, P, P, P]
        L.or_barycentric.argtypes = [P, C.c_int32, P, P]
        L.or_quad_emission.argtypes = [P, P, P, P]
        L.or_quad_emission_field.argtypes = [P, P, P, P, P]
        L.or_set_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
    return _libs[parallel]


def set_threads(n: int) -> int:
    """Threads of the OpenMP build (n <= 0 leaves them); returns the count."""
    return lib(True).or_set_threads(int(n))


def _p(a):
    return a.ctypes.data if a is not None else None


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != OK:
        raise OracleError(f"{what} failed with status {st}")


def fn_current(F, phi, model=FN_MURPHY_GOOD) -> float:
    return lib().or_fn_current(float(F), float(phi), int(model))


def uniform(seed, step, quad, j, slot) -> float:
    return lib().or_uniform(seed, step, quad, j, slot)


def splitmix64_sequence(seed: int, n: int):
    s = C.c_uint64(seed)
    return [lib().or_splitmix64_next(C.byref(s)) for _ in range(n)]


def element_stiffness(x4x3) -> np.ndarray:
    x = np.ascontiguousarray(x4x3, np.float64).reshape(4, 3)
    k = np.zeros((4, 4))
    lib().or_element_stiffness(_p(x), _p(k))
    return k


class Oracle:
    """One oracle PIC context over one mesh (parallel: the OpenMP build)."""

    def __init__(self, mesh, params: dict, parallel: bool = False):
        self.mesh = mesh
        self.params = dict(params)
        self.L = lib(parallel)
        p = Params(**{k: params.get(k, 0) for k, _ in Params._fields_})
        self._keep = p
        self.h = self.L.or_create(C.byref(p))
        arrs = mesh.arrays()
        self._arrs = arrs
        xyz, tet, nbr, pnbr, dirichlet, fnodes, ftet, wf = arrs
        st = self.L.or_mesh_load(self.h, mesh.n_nodes, _p(xyz), mesh.n_tets, _p(tet), _p(nbr),
                                _p(pnbr), _p(dirichlet), mesh.n_faces, _p(fnodes), _p(ftet),
                                _p(wf))
        _check(st, "or_mesh_load")

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.L.or_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # derived data ---------------------------------------------------------
    @property
    def n_free(self) -> int:
        return self.L.or_n_free(self.h)

    def geometry(self):
        T = self.mesh.n_tets
        jinv, x0, vol = np.zeros((T, 9)), np.zeros((T, 3)), np.zeros(T)
        self.L.or_geometry(self.h, _p(jinv), _p(x0), _p(vol))
        return jinv, x0, vol

    def matrix(self):
        n = self.n_free
        nnz = self.L.or_nnz(self.h)
        dof = np.zeros(self.mesh.n_nodes, np.int32)
        rowptr = np.zeros(n + 1, np.int32)
        col = np.zeros(nnz, np.int32)
        val = np.zeros(nnz)
        fN = np.zeros(n)
        self.L.or_matrix(self.h, _p(dof), _p(rowptr), _p(col), _p(val), _p(fN))
        return dof, rowptr, col, val, fN

    # state ----------------------------------------------------------------
    def init_potential(self):
        it, rr = C.c_int32(0), C.c_double(0)
        _check(self.L.or_init_potential(self.h, C.byref(it), C.byref(rr)), "or_init_potential")
        return it.value, rr.value

    def potential(self) -> np.ndarray:
        phi = np.zeros(self.mesh.n_nodes)
        self.L.or_get_potential(self.h, _p(phi))
        return phi

    def set_potential(self, phi):
        phi = np.ascontiguousarray(phi, np.float64)
        self.L.or_set_potential(self.h, _p(phi))

    def set_dirichlet(self, g):
        """Prescribed potential on the Dirichlet nodes (values elsewhere ignored)."""
        g = np.ascontiguousarray(g, np.float64)
        self.L.or_set_dirichlet(self.h, _p(g))

    def field(self) -> np.ndarray:
        E = np.zeros((self.mesh.n_tets, 3))
        self.L.or_get_field(self.h, _p(E))
        return E

    def particles(self):
        n = self.L.or_num_particles(self.h)
        r, v = np.zeros((n, 3)), np.zeros((n, 3))
        cell, pid = np.zeros(n, np.int32), np.zeros(n, np.int64)
        if n:
            self.L.or_get_particles(self.h, _p(r), _p(v), _p(cell), _p(pid))
        return r, v, cell, pid

    def set_particles(self, r, v, cell, pid):
        r = np.ascontiguousarray(r, np.float64)
        v = np.ascontiguousarray(v, np.float64)
        cell = np.ascontiguousarray(cell, np.int32)
        pid = np.ascontiguousarray(pid, np.int64)
        _check(self.L.or_set_particles(self.h, len(cell), _p(r), _p(v), _p(cell), _p(pid)),
               "or_set_particles")

    def charge(self) -> np.ndarray:
        W = np.zeros(self.mesh.n_nodes, np.int64)
        self.L.or_get_charge(self.h, _p(W))
        return W

    @property
    def step_index(self) -> int:
        return self.L.or_step_index(self.h)

    @step_index.setter
    def step_index(self, k):
        self.L.or_set_step_index(self.h, int(k))

    def set_work_function(self, wf):
        wf = np.ascontiguousarray(wf, np.float64)
        self.L.or_set_work_function(self.h, _p(wf))

    # the steps --------------------------------------------------------------
    def inject(self, step) -> int:
        n = C.c_int64(0)
        _check(self.L.or_inject(self.h, int(step), C.byref(n)), "or_inject")
        return n.value

    def push_relocate(self, step) -> Stats:
        st = Stats()
        _check(self.L.or_push_relocate(self.h, int(step), C.byref(st)), "or_push_relocate")
        return st

    def collide(self, step):
        """Binary collisions of the SPs in flight (App. F) for step `step`."""
        self.L.or_collide(self.h, int(step))

    def deposit(self) -> np.ndarray:
        _check(self.L.or_deposit(self.h), "or_deposit")
        return self.charge()

    def poisson_solve(self):
        it, rr = C.c_int32(0), C.c_double(0)
        _check(self.L.or_poisson_solve(self.h, C.byref(it), C.byref(rr)), "or_poisson_solve")
        return it.value, rr.value

    def solve(self, f, x0=None, rtol=1e-13, max_iter=200_000):
        """x with M x = f (free DOFs in the numbering of ``matrix``), Jacobi-PCG
        from x0 (zero) to the relative residual rtol."""
        f = np.ascontiguousarray(f, np.float64)
        x = np.zeros_like(f) if x0 is None else np.array(x0, np.float64, copy=True)
        it, rr = C.c_int32(0), C.c_double(0)
        _check(self.L.or_solve(self.h, _p(f), _p(x), float(rtol), int(max_iter), C.byref(it),
                               C.byref(rr)), "or_solve")
        return x

    def step(self, n=1):
        stats = (Stats * max(1, n))()
        _check(self.L.or_step(self.h, int(n), stats), "or_step")
        return list(stats)[:n]

    def locate(self, r, cell):
        r = np.array(r, np.float64, copy=True).reshape(-1, 3)
        cell = np.array(cell, np.int32, copy=True).reshape(-1)
        fate = np.zeros(len(cell), np.int32)
        wl = np.zeros(len(cell), np.int32)
        _check(self.L.or_locate(self.h, len(cell), _p(r), _p(cell), _p(fate), _p(wl)), "or_locate")
        return r, cell, fate, wl

    def barycentric(self, t, r):
        r = np.ascontiguousarray(r, np.float64)
        lam = np.zeros(4)
        self.L.or_barycentric(self.h, int(t), _p(r), _p(lam))
        return lam

    def quad_emission(self, field=None):
        """Per quadrangle: F, J_FN and n_sp (eq. nsp) of the oracle's current
        field, or of `field` [n_tets, 3] when given."""
        nq = 3 * self.mesh.n_faces
        F, J, n = np.zeros(nq), np.zeros(nq), np.zeros(nq)
        if field is None:
            self.L.or_quad_emission(self.h, _p(F), _p(J), _p(n))
        else:
            E = np.ascontiguousarray(field, np.float64).reshape(self.mesh.n_tets, 3)
            self.L.or_quad_emission_field(self.h, _p(E), _p(F), _p(J), _p(n))
        return F, J, n
