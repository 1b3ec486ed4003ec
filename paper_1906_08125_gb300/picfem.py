"""ctypes binding of libpicfem (include/picfem.h): argument marshalling only.

Every step of the PIC cycle runs in the library's CUDA kernels; PyTorch
provides device memory (``torch.Tensor.data_ptr()``) and the stream.  There is
no CPU fallback: loading fails loudly when the library is missing or no CUDA
device is present.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

PIC_OK = 0
ERRORS = {-1: "PIC_ERR_ARG", -2: "PIC_ERR_CUDA", -3: "PIC_ERR_MESH", -4: "PIC_ERR_CAPACITY",
          -5: "PIC_ERR_WALK_LIMIT", -6: "PIC_ERR_NOT_CONVERGED", -7: "PIC_ERR_NOT_IMPLEMENTED",
          -8: "PIC_ERR_TIMEOUT"}
PREC_FP64, PREC_FP32_IR = 0, 1

EXPORTED = ["pic_create", "pic_destroy", "pic_last_error", "pic_version", "mesh_load",
            "mesh_load_batch", "pic_get_tuning", "pic_set_tuning", "pic_replica_info",
            "pic_mesh_info",
            "pic_init_potential", "inject", "push_relocate", "deposit", "poisson_solve",
            "pic_step", "pic_adjoint", "pic_set_applied_field", "pic_set_dirichlet",
            "pic_collide", "pic_get_step", "pic_set_step", "pic_get_potential",
            "pic_get_potential_async", "pic_set_potential", "pic_get_field", "pic_get_charge", "pic_num_particles",
            "pic_get_particles", "pic_set_particles", "pic_set_work_function",
            "pic_launch_count", "pic_profile_enable", "pic_profile_read", "pic_sync",
            "pic_pcg_solve_static", "pic_measure_fp64_rate"]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("E0", C.c_double), ("w_sp", C.c_double), ("q", C.c_double),
                ("q_over_m", C.c_double), ("eps0", C.c_double), ("e_charge", C.c_double),
                ("pcg_rtol", C.c_double), ("pcg_max_iter", C.c_int32), ("fn_model", C.c_int32),
                ("seed", C.c_uint64), ("capacity", C.c_int64), ("walk_max_steps", C.c_int32),
                ("quant_bits", C.c_int32), ("precision", C.c_int32), ("pcg_variant", C.c_int32),
                ("ir_inner_rtol", C.c_double), ("ir_inner_max_iter", C.c_int32),
                ("pcg_cheb_degree", C.c_int32), ("pcg_cheb_ratio", C.c_double),
                ("graph", C.c_int32), ("collisions", C.c_int32), ("coulomb_log", C.c_double)]


class Tuning(C.Structure):
    _fields_ = [("particle_blocks_per_sm", C.c_int32), ("walk_form", C.c_int32),
                ("pcg_blocks_per_sm", C.c_int32), ("pcg_cheb_degree", C.c_int32),
                ("pcg_balance", C.c_int32), ("pcg_cheb_local", C.c_int32),
                ("sort_cells", C.c_int32), ("pcg_halo_sync", C.c_int32),
                ("wait_limit", C.c_int32), ("pcg_mg_degree0", C.c_int32),
                ("pcg_mg_degree1", C.c_int32)]


class StepStats(C.Structure):
    _fields_ = [("injected", C.c_int64), ("collected", C.c_int64), ("absorbed", C.c_int64),
                ("wrapped", C.c_int64), ("crossings", C.c_int64), ("alive", C.c_int64),
                ("max_walk", C.c_int32), ("pcg_iters", C.c_int32), ("pcg_relres", C.c_double),
                ("collected_charge", C.c_double), ("pcg_outer", C.c_int32),
                ("reserved", C.c_int32), ("walk_warp_iters", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MeshInfo(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_tets", C.c_int32), ("n_faces", C.c_int32),
                ("n_free", C.c_int32), ("nnz", C.c_int64), ("sell_len", C.c_int64),
                ("pcg_grid", C.c_int32), ("particle_grid", C.c_int32),
                ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
                ("n_rep", C.c_int32), ("n_rows", C.c_int32), ("pcg_resident", C.c_int32),
                ("graph", C.c_int32), ("mg_levels", C.c_int32), ("mg_coarse_rows", C.c_int32)]


PROF_MAX = 16


class ProfileReport(C.Structure):
    _fields_ = [("n", C.c_int32), ("name", C.c_char_p * PROF_MAX),
                ("launches", C.c_int64 * PROF_MAX), ("ms", C.c_double * PROF_MAX)]


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpicfem.so (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise OSError(f"libpicfem not built at {path}")
    L = C.CDLL(path)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "pic_create": [C.POINTER(P), C.POINTER(Params), P],
        "pic_destroy": [P],
        "pic_last_error": [P],
        "pic_version": [],
        "mesh_load": [P, I32, P, I32, P, P, P, P, I32, P, P, P],
        "mesh_load_batch": [P, I32, P, P, P, I32, P, I32, P, P, P, P, I32, P, P, P],
        "pic_mesh_info": [P, C.POINTER(MeshInfo)],
        "pic_get_tuning": [P, C.POINTER(Tuning)],
        "pic_replica_info": [P, P, P, P, P],
        "pic_set_tuning": [P, C.POINTER(Tuning)],
        "pic_init_potential": [P, C.POINTER(I32), C.POINTER(D)],
        "inject": [P, I64, C.POINTER(I64)],
        "push_relocate": [P, I64, C.POINTER(StepStats)],
        "deposit": [P, P],
        "poisson_solve": [P, P, C.POINTER(I32), C.POINTER(D)],
        "pic_step": [P, I64, C.POINTER(StepStats)],
        "pic_adjoint": [P, I64, I32, P, P, P],
        "pic_set_applied_field": [P, P],
        "pic_set_dirichlet": [P, P],
        "pic_collide": [P, I64],
        "pic_get_step": [P, C.POINTER(I64)],
        "pic_set_step": [P, I64],
        "pic_get_potential": [P, P],
        "pic_get_potential_async": [P, P],
        "pic_set_potential": [P, P],
        "pic_get_field": [P, P],
        "pic_get_charge": [P, P],
        "pic_num_particles": [P, C.POINTER(I64)],
        "pic_get_particles": [P, P, P, P, P],
        "pic_set_particles": [P, I64, P, P, P, P],
        "pic_set_work_function": [P, P],
        "pic_launch_count": [P, C.POINTER(I64)],
        "pic_profile_enable": [P, I32],
        "pic_profile_read": [P, C.POINTER(ProfileReport)],
        "pic_sync": [P],
        "pic_pcg_solve_static": [I32, P, P, P, P, P, D, I32, C.POINTER(I32), C.POINTER(D), P],
        "pic_measure_fp64_rate": [P, I32, C.POINTER(D)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_char_p if name in ("pic_last_error", "pic_version") else C.c_int
    _lib = L
    return L


def measure_fp64_rate(iters: int = 1 << 14, stream=None) -> float:
    """The FP64 FMA rate of the current device in TFLOP/s
    (pic_measure_fp64_rate), on the given torch stream (the current one)."""
    import torch
    L = load()
    s = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_double(0.0)
    rc = L.pic_measure_fp64_rate(C.c_void_p(s.cuda_stream), int(iters), C.byref(out))
    if rc != 0:
        raise PicError(rc, f"pic_measure_fp64_rate failed ({rc})")
    return out.value


def _ptr(x):
    """Address of a numpy array or torch tensor (host or device), or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _params(d: dict) -> Params:
    return Params(**{k: d[k] for k, _ in Params._fields_})


class Context:
    """One libpicfem context (one mesh, one SP population) on the current
    CUDA device and torch stream."""

    def __init__(self, params: dict, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libpicfem needs a CUDA device; there is no CPU fallback")
        self.L = load()
        self.params = dict(params)
        self._p = _params(params)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        self._check(self.L.pic_create(C.byref(h), C.byref(self._p), C.c_void_p(stream.cuda_stream)),
                    ctx=None)
        self.h = h
        self.mesh = None

    def _check(self, rc, ctx="self"):
        if rc != PIC_OK:
            h = self.h if ctx == "self" else None
            msg = self.L.pic_last_error(h)
            raise PicError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.L.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def mesh_load(self, mesh):
        xyz, tet, nbr, pnbr, dirichlet, fnodes, ftet, wf = mesh.arrays()
        self._check(self.L.mesh_load(self.h, mesh.n_nodes, _ptr(xyz), mesh.n_tets, _ptr(tet),
                                     _ptr(nbr), _ptr(pnbr), _ptr(dirichlet), mesh.n_faces,
                                     _ptr(fnodes), _ptr(ftet), _ptr(wf)))
        self.mesh = mesh
        return self

    def mesh_load_batch(self, batch):
        """Load a ``inputs.Batch`` (replica meshes concatenated, with offsets)."""
        mesh = batch.mesh
        xyz, tet, nbr, pnbr, dirichlet, fnodes, ftet, wf = mesh.arrays()
        rno = np.ascontiguousarray(batch.node_off, dtype=np.int32)
        rto = np.ascontiguousarray(batch.tet_off, dtype=np.int32)
        e0 = np.ascontiguousarray(batch.E0, dtype=np.float64)
        self._check(self.L.mesh_load_batch(self.h, len(e0), _ptr(rno), _ptr(rto), _ptr(e0),
                                           mesh.n_nodes, _ptr(xyz), mesh.n_tets, _ptr(tet),
                                           _ptr(nbr), _ptr(pnbr), _ptr(dirichlet), mesh.n_faces,
                                           _ptr(fnodes), _ptr(ftet), _ptr(wf)))
        self.mesh = mesh
        return self

    def replica_info(self) -> dict:
        """Per replica: last solve's CG iterations (batches), stored matrix
        entries, solver rows, free DOFs."""
        R = self.info()["n_rep"]
        it, st = np.zeros(R, np.int32), np.zeros(R, np.int64)
        rows, free = np.zeros(R, np.int32), np.zeros(R, np.int32)
        self._check(self.L.pic_replica_info(self.h, _ptr(it), _ptr(st), _ptr(rows), _ptr(free)))
        return {"pcg_iters": it, "stored": st, "rows": rows, "free_dofs": free}

    def tuning(self) -> dict:
        t = Tuning()
        self._check(self.L.pic_get_tuning(self.h, C.byref(t)))
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def set_tuning(self, **kw):
        """Change launch knobs (see pic_set_tuning); unnamed ones are kept."""
        cur = self.tuning()
        unknown = set(kw) - set(cur)
        if unknown:
            raise KeyError(f"unknown tuning knobs {sorted(unknown)}")
        cur.update(kw)
        t = Tuning(**{k: int(v) for k, v in cur.items()})
        self._check(self.L.pic_set_tuning(self.h, C.byref(t)))
        return self

    def info(self) -> dict:
        m = MeshInfo()
        self._check(self.L.pic_mesh_info(self.h, C.byref(m)))
        d = {k: getattr(m, k) for k, _ in MeshInfo._fields_}
        d["box_lo"], d["box_hi"] = list(m.box_lo), list(m.box_hi)
        return d

    def init_potential(self):
        it, rr = C.c_int32(0), C.c_double(0)
        self._check(self.L.pic_init_potential(self.h, C.byref(it), C.byref(rr)))
        return it.value, rr.value

    def inject(self, step, sync=True):
        n = C.c_int64(0)
        self._check(self.L.inject(self.h, int(step), C.byref(n) if sync else None))
        return n.value if sync else None

    def push_relocate(self, step, sync=True):
        st = StepStats()
        self._check(self.L.push_relocate(self.h, int(step), C.byref(st) if sync else None))
        return st if sync else None

    def deposit(self, out=None):
        """out: int64 device tensor [n_nodes] (nullable)."""
        self._check(self.L.deposit(self.h, _ptr(out)))
        return out

    def poisson_solve(self, phi_out=None):
        it, rr = C.c_int32(0), C.c_double(0)
        self._check(self.L.poisson_solve(self.h, _ptr(phi_out), C.byref(it), C.byref(rr)))
        return it.value, rr.value

    def step(self, n=1, stats=True):
        arr = (StepStats * max(1, n))() if stats else None
        self._check(self.L.pic_step(self.h, int(n), arr))
        return list(arr)[:n] if stats else None

    def adjoint(self, n_steps, ckpt_every=20):
        """Collected charge Q over n_steps steps and (dQ/dE0 per replica,
        dQ/dphi per face) by reverse mode (pic_adjoint); leaves the context
        after the n_steps steps."""
        Q = np.zeros(1)
        gE0 = np.zeros(self.info()["n_rep"])
        gwf = np.zeros(max(1, self.mesh.n_faces))
        self._check(self.L.pic_adjoint(self.h, int(n_steps), int(ckpt_every), _ptr(Q), _ptr(gE0),
                                       _ptr(gwf)))
        return float(Q[0]), gE0, gwf[:self.mesh.n_faces]

    def collide(self, step):
        """Binary collisions of the SPs in flight (pic_collide)."""
        self._check(self.L.pic_collide(self.h, int(step)))

    def set_dirichlet(self, values):
        """Prescribed potential on the Dirichlet nodes (per node; other
        entries ignored)."""
        g = np.ascontiguousarray(values, np.float64)
        if len(g) != self.mesh.n_nodes:
            raise ValueError("one value per node")
        self._check(self.L.pic_set_dirichlet(self.h, _ptr(g)))

    def set_applied_field(self, E0):
        """E0 of each replica (a scalar for a single mesh); rebuilds the
        Neumann load, does not re-solve."""
        e = np.ascontiguousarray(np.atleast_1d(np.asarray(E0, np.float64)))
        if len(e) != self.info()["n_rep"]:
            raise ValueError("one E0 per replica")
        self._check(self.L.pic_set_applied_field(self.h, _ptr(e)))

    # state ---------------------------------------------------------------
    @property
    def step_index(self):
        k = C.c_int64(0)
        self._check(self.L.pic_get_step(self.h, C.byref(k)))
        return k.value

    @step_index.setter
    def step_index(self, k):
        self._check(self.L.pic_set_step(self.h, int(k)))

    def potential(self, out=None):
        if out is None:
            out = np.zeros(self.mesh.n_nodes)
        self._check(self.L.pic_get_potential(self.h, _ptr(out)))
        return out

    def get_potential_async(self, out):
        """Queue the copy of the potential into `out` (pinned host memory or a
        device tensor) on the context's stream; it is there once the stream
        has passed this call (an event recorded after it, or sync())."""
        self._check(self.L.pic_get_potential_async(self.h, _ptr(out)))
        return out

    def set_potential(self, phi):
        phi = np.ascontiguousarray(phi, np.float64) if isinstance(phi, np.ndarray) else phi
        self._check(self.L.pic_set_potential(self.h, _ptr(phi)))

    def field(self):
        E = np.zeros((self.mesh.n_tets, 3))
        self._check(self.L.pic_get_field(self.h, _ptr(E)))
        return E

    def charge(self):
        W = np.zeros(self.mesh.n_nodes, np.int64)
        self._check(self.L.pic_get_charge(self.h, _ptr(W)))
        return W

    def num_particles(self):
        n = C.c_int64(0)
        self._check(self.L.pic_num_particles(self.h, C.byref(n)))
        return n.value

    def particles(self):
        n = self.num_particles()
        r, v = np.zeros((n, 3)), np.zeros((n, 3))
        cell, pid = np.zeros(n, np.int32), np.zeros(n, np.int64)
        if n:
            self._check(self.L.pic_get_particles(self.h, _ptr(r), _ptr(v), _ptr(cell), _ptr(pid)))
        return r, v, cell, pid

    def set_particles(self, r, v, cell, pid):
        conv = lambda a, t: np.ascontiguousarray(a, t) if isinstance(a, np.ndarray) else a
        r, v = conv(r, np.float64), conv(v, np.float64)
        cell, pid = conv(cell, np.int32), conv(pid, np.int64)
        self._check(self.L.pic_set_particles(self.h, len(cell), _ptr(r), _ptr(v), _ptr(cell),
                                             _ptr(pid)))

    def set_work_function(self, wf):
        wf = np.ascontiguousarray(wf, np.float64) if isinstance(wf, np.ndarray) else wf
        self._check(self.L.pic_set_work_function(self.h, _ptr(wf)))

    # counters ------------------------------------------------------------
    def launch_count(self):
        n = C.c_int64(0)
        self._check(self.L.pic_launch_count(self.h, C.byref(n)))
        return n.value

    def profile(self, enable=True):
        self._check(self.L.pic_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self):
        rep = ProfileReport()
        self._check(self.L.pic_profile_read(self.h, C.byref(rep)))
        return {rep.name[i].decode(): (rep.launches[i], rep.ms[i]) for i in range(rep.n)}

    def sync(self):
        self._check(self.L.pic_sync(self.h))
