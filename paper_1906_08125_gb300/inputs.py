"""Seeded synthetic inputs: tetrahedral meshes of the vacuum above a cathode
(flat plate or field-emitting tip) and superparticle states.

This module builds input data only.  It holds none of the PIC/FEM arithmetic
(no fields, no emission, no push, no solve), so that the CUDA library and the
CPU oracle can both be fed from it without sharing any of the method.

Meshes follow the paper's setup (Sec. III.C): the vacuum domain Omega_1 sits in
a box whose bottom z = 0 is the cathode surface Gamma_3, whose top is the
far-field boundary Gamma_1 and whose sides Gamma_2 are laterally periodic.  The
paper meshes with FEMOCS (hexahedra split into tetrahedra, graded density);
here a tensor-product graded grid is split into the six Kuhn tetrahedra per
hexahedron, which is conforming and translation invariant (so opposite side
faces match for the periodic wrap), and tetrahedra whose centroid lies inside
the metal tip are removed.

Neighbour table convention: ``nbr[t, k]`` is the tetrahedron across the face
opposite local vertex k, or -1 (top, Gamma_1), -2 (cathode, Gamma_3) or
-3 (side, Gamma_2; the partner across the periodic boundary is
``periodic_nbr[t, k]``).
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

TOP, CATHODE, SIDE = -1, -2, -3


@dataclasses.dataclass
class Mesh:
    xyz: np.ndarray            # (N, 3) float64 [m]
    tet: np.ndarray            # (T, 4) int32, positively oriented
    nbr: np.ndarray            # (T, 4) int32
    periodic_nbr: np.ndarray   # (T, 4) int32, -1 where not a side face
    dirichlet: np.ndarray      # (N,) uint8, 1 on Gamma_3 nodes
    face_nodes: np.ndarray     # (F, 3) int32, (B-A)x(C-A) points into vacuum
    face_tet: np.ndarray       # (F,) int32, tetrahedron on the vacuum side
    work_function: np.ndarray  # (F,) float64 [eV]
    box_lo: np.ndarray
    box_hi: np.ndarray
    name: str = ""

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tet.shape[0])

    @property
    def n_faces(self) -> int:
        return int(self.face_nodes.shape[0])

    def arrays(self):
        """Contiguous arrays in the order the loaders take them."""
        c = np.ascontiguousarray
        return (c(self.xyz, np.float64), c(self.tet, np.int32), c(self.nbr, np.int32),
                c(self.periodic_nbr, np.int32), c(self.dirichlet, np.uint8),
                c(self.face_nodes, np.int32), c(self.face_tet, np.int32),
                c(self.work_function, np.float64))


# ---------------------------------------------------------------------------
# 1-D graded axes
# ---------------------------------------------------------------------------
def graded_half_axis(length: float, h_fine: float, fine_extent: float,
                     growth: float, h_max: float) -> np.ndarray:
    """Node coordinates from 0 to ``length``: spacing ``h_fine`` up to
    ``fine_extent``, then growing geometrically by ``growth`` up to ``h_max``;
    the whole axis is rescaled so that the last node lands on ``length``."""
    x = [0.0]
    h = h_fine
    while x[-1] < length:
        if x[-1] >= fine_extent:
            h = min(h * growth, h_max)
        x.append(x[-1] + h)
    if len(x) > 2 and x[-1] - length > 0.5 * (x[-1] - x[-2]):
        x.pop()
    x = np.asarray(x)
    return x * (length / x[-1])


def symmetric_axis(half: float, h_fine: float, fine_extent: float, growth: float,
                   h_max: float) -> np.ndarray:
    pos = graded_half_axis(half, h_fine, fine_extent, growth, h_max)
    return np.concatenate([-pos[:0:-1], pos])


# ---------------------------------------------------------------------------
# Kuhn split of a tensor-product grid
# ---------------------------------------------------------------------------
def _morton3(i, j, k):
    def spread(v):
        v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
        v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
        v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
        v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
        v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
        return v
    return spread(i) | (spread(j) << np.uint64(1)) | (spread(k) << np.uint64(2))


def kuhn_mesh(xs, ys, zs, inside_metal=None, work_function=4.5,
              work_function_spread=0.0, seed=0, name="") -> Mesh:
    """Split the grid xs x ys x zs into 6 Kuhn tetrahedra per hexahedron,
    remove tetrahedra whose centroid satisfies ``inside_metal(x, y, z)``, and
    build the neighbour, periodic and boundary tables."""
    xs, ys, zs = (np.asarray(a, np.float64) for a in (xs, ys, zs))
    nx, ny, nz = len(xs) - 1, len(ys) - 1, len(zs) - 1
    if nx < 2 or ny < 2 or nz < 1:
        raise ValueError("need at least 2 x 2 x 1 hexahedra")
    NX, NY = nx + 1, ny + 1

    def nid(i, j, k):
        return i + NX * (j + NY * k)

    hi, hj, hk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    hi, hj, hk = hi.ravel(), hj.ravel(), hk.ravel()
    order = np.argsort(_morton3(hi, hj, hk), kind="stable")
    hi, hj, hk = hi[order], hj[order], hk[order]

    unit = np.eye(3, dtype=np.int64)
    tets = []
    for perm in itertools.permutations(range(3)):
        a, b, _ = perm
        corners = [np.zeros(3, np.int64), unit[a], unit[a] + unit[b], np.ones(3, np.int64)]
        tets.append(np.stack([nid(hi + c[0], hj + c[1], hk + c[2]) for c in corners], axis=1))
    tet = np.stack(tets, axis=1).reshape(-1, 4)  # hex-major, 6 per hex

    gi = np.arange(NX * NY * (nz + 1))
    node_i = gi % NX
    node_j = (gi // NX) % NY
    node_k = gi // (NX * NY)
    xyz = np.stack([xs[node_i], ys[node_j], zs[node_k]], axis=1)

    # orientation: make det[x1-x0, x2-x0, x3-x0] > 0
    P = xyz[tet]
    d = np.einsum("ij,ij->i", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))
    neg = d < 0
    tet[neg, 2], tet[neg, 3] = tet[neg, 3].copy(), tet[neg, 2].copy()

    if inside_metal is not None:
        cen = xyz[tet].mean(axis=1)
        keep = ~inside_metal(cen[:, 0], cen[:, 1], cen[:, 2])
        tet = tet[keep]

    # drop unused nodes; number the rest along a Morton curve
    used = np.unique(tet)
    mort = _morton3(node_i[used], node_j[used], node_k[used])
    used = used[np.argsort(mort, kind="stable")]
    remap = -np.ones(xyz.shape[0], np.int64)
    remap[used] = np.arange(used.size)
    grid_of_new = used
    tet = remap[tet]
    xyz = xyz[used]
    T, N = tet.shape[0], xyz.shape[0]
    if N >= (1 << 21):
        raise ValueError("mesh too large for the 63-bit face keys")

    # faces: face k is opposite vertex k
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    fn = tet[:, loc]                      # (T, 4, 3)
    fs = np.sort(fn, axis=2).reshape(-1, 3)
    key = (fs[:, 0] << 42) | (fs[:, 1] << 21) | fs[:, 2]
    o = np.argsort(key, kind="stable")
    ks = key[o]
    same = ks[1:] == ks[:-1]
    nbr = np.full(4 * T, 0, np.int64)
    paired = np.zeros(4 * T, bool)
    a_idx, b_idx = o[:-1][same], o[1:][same]
    nbr[a_idx] = b_idx // 4
    nbr[b_idx] = a_idx // 4
    paired[a_idx] = True
    paired[b_idx] = True

    lo = np.array([xs[0], ys[0], zs[0]])
    hi_ = np.array([xs[-1], ys[-1], zs[-1]])
    bnd = np.nonzero(~paired)[0]
    fxyz = xyz[fs[bnd]]                    # (B, 3, 3)
    on = lambda ax, val: np.all(fxyz[:, :, ax] == val, axis=1)
    code = np.full(bnd.size, CATHODE, np.int64)
    side = on(0, lo[0]) | on(0, hi_[0]) | on(1, lo[1]) | on(1, hi_[1])
    code[side] = SIDE
    code[on(2, hi_[2])] = TOP
    code[on(2, lo[2])] = CATHODE
    nbr[bnd] = code

    # periodic partners: translate grid index i=0 <-> i=nx (and j)
    pnbr = np.full(4 * T, -1, np.int64)
    sb = bnd[code == SIDE]
    if sb.size:
        gn = grid_of_new[fs[sb]]           # grid ids of the face nodes
        gi_, gj_, gk_ = gn % NX, (gn // NX) % NY, gn // (NX * NY)
        newid_of_grid = -np.ones(NX * NY * (nz + 1), np.int64)
        newid_of_grid[grid_of_new] = np.arange(N)
        for ax, (lo_i, hi_i) in ((0, (0, nx)), (1, (0, ny))):
            comp = gi_ if ax == 0 else gj_
            at_lo = np.all(comp == lo_i, axis=1)
            at_hi = np.all(comp == hi_i, axis=1)

            def mapped_key(sel, to):
                ii, jj, kk = gi_[sel].copy(), gj_[sel].copy(), gk_[sel]
                if ax == 0:
                    ii[:] = to
                else:
                    jj[:] = to
                m = np.sort(newid_of_grid[ii + NX * (jj + NY * kk)], axis=1)
                return (m[:, 0] << 42) | (m[:, 1] << 21) | m[:, 2]

            klo = mapped_key(at_lo, hi_i)          # lo faces moved to hi
            khi = key[sb[at_hi]]                   # hi faces as they are
            ohi = np.argsort(khi)
            pos = np.searchsorted(khi[ohi], klo)
            if np.any(pos >= khi.size) or np.any(khi[ohi][np.minimum(pos, khi.size - 1)] != klo):
                raise ValueError("periodic side faces do not match")
            lo_faces = sb[at_lo]
            hi_faces = sb[at_hi][ohi[pos]]
            pnbr[lo_faces] = hi_faces // 4
            pnbr[hi_faces] = lo_faces // 4

    # cathode faces (the emitters) with the normal pointing into the vacuum
    cb = bnd[code == CATHODE]
    ft = cb // 4
    fk = cb % 4
    fnodes = fn.reshape(-1, 3)[cb].copy()
    A, B, C = xyz[fnodes[:, 0]], xyz[fnodes[:, 1]], xyz[fnodes[:, 2]]
    nrm = np.cross(B - A, C - A)
    opp = xyz[tet[ft, fk]]
    flip = np.einsum("ij,ij->i", nrm, opp - A) < 0
    fnodes[flip, 1], fnodes[flip, 2] = fnodes[flip, 2].copy(), fnodes[flip, 1].copy()

    dirichlet = np.zeros(N, np.uint8)
    dirichlet[fnodes.ravel()] = 1

    rng = np.random.default_rng(seed)
    wf = np.full(cb.size, float(work_function))
    if work_function_spread > 0:
        wf = wf + rng.uniform(-work_function_spread, work_function_spread, cb.size)

    return Mesh(xyz=xyz, tet=tet.astype(np.int32), nbr=nbr.reshape(T, 4).astype(np.int32),
                periodic_nbr=pnbr.reshape(T, 4).astype(np.int32), dirichlet=dirichlet,
                face_nodes=fnodes.astype(np.int32), face_tet=ft.astype(np.int32),
                work_function=wf, box_lo=lo, box_hi=hi_, name=name)


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------
NM = 1e-9


def plate_mesh(nx=20, ny=20, nz=40, lx=100 * NM, ly=100 * NM, lz=200 * NM,
               work_function=4.5, name="plate") -> Mesh:
    """Parallel-plate gap: uniform nx x ny x nz cubes, 6 tetrahedra each."""
    return kuhn_mesh(np.linspace(0, lx, nx + 1), np.linspace(0, ly, ny + 1),
                     np.linspace(0, lz, nz + 1), work_function=work_function, name=name)


def tip_mesh(radius=3 * NM, height=30 * NM, width=60 * NM, box_height=230 * NM,
             h_fine=0.4 * NM, lateral_growth=1.22, h_lat_max=3 * NM,
             h_shank=1.5 * NM, h_top_max=6 * NM, vertical_growth=1.2,
             work_function=4.5, work_function_spread=0.0, seed=0, name="tip") -> Mesh:
    """Hemisphere-capped cylinder (the field emitter) standing on the cathode
    plane, in a laterally periodic vacuum box; graded grid, finest around the
    tip and its apex."""
    R, h = radius, height
    xs = symmetric_axis(width / 2, h_fine, R + 2 * h_fine, lateral_growth, h_lat_max)
    # z: shank at h_shank, apex region at h_fine, then growing to h_top_max
    z_apex_lo, z_apex_hi = h - R - 1 * NM, h + 2 * NM
    zs = list(np.linspace(0.0, z_apex_lo, max(2, int(np.ceil(z_apex_lo / h_shank))) + 1))
    napex = int(np.ceil((z_apex_hi - z_apex_lo) / h_fine))
    zs += list(np.linspace(z_apex_lo, z_apex_hi, napex + 1)[1:])
    upper = graded_half_axis(box_height - z_apex_hi, h_fine, 0.0, vertical_growth, h_top_max)
    zs += list(z_apex_hi + upper[1:])
    zs = np.asarray(zs)

    def inside(x, y, z):
        rho2 = x * x + y * y
        cyl = (z <= h - R) & (rho2 < R * R)
        cap = (z > h - R) & (rho2 + (z - (h - R)) ** 2 < R * R)
        return cyl | cap

    return kuhn_mesh(xs, xs, zs, inside_metal=inside, work_function=work_function,
                     work_function_spread=work_function_spread, seed=seed, name=name)


# ---------------------------------------------------------------------------
# superparticle states
# ---------------------------------------------------------------------------
def random_particles(mesh: Mesh, n: int, seed: int = 0, v_scale: float = 1.0e7,
                     v_up: float = 1.0e7, z_min_frac: float = 0.0):
    """n SPs at uniformly random points of randomly chosen tetrahedra, with
    random velocities (isotropic part of scale ``v_scale`` plus ``v_up`` along
    +z).  Returns (r[n,3], v[n,3], cell[n], id[n]); the ids carry bit 62 so
    they never collide with the ids of injected SPs ((step << 42) | ...)."""
    rng = np.random.default_rng(seed)
    T = mesh.n_tets
    cand = np.arange(T)
    if z_min_frac > 0:
        zc = mesh.xyz[mesh.tet].mean(axis=1)[:, 2]
        zmin = mesh.box_lo[2] + z_min_frac * (mesh.box_hi[2] - mesh.box_lo[2])
        cand = cand[zc >= zmin]
    cell = rng.choice(cand, size=n).astype(np.int32)
    lam = rng.dirichlet(np.ones(4), size=n)
    r = np.einsum("ij,ijk->ik", lam, mesh.xyz[mesh.tet[cell]])
    v = rng.normal(0.0, v_scale, size=(n, 3))
    v[:, 2] += v_up
    pid = (np.int64(1) << np.int64(62)) + np.arange(n, dtype=np.int64)
    return r, v, cell, pid


# ---------------------------------------------------------------------------
# ensembles: several independent meshes in one batch
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Batch:
    """Replica meshes concatenated into one: replica r owns nodes
    [node_off[r], node_off[r+1]), tetrahedra [tet_off[r], tet_off[r+1]) and
    emitting faces [face_off[r], face_off[r+1]); it keeps its own coordinates
    (replicas overlap in space but share no tetrahedron).  E0[r] is its
    applied field and members[r] its own mesh."""
    mesh: Mesh
    node_off: np.ndarray
    tet_off: np.ndarray
    face_off: np.ndarray
    E0: np.ndarray
    members: list

    @property
    def n_rep(self) -> int:
        return len(self.members)


def batch_meshes(meshes, E0, name="batch") -> Batch:
    """Concatenate ``meshes`` with node/tetrahedron/face index offsets."""
    node_off = np.concatenate([[0], np.cumsum([m.n_nodes for m in meshes])]).astype(np.int64)
    tet_off = np.concatenate([[0], np.cumsum([m.n_tets for m in meshes])]).astype(np.int64)
    face_off = np.concatenate([[0], np.cumsum([m.n_faces for m in meshes])]).astype(np.int64)
    if node_off[-1] >= 2 ** 31 or tet_off[-1] >= 2 ** 31:
        raise ValueError("batch too large for 32-bit indices")

    def shifted(a, off):
        a = a.astype(np.int64)
        return np.where(a >= 0, a + off, a)

    lo = np.min([m.box_lo for m in meshes], axis=0)
    hi = np.max([m.box_hi for m in meshes], axis=0)
    mesh = Mesh(
        xyz=np.concatenate([m.xyz for m in meshes]),
        tet=np.concatenate([m.tet.astype(np.int64) + node_off[r]
                            for r, m in enumerate(meshes)]).astype(np.int32),
        nbr=np.concatenate([shifted(m.nbr, tet_off[r])
                            for r, m in enumerate(meshes)]).astype(np.int32),
        periodic_nbr=np.concatenate([shifted(m.periodic_nbr, tet_off[r])
                                     for r, m in enumerate(meshes)]).astype(np.int32),
        dirichlet=np.concatenate([m.dirichlet for m in meshes]),
        face_nodes=np.concatenate([m.face_nodes.astype(np.int64) + node_off[r]
                                   for r, m in enumerate(meshes)]).astype(np.int32),
        face_tet=np.concatenate([m.face_tet.astype(np.int64) + tet_off[r]
                                 for r, m in enumerate(meshes)]).astype(np.int32),
        work_function=np.concatenate([m.work_function for m in meshes]),
        box_lo=lo, box_hi=hi, name=name)
    return Batch(mesh=mesh, node_off=node_off, tet_off=tet_off, face_off=face_off,
                 E0=np.asarray(E0, dtype=np.float64), members=list(meshes))


# tip resolutions of the ensemble: mesh spacings scaled by these factors give
# about 1.0M, 485k, 260k, 137k and 64k tetrahedra at radius 3 nm (60 nm box)
# and 947k, 470k, 244k and 112k at radius 6 nm (80 nm box)
ENSEMBLE_SCALES = {3: (1.0, 1.4, 2.0, 2.8, 4.0), 6: (1.4, 2.0, 2.8, 4.0)}


def ensemble_tip(radius_nm: int, scale: float) -> Mesh:
    """Tip of the ensemble: radius 3 or 6 nm, all spacings times ``scale``."""
    width = 60 * NM if radius_nm == 3 else 80 * NM
    return tip_mesh(radius=radius_nm * NM, width=width, h_fine=0.4 * NM * scale,
                    h_shank=1.5 * NM * scale, h_lat_max=3 * NM * scale,
                    h_top_max=6 * NM * scale, name=f"tip_r{radius_nm}_s{scale}")


def ensemble(n_rep=64, seed=0, E0_range=(8e9, 12e9), scales=None) -> Batch:
    """Seeded ensemble of field-emitter replicas: radius 3 or 6 nm (equal
    odds), a mesh resolution drawn from ``scales`` (default
    ``ENSEMBLE_SCALES``), E0 ~ U(E0_range).  Identical meshes are built once."""
    rng = np.random.default_rng(seed)
    scales = scales or ENSEMBLE_SCALES
    cache, meshes, E0 = {}, [], []
    for _ in range(n_rep):
        rad = int(rng.choice(sorted(scales)))
        sc = float(rng.choice(scales[rad]))
        if (rad, sc) not in cache:
            cache[(rad, sc)] = ensemble_tip(rad, sc)
        meshes.append(cache[(rad, sc)])
        E0.append(rng.uniform(*E0_range))
    return batch_meshes(meshes, E0, name=f"ensemble{n_rep}")


# ---------------------------------------------------------------------------
# planar diode (the I-V validation of Sec. III)
# ---------------------------------------------------------------------------
def diode_mesh(area=135 * NM * NM, gap=18.2 * NM, n_lat=4, h_cathode=0.04 * NM,
               growth=1.06, h_max=0.5 * NM, work_function=4.5, name="diode") -> Mesh:
    """Planar cathode-anode gap: a square of the given area (laterally
    periodic) and height `gap`, z spacing `h_cathode` at the cathode growing
    geometrically to `h_max`; the cathode (z = 0) and the anode (z = gap)
    nodes are Dirichlet, every cathode face emits."""
    side = float(np.sqrt(area))
    zs = graded_half_axis(gap, h_cathode, 0.0, growth, h_max)
    xs = np.linspace(0.0, side, n_lat + 1)
    m = kuhn_mesh(xs, xs, zs, work_function=work_function, name=name)
    top = m.xyz[:, 2] >= m.box_hi[2]
    m.dirichlet = np.where(top, 1, m.dirichlet).astype(np.uint8)
    return m


def diode_potential(mesh: Mesh, V: float) -> np.ndarray:
    """Node values for pic_set_dirichlet: 0 on the cathode, V on the anode."""
    return np.where(mesh.xyz[:, 2] >= mesh.box_hi[2], float(V), 0.0)
