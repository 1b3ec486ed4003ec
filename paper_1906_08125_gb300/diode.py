"""The planar cathode-anode diode of the paper's PIC validation (Sec. III):
the self-consistent one-dimensional current density J(V) against which the
3D PIC steady state is compared.

Electrons leave the cathode (z = 0, Phi = 0) at rest with the field-emission
current density J = J_FN(F, phi_w) set by the cathode field F, and cross to
the anode (z = d, Phi = V).  In steady state the charge density is
rho = J / v(z) with v = sqrt(2 e Phi / m) (energy conservation), so Poisson's
equation reads Phi'' = k Phi^(-1/2), k = (J / eps0) sqrt(m / 2e).  Its first
integral with Phi'(0) = F is Phi'^2 = F^2 + 4 k sqrt(Phi), so the gap that
the potential V needs is

    d(F) = int_0^V dPhi / sqrt(F^2 + 4 k sqrt(Phi))
         = int_0^sqrt(V) 2u du / sqrt(F^2 + 4 k u),

which decreases monotonically in F (a larger F gives a larger integrand
denominator and, through J_FN, a larger k).  d(F) = d is solved by bisection
on (0, V/d] (at F = V/d the space charge already makes d(F) <= d); the
integral is taken by Gauss-Legendre quadrature (smooth integrand).  For
large V the result tends to the Child-Langmuir law
J_CL = (4 eps0 / 9) sqrt(2e/m) V^(3/2) / d^2, for small V to J_FN(V/d).

J_FN is the same closed form as the library's injection (Murphy-Good with
Forbes' v(f), t(f), f clamped to 1), written here for the host.
"""
from __future__ import annotations

import numpy as np

from . import configs as K

_A_FN, _B_FN, _CS2 = 1.541434e-6, 6.830890, 1.439964
_GL_X, _GL_W = np.polynomial.legendre.leggauss(64)


def fn_current(F, phi, model=K.FN_MURPHY_GOOD):
    """J_FN [A/m^2] for a field F [V/m] and a work function phi [eV]."""
    if not F > 0:
        return 0.0
    Fn = F * 1e-9
    v = t = 1.0
    if model == K.FN_MURPHY_GOOD:
        f = min(_CS2 * Fn / (phi * phi), 1.0)
        lf = np.log(f)
        v = 1.0 - f + f / 6.0 * lf
        t = 1.0 + f / 9.0 - f / 18.0 * lf
    return _A_FN * Fn * Fn / (phi * t * t) * np.exp(-v * _B_FN * phi ** 1.5 / Fn) * 1e18


def gap_needed(F, V, J):
    """d(F): the gap over which the potential rises to V when the cathode field
    is F and the current density J."""
    k = J / K.EPS0 * np.sqrt(K.M_E / (2.0 * K.E_CHARGE))
    s = np.sqrt(V)
    u = 0.5 * s * (_GL_X + 1.0)
    return 0.5 * s * float(np.sum(_GL_W * 2.0 * u / np.sqrt(F * F + 4.0 * k * u)))


def current_density(V, d, phi=4.5, model=K.FN_MURPHY_GOOD):
    """Self-consistent (J [A/m^2], cathode field F [V/m]) of the planar diode."""
    lo, hi = 0.0, V / d
    for _ in range(200):
        F = 0.5 * (lo + hi)
        if gap_needed(F, V, fn_current(F, phi, model)) > d:
            lo = F
        else:
            hi = F
    F = 0.5 * (lo + hi)
    return fn_current(F, phi, model), F


def child_langmuir(V, d):
    return 4.0 * K.EPS0 / 9.0 * np.sqrt(2.0 * K.E_CHARGE / K.M_E) * V ** 1.5 / (d * d)


# ---------------------------------------------------------------------------
# the 3D PIC sweep
# ---------------------------------------------------------------------------
VOLTAGES = (150.0, 200.0, 300.0, 400.0, 600.0, 800.0, 1000.0)
MESH = dict(area=135e-18, gap=18.2e-9, n_lat=4, h_cathode=0.01e-9, growth=1.03, h_max=0.3e-9)


def pic_current(picfem, mesh, V, dt=0.05e-15, sp_per_step=400, transits=4, precision=None):
    """Steady anode current density [A/m^2] of the PIC cycle on `mesh` with
    the anode at V: the SP weight gives about `sp_per_step` new SPs per step
    at the 1D current, the run takes `transits` space-charge transit times
    3d/v(V) to settle and the next `transits` to average the collected charge."""
    from . import inputs
    d = float(mesh.box_hi[2] - mesh.box_lo[2])
    A = float(np.prod(mesh.box_hi[:2] - mesh.box_lo[:2]))
    J1, _ = current_density(V, d, float(mesh.work_function[0]))
    w_sp = J1 * A * dt / (K.E_CHARGE * sp_per_step)
    t_tr = 3.0 * d / np.sqrt(2.0 * K.E_CHARGE * V / K.M_E)
    n = int(transits * t_tr / dt)
    p = K.params(dt=dt, E0=0.0, w_sp=w_sp, pcg_rtol=1e-10, capacity=2_000_000,
                 precision=K.PREC_FP64 if precision is None else precision, pcg_cheb_degree=0)
    c = picfem.Context(p).mesh_load(mesh)
    c.set_dirichlet(inputs.diode_potential(mesh, V))
    c.init_potential()
    c.step(n, stats=False)
    st = c.step(n)
    c.close()
    collected = np.array([s.collected for s in st], float)
    return collected.mean() * w_sp * K.E_CHARGE / dt / A, J1


def iv_sweep(picfem, voltages=VOLTAGES, mesh_kw=None, **kw):
    """PIC and 1D current densities over the voltages, and the RMS of the
    relative deviation."""
    from . import inputs
    mesh = inputs.diode_mesh(**(mesh_kw or MESH))
    rows = [(V,) + pic_current(picfem, mesh, V, **kw) for V in voltages]
    rel = np.array([jp / j1 - 1.0 for _, jp, j1 in rows])
    return {"voltages": [r[0] for r in rows], "J_pic": [r[1] for r in rows],
            "J_1d": [r[2] for r in rows], "rel_dev": rel.tolist(),
            "rms": float(np.sqrt(np.mean(rel ** 2))), "tets": int(mesh.n_tets),
            "layers": int(len(np.unique(mesh.xyz[:, 2])) - 1)}
