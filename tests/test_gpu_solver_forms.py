"""The inner FP32 solver forms of the FP32_IR Poisson solve (PIC_PCG_*)
against the oracle's tight FP64 solve: standard and merged (p.Ap summed on
the Chebyshev polynomial's first grid barrier, one barrier fewer per
iteration) with Jacobi, the whole-matrix Chebyshev polynomial, the
polynomial with the coarse correction and the multigrid V-cycle (where the
merged form does not apply it runs the standard one); the V-cycle in FP64;
pipelined (Jacobi only) on the
uniform plate, since its FP32 recurrences stagnate on the graded tip.  Every
form reaches the requested tolerance; the merged form takes the iterations
of the standard one, and where it does not apply (Jacobi, block-local
polynomials) it is the standard form bit for bit."""
import numpy as np
import pytest

from paper_1906_08125_gb300 import configs as K
from paper_1906_08125_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def picfem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_08125_gb300 import picfem as P
    P.load()
    return P


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def oracle_phi(oracle_mod, tip_small):
    """The oracle's tight charge-free and space-charge potentials of the
    small tip with a seeded SP population."""
    p = K.params(E0=1e10, w_sp=0.5, pcg_rtol=1e-13, pcg_max_iter=50000, capacity=100_000)
    orc = oracle_mod.Oracle(tip_small, p)
    orc.init_potential()
    phi0 = orc.potential()
    parts = inputs.random_particles(tip_small, 20000, seed=8, v_scale=3e6, v_up=6e6)
    orc.set_particles(*parts)
    orc.deposit()
    orc.poisson_solve()
    return phi0, orc.potential(), parts


PRECONDS = {"jacobi": dict(pcg_cheb_degree=0),
            "chebyshev": dict(pcg_cheb_degree=6),
            "chebyshev+coarse": dict(pcg_cheb_degree=6),
            "multigrid": dict(pcg_cheb_degree=6)}
LOCAL = {"chebyshev": 0, "chebyshev+coarse": 3, "multigrid": 4}


def solve(picfem, mesh, parts, variant, precond, rtol=1e-8):
    p = K.params(E0=1e10, w_sp=0.5, capacity=100_000, precision=K.PREC_FP32_IR,
                 pcg_rtol=rtol, pcg_variant=variant, **PRECONDS[precond])
    c = picfem.Context(p).mesh_load(mesh)
    if precond in LOCAL:
        c.set_tuning(pcg_cheb_local=LOCAL[precond])
    assert c.info()["pcg_resident"] == 1
    it0, rr0 = c.init_potential()
    phi0 = c.potential()
    c.set_particles(*parts)
    c.deposit()
    it1, rr1 = c.poisson_solve()
    return phi0, c.potential(), (it0, it1), (rr0, rr1), c


@pytest.mark.parametrize("precond", list(PRECONDS))
@pytest.mark.parametrize("variant", [K.PCG_STANDARD, K.PCG_MERGED, K.PCG_SINGLE])
def test_forms_reach_tolerance(picfem, tip_small, oracle_phi, variant, precond):
    phi0_o, phi1_o, parts = oracle_phi
    phi0, phi1, its, rrs, c = solve(picfem, tip_small, parts, variant, precond)
    assert max(rrs) <= 1e-8
    assert rel(phi0, phi0_o) <= 1e-7
    assert rel(phi1, phi1_o) <= 1e-7
    c.close()


def test_pipelined_on_uniform_plate(picfem, oracle_mod, plate_small):
    p = K.params(E0=1e10, w_sp=0.5, pcg_rtol=1e-13, pcg_max_iter=50000, capacity=100_000)
    orc = oracle_mod.Oracle(plate_small, p)
    parts = inputs.random_particles(plate_small, 8000, seed=4, v_scale=3e6, v_up=6e6)
    orc.init_potential()
    orc.set_particles(*parts)
    orc.deposit()
    orc.poisson_solve()
    phi0, phi1, its, rrs, c = solve(picfem, plate_small, parts, K.PCG_PIPELINED, "jacobi")
    assert max(rrs) <= 1e-8
    assert rel(phi1, orc.potential()) <= 1e-7
    c.close()


@pytest.mark.parametrize("variant", [K.PCG_MERGED, K.PCG_SINGLE])
@pytest.mark.parametrize("precond", ["chebyshev", "chebyshev+coarse"])
def test_merged_iterations_close_to_standard(picfem, tip_small, oracle_phi, precond, variant):
    """The merged and one-reduction forms take the standard form's iterations."""
    parts = oracle_phi[2]
    _, _, it_s, _, cs = solve(picfem, tip_small, parts, K.PCG_STANDARD, precond, rtol=1e-6)
    _, _, it_m, _, cm = solve(picfem, tip_small, parts, variant, precond, rtol=1e-6)
    for a, b in zip(it_m, it_s):
        assert abs(a - b) <= 0.05 * b + 2, (it_m, it_s)
    cs.close()
    cm.close()


@pytest.mark.parametrize("variant", [K.PCG_MERGED, K.PCG_SINGLE])
def test_merged_falls_back_to_standard_bit_for_bit(picfem, tip_small, oracle_phi, variant):
    """Where the merged or one-reduction form does not apply (Jacobi, the
    block-local polynomial) the standard form runs, bit for bit."""
    parts = oracle_phi[2]
    for precond, local in (("jacobi", None), ("chebyshev", 1)):
        out = []
        for variant_k in (K.PCG_STANDARD, variant):
            p = K.params(E0=1e10, w_sp=0.5, capacity=100_000, precision=K.PREC_FP32_IR,
                         pcg_rtol=1e-8, pcg_variant=variant_k, **PRECONDS[precond])
            c = picfem.Context(p).mesh_load(tip_small)
            if local is not None:
                c.set_tuning(pcg_cheb_local=local)
            c.init_potential()
            c.set_particles(*parts)
            c.deposit()
            it = c.poisson_solve()
            out.append((c.potential(), it))
            c.close()
        assert np.array_equal(out[0][0], out[1][0]), precond
        assert out[0][1] == out[1][1], precond


def test_merged_fused_steps_match_standard(picfem, tip_small):
    """Fused FP32_IR steps with the merged form: the same SPs as with the
    standard form (the potentials differ only within the solver tolerance,
    which moves no SP across a face on this case) and graph replays equal
    direct launches."""
    base = dict(E0=1e10, w_sp=0.5, capacity=100_000, seed=3, precision=K.PREC_FP32_IR,
                pcg_rtol=1e-10, pcg_cheb_degree=6)
    parts = inputs.random_particles(tip_small, 4000, seed=5, v_scale=4e6, v_up=6e6)
    res = {}
    for name, kw in (("std", dict(pcg_variant=K.PCG_STANDARD)),
                     ("merged", dict(pcg_variant=K.PCG_MERGED)),
                     ("merged_direct", dict(pcg_variant=K.PCG_MERGED, graph=0))):
        c = picfem.Context(K.params(**base, **kw)).mesh_load(tip_small)
        c.init_potential()
        c.set_particles(*parts)
        st = c.step(4)
        x, v, cell, pid = c.particles()
        o = np.argsort(pid)
        res[name] = (x[o], cell[o], pid[o], c.potential(), [s.pcg_relres for s in st])
        c.close()
    assert all(r <= 1e-10 for r in res["merged"][4])
    for k in range(3):
        assert np.array_equal(res["merged"][k], res["merged_direct"][k])
    assert np.array_equal(res["merged"][3], res["merged_direct"][3])
    assert np.array_equal(res["merged"][2], res["std"][2])
    assert np.abs(res["merged"][0] - res["std"][0]).max() <= 1e-6 * np.abs(res["std"][0]).max()
    assert rel(res["merged"][3], res["std"][3]) <= 1e-8


@pytest.mark.parametrize("variant", [K.PCG_STANDARD, K.PCG_MERGED])
@pytest.mark.parametrize("local", [0, 3, 4])
def test_tagged_exchange_equals_grid_barrier(picfem, tip_small, oracle_phi, variant, local):
    """The Chebyshev steps' neighbour exchange through tagged words
    (pcg_halo_sync = 1) moves the same values in the same order as the grid
    barrier form (0): identical potentials and iteration counts."""
    parts = oracle_phi[2]
    out = []
    for sync in (0, 1):
        p = K.params(E0=1e10, w_sp=0.5, capacity=100_000, precision=K.PREC_FP32_IR,
                     pcg_rtol=1e-8, pcg_variant=variant, pcg_cheb_degree=6)
        c = picfem.Context(p).mesh_load(tip_small)
        c.set_tuning(pcg_cheb_local=local, pcg_halo_sync=sync)
        assert c.tuning()["pcg_halo_sync"] == sync
        it0 = c.init_potential()
        c.set_particles(*parts)
        c.deposit()
        it1 = c.poisson_solve()
        out.append((c.potential(), it0, it1))
        c.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]


def test_tagged_exchange_over_many_launches(picfem, tip_small, oracle_phi):
    """300 solves of the same system from the same start in one context (the
    tag epoch wraps after 255 launches): every one equals the first bit for
    bit, so no launch ever took a value left over from an earlier one."""
    parts = oracle_phi[2]
    p = K.params(E0=1e10, w_sp=0.5, capacity=100_000, precision=K.PREC_FP32_IR,
                 pcg_rtol=1e-8, pcg_cheb_degree=6)
    c = picfem.Context(p).mesh_load(tip_small)
    c.init_potential()
    phi0 = c.potential()
    c.set_particles(*parts)
    c.deposit()
    first = None
    for k in range(300):
        c.set_potential(phi0)
        it = c.poisson_solve()
        phi = c.potential()
        if first is None:
            first = (phi, it)
        else:
            assert it == first[1], k
            assert np.array_equal(phi, first[0]), k
    c.close()


def test_tagged_exchange_graph_steps(picfem, tip_small):
    """Fused steps replayed from CUDA graphs with the tagged exchange equal
    direct launches with grid barriers, bit for bit."""
    base = dict(E0=1e10, w_sp=0.5, capacity=100_000, seed=3, precision=K.PREC_FP32_IR,
                pcg_rtol=1e-6, pcg_cheb_degree=6)
    parts = inputs.random_particles(tip_small, 4000, seed=5, v_scale=4e6, v_up=6e6)
    res = []
    for graph, sync in ((1, 1), (0, 0)):
        c = picfem.Context(K.params(graph=graph, **base)).mesh_load(tip_small)
        c.set_tuning(pcg_halo_sync=sync)
        c.init_potential()
        c.set_particles(*parts)
        st = c.step(7)
        x, v, cell, pid = c.particles()
        o = np.argsort(pid)
        res.append((x[o], v[o], cell[o], pid[o], c.potential(), [s.pcg_iters for s in st]))
        c.close()
    for a, b in zip(res[0], res[1]):
        if isinstance(a, list):
            assert a == b
        else:
            assert np.array_equal(a, b)


@pytest.mark.parametrize("variant", [K.PCG_STANDARD, K.PCG_MERGED, K.PCG_SINGLE])
def test_fp32_inner_solve_scale_invariant(picfem, tip_small, variant):
    """The FP32 inner solves work on the residual scaled by a power of two, so
    an applied field 2^+-100 times the usual one (right sides far outside the
    FP32 range) gives the usual potential times 2^+-100 bit for bit, with the
    same iterations."""
    out = {}
    for e in (0, -100, 100):
        p = K.params(E0=1e10 * 2.0 ** e, w_sp=0.5, capacity=1000, precision=K.PREC_FP32_IR,
                     pcg_rtol=1e-8, pcg_variant=variant, pcg_cheb_degree=6)
        c = picfem.Context(p).mesh_load(tip_small)
        it, rr = c.init_potential()
        out[e] = (c.potential() * 2.0 ** -e, it, rr)
        c.close()
    for e in (-100, 100):
        assert np.array_equal(out[e][0], out[0][0]), e
        assert out[e][1] == out[0][1] and out[e][2] == out[0][2], e


def test_single_reduction_fused_steps(picfem, tip_small):
    """Fused FP32_IR steps with the one-reduction form: graph replays equal
    direct launches bit for bit, and the SPs and potentials stay within the
    solver tolerance of the standard form's."""
    base = dict(E0=1e10, w_sp=0.5, capacity=100_000, seed=3, precision=K.PREC_FP32_IR,
                pcg_rtol=1e-10, pcg_cheb_degree=6)
    parts = inputs.random_particles(tip_small, 4000, seed=5, v_scale=4e6, v_up=6e6)
    res = {}
    for name, kw in (("std", dict(pcg_variant=K.PCG_STANDARD)),
                     ("single", dict(pcg_variant=K.PCG_SINGLE)),
                     ("single_direct", dict(pcg_variant=K.PCG_SINGLE, graph=0))):
        c = picfem.Context(K.params(**base, **kw)).mesh_load(tip_small)
        c.init_potential()
        c.set_particles(*parts)
        st = c.step(5)
        x, v, cell, pid = c.particles()
        o = np.argsort(pid)
        res[name] = (x[o], cell[o], pid[o], c.potential(), [s.pcg_relres for s in st])
        c.close()
    assert all(r <= 1e-10 for r in res["single"][4])
    for k in range(4):
        assert np.array_equal(res["single"][k], res["single_direct"][k])
    assert np.array_equal(res["single"][2], res["std"][2])
    assert np.abs(res["single"][0] - res["std"][0]).max() <= 1e-6 * np.abs(res["std"][0]).max()
    assert rel(res["single"][3], res["std"][3]) <= 1e-8


@pytest.mark.parametrize("precision", [K.PREC_FP64, K.PREC_FP32_IR])
def test_multigrid_against_the_oracle(picfem, tip_small, oracle_phi, precision):
    """The multigrid V-cycle (pcg_cheb_local = 4, the default where the
    hierarchy is built) in both precisions: the oracle's potentials to the
    requested tolerance, in fewer CG iterations than the two-level
    Chebyshev form, and the same result whether its exchanges go through
    tagged words or grid barriers."""
    phi0_o, phi1_o, parts = oracle_phi
    rtol = 1e-11 if precision == K.PREC_FP64 else 1e-8
    its = {}
    for local in (3, 4):
        p = K.params(E0=1e10, w_sp=0.5, capacity=100_000, precision=precision, pcg_rtol=rtol,
                     pcg_cheb_degree=6)
        c = picfem.Context(p).mesh_load(tip_small)
        assert c.tuning()["pcg_cheb_local"] == 4           # the default
        c.set_tuning(pcg_cheb_local=local)
        it0, rr0 = c.init_potential()
        assert rel(c.potential(), phi0_o) <= (1e-9 if precision == K.PREC_FP64 else 1e-7)
        c.set_particles(*parts)
        c.deposit()
        it1, rr1 = c.poisson_solve()
        assert max(rr0, rr1) <= rtol
        assert rel(c.potential(), phi1_o) <= (1e-9 if precision == K.PREC_FP64 else 1e-7)
        its[local] = it0 + it1
        c.close()
    assert its[4] < its[3], its
