"""The measurement arithmetic of bench.py, on the CPU: the roofline object
(achieved = algorithmic bytes of the dominant kernel / its event time, frac =
achieved / the measured peak), the gate on the committed ncu traffic (used
only with the kernel source it was measured on), the structure of the
solver's byte model (k SpMVs per iteration at 8 bytes per stored FP32 entry,
linear in the iterations), and the per-step statistics layout shared with
the C header."""
import ctypes
import json
import os

import numpy as np
import pytest

import bench

INFO = dict(n_free=1000, nnz=14000, n_tets=5000, n_nodes=1100, n_faces=50)


def stats(n, iters=10, outer=1):
    st = np.zeros(n, dtype=bench.STAT_DTYPE)
    st["pcg_iters"] = iters
    st["pcg_outer"] = outer
    st["alive"] = 100
    st["injected"] = 5
    st["crossings"] = 1000
    return st


def test_roofline_takes_the_dominant_kernel_and_the_measured_peak(monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: (6000.0, "measured"))
    monkeypatch.setattr(bench, "ncu_traffic", lambda kernel, workload: 12345)
    st = stats(3)
    res = dict(info=INFO, stats=st, prof={"pcg": (3, 2.0), "step_fused": (3, 1.0)},
               prev_alive=np.array([100, 100, 100]), params={"pcg_cheb_degree": 6})
    roof, k = bench.roofline(res, fp64=False)
    alg = sum(bench.bytes_pcg_min(r, INFO, False) for r in st)
    alg_pre = sum(bench.bytes_pcg(r, INFO, False, 6) for r in st)
    assert roof["kernel"] == "pcg" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["achieved"] == pytest.approx(alg / 2.0e-3 / 1e9, abs=0.051)   # 0.1 GB/s steps
    assert roof["peak"] == 6000.0 and roof["peak_source"] == "measured"
    assert roof["frac"] == pytest.approx(roof["achieved"] / 6000.0, abs=1e-4)
    assert roof["alg_frac_incl_precond"] == pytest.approx(alg_pre / 2.0e-3 / 1e9 / 6000.0,
                                                          abs=1e-4)
    assert roof["traffic"] == 12345
    assert k["pcg"]["share"] == pytest.approx(2.0 / 3.0, abs=1e-4)
    assert k["pcg"]["alg_bytes_per_launch"] == int(alg / 3)
    assert k["step_fused"]["launches"] == 3


def test_minimal_solver_bytes_follow_the_scope_table():
    """One SpMV per CG iteration: I (nnz (s + 4) + 4 (n + 1) + 80 n) with s
    the value bytes, plus, in the FP32 form, 12 nnz + 24 n per refinement."""
    row = stats(1, iters=93, outer=2)[0]
    n, nnz = INFO["n_free"], INFO["nnz"]
    assert bench.bytes_pcg_min(row, INFO, True) == 93 * (nnz * 12 + 4 * (n + 1) + 80 * n)
    assert bench.bytes_pcg_min(row, INFO, False) == (93 * (nnz * 8 + 4 * (n + 1) + 80 * n)
                                                     + 2 * (12 * nnz + 24 * n))
    # never more than the count with every preconditioner SpMV
    assert bench.bytes_pcg_min(row, INFO, False) <= bench.bytes_pcg(row, INFO, False, 6)


def test_solver_byte_model_structure():
    row = stats(1)[0]

    def b(it, outer, k, fp64=False):
        r = row.copy()
        r["pcg_iters"] = it
        r["pcg_outer"] = outer
        return bench.bytes_pcg(r, INFO, fp64, k)

    def per_it(k, fp64=False):
        return b(11, 1, k, fp64) - b(10, 1, k, fp64)

    assert b(20, 1, 6) - b(10, 1, 6) == 10 * per_it(6)
    # every extra Chebyshev degree is one more SpMV: the FP32 matrix (value +
    # column index, 8 bytes per stored entry) and its vector update
    assert per_it(7) - per_it(6) == 8 * INFO["nnz"] + 20 * INFO["n_free"]
    assert per_it(1) >= 8 * INFO["nnz"]
    # FP64 values: 12 bytes per stored entry
    assert per_it(1, fp64=True) >= 12 * INFO["nnz"] > per_it(1)
    # each refinement adds an FP64 residual (matrix read once more)
    assert b(10, 2, 6) - b(10, 1, 6) >= 12 * INFO["nnz"]


def test_particle_kernel_onchip_roofline(monkeypatch):
    """When the fused particle kernel dominates, its roofline carries the L1
    data-stage figure from the committed capture: wavefronts over the
    captured duration against one wavefront per clock and SM."""
    monkeypatch.setattr(bench, "peaks", lambda: (6000.0, "measured"))
    monkeypatch.setattr(bench, "ncu_traffic", lambda kernel, workload: None)
    oc = dict(l1_wavefronts_per_launch=3.0e8, duration_ns=1.5e6, sms=152, sm_mhz=2000,
              l1_wavefronts_pct_of_peak_ncu=66.0)
    monkeypatch.setattr(bench, "ncu_onchip", lambda kernel, workload: oc if kernel == "step_fused" else None)
    st = stats(3)
    res = dict(info=INFO, stats=st, prof={"pcg": (3, 1.0), "step_fused": (3, 2.0)},
               prev_alive=np.array([100, 100, 100]), params={"pcg_cheb_degree": 6})
    roof, _ = bench.roofline(res, fp64=False)
    assert roof["kernel"] == "step_fused"
    o = roof["onchip"]
    assert o["achieved"] == pytest.approx(3.0e8 / 1.5e-3 / 1e9, abs=0.051)
    assert o["peak"] == pytest.approx(152 * 2.0, abs=0.051)
    assert o["frac"] == pytest.approx(o["achieved"] / o["peak"], abs=1e-4)
    assert o["frac_ncu"] == 66.0 and roof["solver"]["kernel"] == "pcg"


def test_fp64_walk_roofline_against_the_measured_rate(monkeypatch):
    """The FP64 arms' fused-kernel roofline: FP64 flops counted from the step
    statistics (per crossing and per SP) over the kernel's event time, against
    the rate pic_measure_fp64_rate returns."""
    import types
    fake = types.SimpleNamespace(measure_fp64_rate=lambda: 1.25)
    monkeypatch.setitem(__import__("sys").modules, "paper_1906_08125_gb300.picfem", fake)
    import paper_1906_08125_gb300
    monkeypatch.setattr(paper_1906_08125_gb300, "picfem", fake, raising=False)
    monkeypatch.setattr(bench, "_FP64_RATE", [])
    st = stats(2)
    r = dict(prof={"step_fused": (2, 4.0)}, prof_stats=st, prof_prev_alive=np.array([100, 100]))
    roof = bench.fp64_walk_roofline(r)
    flops = sum(bench.FP64_FLOPS_PER_CROSSING * 1000 + bench.FP64_FLOPS_PER_SP * (100 + 5)
                for _ in range(2))
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s" and roof["peak"] == 1.25
    assert roof["achieved"] == pytest.approx(flops / 4.0e-3 / 1e12, abs=1e-4)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 1.25, abs=1e-4)


def test_preconditioner_products_and_names():
    """Fine-level products per CG iteration: k for the Chebyshev polynomial
    of degree k, 2 k0 + 1 for the V-cycle with fine smoothing degree k0."""
    assert bench.precond_products({"pcg_cheb_local": 4, "pcg_mg_degree0": 3}, {}) == 7
    assert bench.precond_products({"pcg_cheb_local": 4, "pcg_mg_degree0": 1}, {}) == 3
    assert bench.precond_products({"pcg_cheb_local": 3}, {"pcg_cheb_degree": 6}) == 6
    info = {"mg_levels": 3, "mg_coarse_rows": 980}
    assert "V-cycle, 3 levels" in bench.precond_name(
        {"pcg_cheb_local": 4, "pcg_mg_degree0": 1, "pcg_mg_degree1": 3}, info)
    assert bench.precond_name({"pcg_cheb_local": 0, "pcg_cheb_degree": 0}, info) == "Jacobi"
    assert "coarse correction" in bench.precond_name({"pcg_cheb_local": 3, "pcg_cheb_degree": 6}, info)


def test_ncu_traffic_only_with_the_measured_source(monkeypatch):
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")))
    e = d["pcg"]
    monkeypatch.setattr(bench, "source_sha", lambda: e["source_sha"])
    assert bench.ncu_traffic("pcg", e["workload"]) == e["dram_bytes_per_launch"]
    assert bench.ncu_traffic("pcg", "another_workload") is None
    assert bench.ncu_traffic("no_such_kernel", e["workload"]) is None
    monkeypatch.setattr(bench, "source_sha", lambda: "0" * 16)
    assert bench.ncu_traffic("pcg", e["workload"]) is None


def test_source_sha_is_a_digest_of_the_kernel_sources():
    a, b = bench.source_sha(), bench.source_sha()
    assert a == b and len(a) == 16 and int(a, 16) >= 0


def test_step_stats_layout_matches_the_binding():
    from paper_1906_08125_gb300 import picfem
    assert bench.STAT_DTYPE.itemsize == ctypes.sizeof(picfem.StepStats)
    assert list(bench.STAT_DTYPE.names) == [f for f, _ in picfem.StepStats._fields_]
    for f, t in picfem.StepStats._fields_:
        assert bench.STAT_DTYPE.fields[f][1] == getattr(picfem.StepStats, f).offset, f
        assert bench.STAT_DTYPE.fields[f][0].itemsize == ctypes.sizeof(t), f


def test_pcg_variants_match_the_configs():
    from paper_1906_08125_gb300 import configs as K
    assert bench.PCG_VARIANTS == {"standard": K.PCG_STANDARD, "pipelined": K.PCG_PIPELINED,
                                  "merged": K.PCG_MERGED, "single": K.PCG_SINGLE}
