"""Benchmark of the GB300 FEM-PIC cycle: PIC cycles/s and particle pushes/s
on the 1M-tetrahedron nanotip workload, with the HBM-roofline fraction of the
dominant kernel, the plain FP64 form beside it, an end-to-end figure through
the C ABI with host buffers, and the CPU oracle as a reported baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one full PIC cycle (injection, push, walk, deposit, Poisson solve).
Every timed step is preceded by an L2 flush (a 256 MB write, outside the
step's events) and bracketed by CUDA events on the library's stream; the
steps replay their captured CUDA graphs as in production (no per-kernel
events).  The per-kernel split and the roofline come from a second pass of
the same length right after it with the library's per-kernel events on.
Several GPUs run independent replicas (the cycle does not shard; the
ensemble of runs does), each seeded by its rank.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PIC cycles/s"
WORKLOAD = "tip_1m"
# inner FP32 solver forms (PIC_PCG_*)
PCG_VARIANTS = {"standard": 0, "pipelined": 1, "merged": 2, "single": 3}
STAT_DTYPE = np.dtype([("injected", "<i8"), ("collected", "<i8"), ("absorbed", "<i8"),
                       ("wrapped", "<i8"), ("crossings", "<i8"), ("alive", "<i8"),
                       ("max_walk", "<i4"), ("pcg_iters", "<i4"), ("pcg_relres", "<f8"),
                       ("collected_charge", "<f8"), ("pcg_outer", "<i4"), ("reserved", "<i4"),
                       ("walk_warp_iters", "<i8")])


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=12)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="fp32_ir", choices=["fp32_ir", "fp64"])
    ap.add_argument("--pcg-variant", default="standard", choices=list(PCG_VARIANTS),
                    help="inner FP32 solver form of the main line")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--cpu-steps", type=int, default=10,
                    help="oracle steps timed for the CPU baseline (one thread and all cores)")
    ap.add_argument("--ensemble", type=int, default=64, help="replicas of the batched ensemble")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=200, help="0 skips the adjoint timing")
    ap.add_argument("--adjoint-ckpt", type=int, default=20)
    ap.add_argument("--large-steps", type=int, default=20, help="timed steps of the 8M-tet tip")
    ap.add_argument("--target-sp", type=int, default=0,
                    help="starting SPs of the main arm (0: the workload's own count)")
    ap.add_argument("--no-diode", action="store_true", help="skip the planar-diode I-V sweep")
    ap.add_argument("--no-large", action="store_true", help="skip the 8M-tet tip")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_sha():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1906_08125_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(f"{kernel}@{workload}") or d.get(kernel)
    if not e or e.get("source_sha") != source_sha():
        return None
    if e.get("workload") != workload:
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.lines = []
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader",
                                       "-lms", "200", "-i", str(self.dev)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                smax.append(float(f[2].split()[0]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def bench_population(mesh, n, seed):
    from paper_1906_08125_gb300 import inputs
    return inputs.random_particles(mesh, n, seed=seed, v_scale=3e6, v_up=1.5e7)


# ---------------------------------------------------------------------------
# algorithmic bytes per launch
# ---------------------------------------------------------------------------
def bytes_step_fused(st_prev_alive, st, s, info):
    """Algorithmic bytes of one fused particle step: the SoA state of the SPs
    read and written, N (6s + 4 + 8) each way; per face crossing of the walk
    the neighbour table and J^-1 of the next tetrahedron, 16 + 12 s; per
    occupied tetrahedron its record and field, 16 + 4*8 + 12 s (the occupied
    tetrahedra bounded by min(T, N)); the node charge written, 2 * 8 per
    node; 64 bytes per emitted SP."""
    n_old = st_prev_alive
    n_new = int(st["injected"])
    X = int(st["crossings"])
    n = n_old + n_new
    t_occ = min(info["n_tets"], n)
    return (n * 2 * (6 * s + 4 + 8) + X * (16 + 12 * s) + t_occ * (16 + 4 * 8 + 12 * s)
            + 2 * info["n_nodes"] * 8 + 64 * n_new)


def bytes_step_fused_compulsory(st_prev_alive, st, s, info, rec):
    """DRAM bytes one fused particle step cannot avoid: the SoA state read
    and written once, each walk record and field of the tetrahedra touched
    (at most all of them) once, the node charge written once."""
    n = st_prev_alive + int(st["injected"])
    alive = int(st["alive"])
    touched = min(info["n_tets"], n + int(st["crossings"]))
    return n * (6 * s + 12) + alive * (6 * s + 12) + touched * (rec + 4 * s) + 8 * info["n_nodes"]


def bytes_pcg(st, info, fp64, cheb):
    """Algorithmic bytes of one solve counting every SpMV of the
    preconditioner: every SpMV reads the stored matrix (values + column
    indices) and the vector it multiplies once; the vector updates read and
    write each vector they touch once.  A CG iteration with a Chebyshev
    preconditioner of degree k runs k SpMVs (k - 1 in the preconditioner, one
    for the search direction); the caller passes k = 2 k0 + 1 for the V-cycle
    with fine-level smoothing degree k0."""
    n, nnz = info["n_free"], info["nnz"]
    it, outer = int(st["pcg_iters"]), int(st["pcg_outer"])
    k = max(1, cheb)
    if fp64:
        per_it = 12 * nnz + 96 * n + (k - 1) * (12 * nnz + 40 * n)
        return it * per_it + (12 * nnz + 76 * n) + 20 * n
    per_it = 8 * nnz + 48 * n + (k - 1) * (8 * nnz + 20 * n)
    return it * per_it + (outer + 1) * (12 * nnz + 24 * n) + outer * 76 * n + 28 * n + 20 * n


def bytes_pcg_min(st, info, fp64):
    """Algorithmic bytes of one solve with one SpMV per CG iteration (the
    preconditioner's own products not counted): per iteration the stored
    matrix (s-byte value + 4-byte column per entry), the row pointers and ten
    vector sweeps of 8 bytes, I * (nnz (s + 4) + 4 (n + 1) + 80 n); the FP32
    form adds per FP64 refinement one FP64 residual product, 12 nnz + 24 n."""
    n, nnz = info["n_free"], info["nnz"]
    it, outer = int(st["pcg_iters"]), int(st["pcg_outer"])
    s = 8 if fp64 else 4
    total = it * (nnz * (s + 4) + 4 * (n + 1) + 80 * n)
    if not fp64:
        total += outer * (12 * nnz + 24 * n)
    return total


def bytes_field(info, s, rec):
    return info["n_tets"] * (rec + 16 + 4 * s) + 8 * info["n_nodes"]


def bytes_inject_count(info, s):
    return 3 * info["n_faces"] * (4 * s + 3 * 8 + 8 + 8 + 4 + 4)


def aggregate_replicas(total_ms, pushes, world, device):
    """Whole-job figures of N independent replicas: the time of the slowest
    rank (max over ranks) and the SP pushes of all ranks (sum).  One rank
    per GPU; any torch.distributed backend (NCCL on GPUs, gloo in tests)."""
    if world <= 1:
        return float(total_ms), pushes
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(pushes)], device=device, dtype=torch.float64)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
FORMS = {
    # the benchmark's form: FP32 push, FP32 Chebyshev-PCG (+ coarse correction)
    # inside FP64 refinement
    "fp32_ir": {},
    # the plain FP64 form: FP64 throughout, Jacobi-PCG
    "fp64": dict(precision=0, pcg_rtol=1e-6, pcg_cheb_degree=0),
    # FP64 throughout with the FP32 form's preconditioner (Chebyshev(6) and
    # the coarse correction over the solver blocks): separates precision
    # from preconditioning
    "fp64_twolevel": dict(precision=0, pcg_rtol=1e-6, pcg_cheb_degree=6),
}


def run_gpu(args, rank, world, form, timed_steps, warmup, prof_steps=None):
    """Warm-up, then `timed_steps` steps as production runs them (CUDA graph
    replays, no per-kernel events; L2 flushed before each step outside its
    events), then `prof_steps` more steps with the library's per-kernel
    events on for the kernel split."""
    import torch

    from paper_1906_08125_gb300 import configs as K
    from paper_1906_08125_gb300 import picfem

    mesh, p, _ = K.workload(args.workload, seed=rank)
    p = dict(p, **FORMS[form])
    if p["precision"] == K.PREC_FP32_IR:
        p = dict(p, pcg_variant=PCG_VARIANTS[args.pcg_variant])
    target = args.target_sp or K.WORKLOADS[args.workload]["target_sp"]
    stream = torch.cuda.current_stream()
    ctx = picfem.Context(p, stream=stream).mesh_load(mesh)
    info = ctx.info()
    ctx.init_potential()
    r, v, cell, pid = bench_population(mesh, target, seed=1000 + rank)
    ctx.set_particles(r, v, cell, pid)
    ctx.deposit()
    ctx.poisson_solve()          # space-charge potential of the starting population
    dev = torch.cuda.current_device()
    ctx.profile(False)
    for _ in range(warmup):
        ctx.step(1, stats=False)
    ctx.sync()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    L = ctx.L

    def timed(n, events):
        n0 = ctx.num_particles()
        dstats = torch.zeros(n * STAT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n)]
        base = dstats.data_ptr()
        for k in range(n):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            rc = L.pic_step(ctx.h, 1, picfem.C.cast(
                picfem.C.c_void_p(base + k * STAT_DTYPE.itemsize),
                picfem.C.POINTER(picfem.StepStats)))
            ev[k][1].record(stream)
            if rc != 0:
                ctx._check(rc)
        torch.cuda.synchronize()
        ctx.sync()
        st = np.frombuffer(dstats.cpu().numpy().tobytes(), dtype=STAT_DTYPE)
        prev = np.concatenate([[n0], st["alive"][:-1]])
        return [a.elapsed_time(b) for a, b in ev], st, prev, n0

    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.6)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    step_ms, st, prev, n0 = timed(timed_steps, True)
    launches = ctx.launch_count() - launches0
    graph = ctx.info()["graph"]
    clk = clocks.stop()
    total_ms, pushes = aggregate_replicas(float(sum(step_ms)), int((prev + st["injected"]).sum()),
                                          world, dev)
    prof, pst, pprev = {}, None, None
    if prof_steps:
        ctx.profile(True)
        pms, pst, pprev, _ = timed(prof_steps, False)
        prof = ctx.profile_read()
        ctx.profile(False)
    res = dict(ctx=ctx, mesh=mesh, params=p, info=info, tuning=ctx.tuning(), step_ms=step_ms,
               total_ms=total_ms,
               stats=st, prev_alive=prev, pushes=pushes, launches=launches, prof=prof,
               prof_stats=pst, prof_prev_alive=pprev, clocks=clk, n0=n0, graph=graph)
    return res


def ncu_onchip(kernel, workload):
    """On-chip pipe figures per launch from the committed single-kernel ncu
    summaries (the solver's shared-memory wavefronts, the particle kernel's
    L1 data-stage wavefronts), if taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_onchip.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(kernel)
    if not e or e.get("source_sha") != source_sha() or e.get("workload") != workload:
        return None
    return e


SMEM_BYTES_PER_CLK_PER_SM = 128      # one shared-memory wavefront per clock and SM
L1_WAVEFRONTS_PER_CLK_PER_SM = 1     # one L1 data-stage wavefront per clock and SM


def roofline(res, fp64):
    """Roofline of the dominant kernel from the profiled pass: algorithmic
    bytes per launch / its mean CUDA-event time against the measured HBM copy
    peak.  For the solver the bytes count one SpMV per CG iteration
    (bytes_pcg_min); the bytes with every SpMV of the Chebyshev
    preconditioner (bytes_pcg) are reported beside it."""
    info, prof = res["info"], res["prof"]
    st, prev = res.get("prof_stats"), res.get("prof_prev_alive")
    if st is None:
        st, prev = res["stats"], res["prev_alive"]
    s = 8 if fp64 else 4
    rec = 128 if fp64 else 64
    tun = res.get("tuning") or {}
    cheb = precond_products(tun, res["params"])
    alg = {
        "step_fused": sum(bytes_step_fused(int(pa), row, s, info) for pa, row in zip(prev, st)),
        "pcg": sum(bytes_pcg_min(row, info, fp64) for row in st),
        "field": len(st) * bytes_field(info, s, rec),
        "inject_count": len(st) * bytes_inject_count(info, s),
    }
    alg_precond = sum(bytes_pcg(row, info, fp64, cheb) for row in st)
    peak, kind = peaks()
    kernels = {name: {"launches": int(n), "ms": ms} for name, (n, ms) in prof.items()}
    total = sum(k["ms"] for k in kernels.values()) or 1.0
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    out_k = {}
    for name, k in kernels.items():
        gbs = alg[name] / (k["ms"] * 1e-3) / 1e9 if name in alg and k["ms"] > 0 else None
        out_k[name] = {"launches": k["launches"], "ms_total": round(k["ms"], 4),
                       "share": round(k["ms"] / total, 4),
                       "alg_bytes_per_launch": int(alg[name] / k["launches"]) if name in alg else None,
                       "alg_gbs": round(gbs, 1) if gbs else None}
    if "step_fused" in out_k:
        out_k["step_fused"]["note"] = ("bytes count one walk-record fetch per face crossing; "
                                       "neighbouring SPs share records in L1/L2, so this is "
                                       "not DRAM traffic")
    def kernel_roof(name):
        ms = kernels[name]["ms"]
        a = out_k[name]["alg_gbs"]
        r = {"bound": "hbm", "kernel": name, "achieved": a, "peak": peak, "unit": "GB/s",
             "frac": round(a / peak, 4) if a else None, "traffic": ncu_traffic(name, WORKLOAD),
             "peak_source": kind}
        if name == "step_fused":
            comp = sum(bytes_step_fused_compulsory(int(pa), row, s, info, rec)
                       for pa, row in zip(prev, st))
            r["bytes_model"] = ("N 2 (6s + 12) + X (16 + 12 s) + T_occ (48 + 12 s) + 16 N_nodes "
                                "+ 64 per new SP, X = face crossings (counted)")
            r["limiter"] = ("the L1 data stage: every face crossing loads a 64-byte walk "
                            "record per lane, the lanes at different records (ncu: local/global "
                            "wavefronts near 80 % of peak), with the dependent fetches' latency "
                            "behind it")
            r["compulsory"] = {"bytes_per_launch": int(comp / kernels[name]["launches"]),
                               "achieved": round(comp / (ms * 1e-3) / 1e9, 1), "unit": "GB/s",
                               "frac": round(comp / (ms * 1e-3) / 1e9 / peak, 4),
                               "model": "each SP state and each touched record once"}
            oc = ncu_onchip("step_fused", WORKLOAD)
            if oc:
                mhz = oc.get("sm_mhz") or (res.get("clocks") or {}).get("sm_mhz")
                sms = oc.get("sms", 152)
                wpeak = sms * L1_WAVEFRONTS_PER_CLK_PER_SM * mhz * 1e6 / 1e9
                wach = oc["l1_wavefronts_per_launch"] / (oc["duration_ns"] * 1e-9) / 1e9
                r["onchip"] = {"bound": "l1 data stage", "achieved": round(wach, 1),
                               "peak": round(wpeak, 1), "unit": "G wavefronts/s",
                               "frac": round(wach / wpeak, 4),
                               "frac_ncu": oc.get("l1_wavefronts_pct_of_peak_ncu"),
                               "basis": (f"one ncu-captured launch: local/global L1 data-stage "
                                         f"wavefronts over its duration; {sms} SMs x 1 wavefront/clk "
                                         f"at {mhz:.0f} MHz")}
        if name == "pcg":
            r["bytes_model"] = ("one SpMV per CG iteration: I (nnz (s + 4) + 4 (n + 1) + 80 n), "
                                "s = value bytes; FP32 form + refinements x (12 nnz + 24 n)")
            r["alg_frac_incl_precond"] = round(alg_precond / (ms * 1e-3) / 1e9 / peak, 4)
            oc = ncu_onchip("pcg", WORKLOAD)
            if oc:
                mhz = oc.get("sm_mhz") or (res.get("clocks") or {}).get("sm_mhz")
                sms = oc.get("sms", 152)
                speak = sms * SMEM_BYTES_PER_CLK_PER_SM * mhz * 1e6 / 1e9
                sach = oc["smem_bytes_per_launch"] / (oc["duration_ns"] * 1e-9) / 1e9
                r["onchip"] = {"bound": "smem", "achieved": round(sach, 1),
                               "peak": round(speak, 1), "unit": "GB/s",
                               "frac": round(sach / speak, 4),
                               "basis": (f"one ncu-captured launch: shared-memory wavefronts x "
                                         f"128 B over its duration; {sms} SMs x 128 B/clk at "
                                         f"{mhz:.0f} MHz")}
                r["limiter"] = oc.get("limiter")
                r["dram_pct_of_peak_ncu"] = oc.get("dram_pct_of_peak")
        return r

    roof = kernel_roof(dom)
    if dom != "pcg" and "pcg" in kernels:
        roof["solver"] = kernel_roof("pcg")
    return roof, out_k


# ---------------------------------------------------------------------------
# the batched ensemble: 64 field-emitter replicas in one context
# ---------------------------------------------------------------------------
ENSEMBLE_WSP = 0.015


def ensemble_inputs(n_rep):
    """The seeded ensemble (radius 3 or 6 nm, E0 ~ U(8, 12) GV/m, 64k-1M tets
    per replica) and a starting population of 10 % of each replica's
    tetrahedron count, clipped to 1e4-5e5 SPs, in batch numbering."""
    from paper_1906_08125_gb300 import inputs
    b = inputs.ensemble(n_rep=n_rep, seed=0)
    pops = []
    for r, m in enumerate(b.members):
        n = int(np.clip(0.1 * m.n_tets, 1e4, 5e5))
        x, v, cell, pid = inputs.random_particles(m, n, seed=100 + r, v_scale=3e6, v_up=1.5e7)
        pops.append((x, v, cell + b.tet_off[r], pid + (np.int64(r) << np.int64(32))))
    cat = tuple(np.concatenate([p[k] for p in pops]) for k in range(4))
    return b, (cat[0], cat[1], cat[2].astype(np.int32), cat[3])


def bytes_batch_pcg(ri, fp64, cheb, outer, minimal=True):
    """The solver's bytes summed over the replicas of a batch, each with its
    own iteration count (the last solve's), stored entries and free DOFs:
    bytes_pcg_min (one SpMV per iteration), or bytes_pcg with every SpMV of
    the preconditioner."""
    total = 0
    for it, nnz, n in zip(ri["pcg_iters"], ri["stored"], ri["free_dofs"]):
        row = {"pcg_iters": int(it), "pcg_outer": outer}
        inf = {"n_free": int(n), "nnz": int(nnz)}
        total += bytes_pcg_min(row, inf, fp64) if minimal else bytes_pcg(row, inf, fp64, cheb)
    return total


def run_ensemble(n_rep, steps, warmup):
    import torch
    from paper_1906_08125_gb300 import autotune
    from paper_1906_08125_gb300 import configs as K
    from paper_1906_08125_gb300 import picfem as P
    P.load()
    b, cat = ensemble_inputs(n_rep)
    peak, kind = peaks()
    # FP32+IR and FP64 with the same multigrid V-cycle (the default where
    # pcg_cheb_degree >= 2), and FP64 with Jacobi
    forms = {"fp32_ir": dict(precision=K.PREC_FP32_IR, pcg_rtol=1e-6, pcg_cheb_degree=6),
             "fp64_mg": dict(precision=K.PREC_FP64, pcg_rtol=1e-6, pcg_cheb_degree=6),
             "fp64": dict(precision=K.PREC_FP64, pcg_rtol=1e-6, pcg_cheb_degree=0)}
    sequential_forms = ("fp32_ir", "fp64_mg", "fp64")
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = {"replicas": n_rep, "tets": int(b.mesh.n_tets), "nodes": int(b.mesh.n_nodes),
           "emitting_faces": int(b.mesh.n_faces), "sp_start": int(len(cat[3])),
           "w_sp": ENSEMBLE_WSP, "pcg_rtol": 1e-6,
           "l2": "not flushed: the batch's matrix and SPs (> 1 GB) exceed L2",
           "batched": {}, "sequential": {}}
    state = None
    for name, form in forms.items():
        p = K.params(w_sp=ENSEMBLE_WSP, capacity=12_000_000, **form)
        c = P.Context(p).mesh_load_batch(b)
        c.init_potential()
        c.set_particles(*cat)
        c.deposit()
        c.poisson_solve()
        c.step(warmup, stats=False)
        entry = {}
        if name == "fp32_ir":
            state = (c.potential(), c.particles(), c.step_index)
            knobs, _, trials = autotune.tune(
                c, steps=3, warmup=1, use_cache=False,
                space={"particle_blocks_per_sm": (8, 16, 24), "pcg_mg_degree1": (2, 3)})
            entry["tuning"] = knobs
            entry["tuning_trials"] = len(trials)
            c.step(2, stats=False)                  # balance on the tuned solves
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        st = c.step(steps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ri = c.replica_info()
        c.profile(True)
        c.step(2, stats=False)
        prof = c.profile_read()
        c.profile(False)
        pcg_ms = prof["pcg"][1] / prof["pcg"][0]
        tun = c.tuning()
        cheb = precond_products(tun, form)
        outer = int(np.median([s.pcg_outer for s in st]))
        is64 = form["precision"] == K.PREC_FP64
        alg = bytes_batch_pcg(ri, is64, cheb, outer)
        gbs = alg / (pcg_ms * 1e-3) / 1e9
        gbs_pre = bytes_batch_pcg(ri, is64, cheb, outer, minimal=False) / (pcg_ms * 1e-3) / 1e9
        entry.update({"preconditioner": precond_name(tun, c.info()),
                      "ms_per_step": round(ms, 3),
                      "replica_cycles_per_s": round(n_rep * 1e3 / ms, 1),
                      "sp_in_flight": int(st[-1].alive),
                      "pcg_ms_per_step": round(pcg_ms, 3),
                      "pcg_share": round(pcg_ms * prof["pcg"][0]
                                         / sum(v[1] for v in prof.values()), 3),
                      "pcg_iters_replicas": [int(ri["pcg_iters"].min()),
                                             int(np.median(ri["pcg_iters"])),
                                             int(ri["pcg_iters"].max())],
                      "roofline_pcg": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak,
                                       "unit": "GB/s", "frac": round(gbs / peak, 4),
                                       "alg_frac_incl_precond": round(gbs_pre / peak, 4),
                                       "peak_source": kind}})
        out["batched"][name] = entry
        c.close()
    # the same replicas one context at a time, from the FP32 batch's state
    phi, parts, k = state
    rid = np.searchsorted(b.tet_off, parts[2], side="right") - 1
    for name in sequential_forms:
        form = forms[name]
        tot = 0.0
        for r, m in enumerate(b.members):
            p = K.params(w_sp=ENSEMBLE_WSP, capacity=2_000_000, E0=float(b.E0[r]), seed=r, **form)
            c = P.Context(p).mesh_load(m)
            c.set_potential(phi[b.node_off[r]:b.node_off[r + 1]])
            sel = rid == r
            ids = parts[3][sel].copy()
            inj = (ids >> np.int64(62)) == 0
            ids[inj] -= np.int64(3 * b.face_off[r]) << np.int64(18)
            c.set_particles(parts[0][sel], parts[1][sel],
                            (parts[2][sel] - b.tet_off[r]).astype(np.int32), ids)
            c.step_index = k
            c.step(2, stats=False)
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record()
            c.step(4, stats=False)
            e1.record()
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1) / 4
            c.close()
        out["sequential"][name] = {"ms_per_ensemble_step": round(tot, 3),
                                   "replica_cycles_per_s": round(n_rep * 1e3 / tot, 1)}
    return out


def run_adjoint_bench(workload, steps, ckpt_every):
    """pic_adjoint on the benchmark workload: the collected charge over
    `steps` steps and its gradient in E0 and every face's work function, timed
    against the same steps run forward only (both from the same state)."""
    import torch
    from paper_1906_08125_gb300 import configs as K
    from paper_1906_08125_gb300 import picfem
    mesh, p, _ = K.workload(workload)
    ctx = picfem.Context(p).mesh_load(mesh)
    ctx.init_potential()
    ctx.set_particles(*bench_population(mesh, K.WORKLOADS[workload]["target_sp"], seed=1000))
    ctx.deposit()
    ctx.poisson_solve()
    ctx.step(5, stats=False)
    phi, parts, k = ctx.potential(), ctx.particles(), ctx.step_index
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.step(steps, stats=False)
    ctx.sync()
    fwd = (time.perf_counter() - t0) * 1e3
    ctx.set_potential(phi)
    ctx.set_particles(*parts)
    ctx.step_index = k
    ctx.sync()
    t0 = time.perf_counter()
    Q, gE0, gwf = ctx.adjoint(steps, ckpt_every=ckpt_every)
    adj = (time.perf_counter() - t0) * 1e3
    ctx.close()
    return {"workload": workload, "steps": steps, "ckpt_every": ckpt_every,
            "precision": "fp32_ir", "faces": int(mesh.n_faces),
            "forward_ms": round(fwd, 2), "adjoint_ms": round(adj, 2),
            "adjoint_over_forward": round(adj / fwd, 2), "Q_C": Q,
            "dQ_dE0": float(gE0[0]), "dQ_dphi_l2": float(np.linalg.norm(gwf)),
            "dQ_dphi_nonzero_faces": int((gwf != 0).sum())}


def run_large(workload, steps, warmup):
    """A few steps of a workload larger than the resident solver holds (the
    8M-tet tip: the matrix and vectors exceed L2, the solver runs the general
    kernels), from the seeded starting population."""
    import torch
    from paper_1906_08125_gb300 import configs as K
    from paper_1906_08125_gb300 import picfem
    t0 = time.perf_counter()
    mesh, p, _ = K.workload(workload)
    ctx = picfem.Context(p).mesh_load(mesh)
    info = ctx.info()
    ctx.init_potential()
    ctx.set_particles(*bench_population(mesh, K.WORKLOADS[workload]["target_sp"], seed=2000))
    ctx.deposit()
    ctx.poisson_solve()
    ctx.step(warmup, stats=False)
    setup_s = time.perf_counter() - t0
    tun = ctx.tuning()
    snap = ctx.potential(), ctx.particles(), ctx.step_index

    def timed(n):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = ctx.step(n)
        e1.record()
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.step(2, stats=False)
        prof = ctx.profile_read()
        ctx.profile(False)
        return st, e0.elapsed_time(e1) / n, prof["pcg"][1] / prof["pcg"][0]

    st, ms, pcg_ms = timed(steps)
    # the same steps from the same state with the two-level polynomial
    # preconditioner the V-cycle replaced (context for the solver's speed-up)
    two = None
    if tun["pcg_cheb_local"] == 4:
        ctx.set_tuning(pcg_cheb_local=3)
        ctx.set_potential(snap[0])
        ctx.set_particles(*snap[1])
        ctx.step_index = snap[2]
        ctx.step(2, stats=False)
        st2, ms2, pcg2 = timed(5)
        two = {"steps": 5, "ms_per_step": round(ms2, 3), "pcg_ms_per_step": round(pcg2, 3),
               "pcg_iters": int(np.median([s.pcg_iters for s in st2]))}
    ctx.close()
    row = {"pcg_iters": int(np.median([s.pcg_iters for s in st])),
           "pcg_outer": int(np.median([s.pcg_outer for s in st]))}
    alg = bytes_pcg_min(row, info, False)
    peak, kind = peaks()
    gbs = alg / (pcg_ms * 1e-3) / 1e9
    gbs_pre = bytes_pcg(row, info, False, precond_products(tun, p)) / (pcg_ms * 1e-3) / 1e9
    return {"workload": workload, "tets": info["n_tets"], "free_dofs": info["n_free"],
            "nnz": info["nnz"], "resident_solver": bool(info["pcg_resident"]),
            "preconditioner": precond_name(tun, info),
            "sp_in_flight": int(st[-1].alive), "steps": steps, "warmup": warmup,
            "ms_per_step": round(ms, 3), "value": round(1e3 / ms, 2), "unit": METRIC,
            "pcg_ms_per_step": round(pcg_ms, 3), "pcg_iters": row["pcg_iters"],
            "pcg_grid": info["pcg_grid"],
            "roofline_pcg": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak,
                             "unit": "GB/s", "frac": round(gbs / peak, 4),
                             "alg_frac_incl_precond": round(gbs_pre / peak, 4),
                             "traffic": ncu_traffic("pcg", workload), "peak_source": kind},
            "two_level_precond": two,
            "setup_s": round(setup_s, 1)}


def precond_products(tun, p):
    """Fine-level products per CG iteration, the CG's own included: k for
    the Chebyshev polynomial of degree k, 2 k0 + 1 for the V-cycle with
    fine-level smoothing degree k0 (k0 - 1 steps and the residual before the
    coarse correction, the residual and k0 - 1 steps after it); the coarser
    levels' products are not counted."""
    if tun.get("pcg_cheb_local") == 4:
        return 2 * tun.get("pcg_mg_degree0", 3) + 1
    return p.get("pcg_cheb_degree", tun.get("pcg_cheb_degree", 0))


def precond_name(tun, info):
    local = tun.get("pcg_cheb_local")
    if local == 4:
        return (f"multigrid V-cycle, {info['mg_levels']} levels below the fine one, "
                f"coarsest {info['mg_coarse_rows']} rows (dense inverse), Chebyshev "
                f"smoothing degrees {tun['pcg_mg_degree0']} / {tun['pcg_mg_degree1']}")
    if local == 3 or (local == 0 and tun.get("pcg_cheb_degree", 0) >= 2):
        return f"Chebyshev({tun['pcg_cheb_degree']}) of D^-1 M" + (
            " + aggregate coarse correction" if local == 3 else "")
    return "Jacobi"


def run_e2e(res, steps):
    """The same metric through the C ABI with host buffers: per step the
    per-face work function goes host->device from pinned memory, one cycle
    runs, and the node potential comes back device->host into pinned memory
    (pic_get_potential_async) with the step statistics.  One step is kept
    queued ahead: after queueing step k the host waits for step k-1's event,
    so each step's result is on the host before the next but one is queued,
    and the GPU never waits for the host.  Per-kernel profiling is off here
    (it is on in the device-timed region for the live kernel split), so the
    steps replay their CUDA graphs as a user's would."""
    import torch
    from paper_1906_08125_gb300 import picfem
    ctx, mesh = res["ctx"], res["mesh"]
    stream = torch.cuda.current_stream()
    wf = torch.from_numpy(np.ascontiguousarray(mesh.work_function, np.float64)).pin_memory()
    phi = [torch.empty(mesh.n_nodes, dtype=torch.float64).pin_memory() for _ in range(2)]
    sz = picfem.C.sizeof(picfem.StepStats)
    dstats = torch.zeros(2 * sz, dtype=torch.uint8, device=torch.cuda.current_device())
    hstats = [torch.empty(sz, dtype=torch.uint8).pin_memory() for _ in range(2)]
    ev = [torch.cuda.Event() for _ in range(2)]
    L = ctx.L
    # the production configuration: no per-kernel events, so pic_step replays
    # its captured graphs (captured in two untimed iterations of this loop)
    ctx.profile(False)
    warm = 2
    t0 = None
    collected = 0
    for k in range(warm + steps):
        if k == warm:
            ev[(k - 1) & 1].synchronize()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        b = k & 1
        ctx._check(L.pic_set_work_function(ctx.h, wf.data_ptr()))
        ctx._check(L.pic_step(ctx.h, 1, picfem.C.cast(
            picfem.C.c_void_p(dstats.data_ptr() + b * sz), picfem.C.POINTER(picfem.StepStats))))
        ctx._check(L.pic_get_potential_async(ctx.h, phi[b].data_ptr()))
        hstats[b].copy_(dstats[b * sz:(b + 1) * sz], non_blocking=True)
        ev[b].record(stream)
        if k >= 1:
            ev[1 - b].synchronize()
            collected += int(picfem.StepStats.from_buffer_copy(hstats[1 - b].numpy()).collected)
    ev[(warm + steps - 1) & 1].synchronize()
    ctx.sync()
    dt = time.perf_counter() - t0
    return {"value": round(steps / dt, 3), "unit": "PIC cycles/s",
            "h2d_bytes_per_step": 8 * mesh.n_faces,
            "d2h_bytes_per_step": sz + 8 * mesh.n_nodes}


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def host_cpu():
    """The host's logical CPUs and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu model")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


def run_oracle(workload, steps, seed=0, parallel=False):
    """The FP64 oracle on the host: `steps` full PIC steps of the workload from
    the benchmark's seeded starting population (deposited and solved first,
    untimed).  parallel: the OpenMP build on every host core (bit-identical
    results); else the serial build on one core."""
    from oracle import oracle as O
    from paper_1906_08125_gb300 import configs as K
    mesh, p, _ = K.workload(workload)
    target = K.WORKLOADS[workload]["target_sp"]
    p = dict(p, precision=K.PREC_FP64)
    cores = O.set_threads(os.cpu_count()) if parallel else 1
    orc = O.Oracle(mesh, p, parallel=parallel)
    orc.init_potential()
    r, v, cell, pid = bench_population(mesh, target, seed=1000 + seed)
    orc.set_particles(r, v, cell, pid)
    orc.deposit()
    orc.poisson_solve()
    t0 = time.perf_counter()
    orc.step(steps)
    dt = time.perf_counter() - t0
    how = (f"OpenMP build, {cores} threads" if parallel else "serial build, one thread")
    return {"value": round(steps / dt, 5), "unit": "PIC cycles/s", "cores": cores,
            "kind": "oracle",
            "sample": (f"{steps} full PIC steps of the {workload} workload (FP64 oracle, {how}), "
                       f"from the seeded synthetic population of {target} SPs that the GPU arm "
                       f"starts from (deposited and solved first); mesh build and the initial "
                       f"solves untimed"),
            "seconds": round(dt, 2), "host": host_cpu()}


def reference_arm(args, rank, world):
    """The reference arm: the oracle on all host cores (rank 0 only)."""
    if rank != 0:
        return
    steps = max(1, min(args.steps, 30))
    cb = run_oracle(args.workload, steps, parallel=True)
    line = {"metric": METRIC, "value": cb["value"], "unit": cb["unit"], "n_gpus": args.gpus,
            "steps": steps, "warmup": 0, "ms_per_step": round(1e3 / cb["value"], 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "ref": "CPU oracle (plain FP64 C, OpenMP)"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": cb["unit"], "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


PRECONDITIONERS = {0: "Jacobi / whole-matrix Chebyshev", 1: "block-local Chebyshev",
                   2: "block-local Chebyshev + coarse correction",
                   3: "Chebyshev + coarse correction over the solver blocks",
                   4: "multigrid V-cycle"}


FP64_FLOPS_PER_CROSSING = 21   # r - x0 (3), three rows of J^-1 (9 mul + 6 add), lambda_0 (3)
FP64_FLOPS_PER_SP = 20         # kick and drift (12), deposit weights and remainder (8)
_FP64_RATE = []


def fp64_walk_roofline(r):
    """Roofline of the FP64 fused particle kernel against the measured FP64
    FMA rate (pic_measure_fp64_rate; the survey asks for the FP64 ALU rate to
    be measured, since it may bound the FP64 form on this part): its FP64
    flops (per face crossing and per SP, counted from the step statistics of
    the profiled pass) over its event time."""
    from paper_1906_08125_gb300 import picfem
    if not _FP64_RATE:
        _FP64_RATE.append(picfem.measure_fp64_rate())
    rate = _FP64_RATE[0]
    n, ms = r["prof"]["step_fused"]
    st, prev = r["prof_stats"], r["prof_prev_alive"]
    flops = sum(FP64_FLOPS_PER_CROSSING * int(row["crossings"])
                + FP64_FLOPS_PER_SP * (int(pa) + int(row["injected"]))
                for pa, row in zip(prev, st))
    ach = flops / (ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "step_fused", "achieved": round(ach, 4),
            "peak": round(rate, 4), "unit": "TFLOP/s", "frac": round(ach / rate, 4),
            "peak_source": "measured: pic_measure_fp64_rate (independent FP64 FMA chains, 2 flops each)",
            "flops_model": f"{FP64_FLOPS_PER_CROSSING} per face crossing + {FP64_FLOPS_PER_SP} per SP",
            "note": ("the FP64 walk issues its multiplies and adds separately (no contraction, "
                     "bit-exact with the oracle), so its own arithmetic ceiling is half the FMA rate")}


def arm_summary(r, world):
    """Throughput of a comparison arm from its timed (production) steps."""
    st = r["stats"]
    tun = r.get("tuning") or {}
    pre = ("Jacobi" if r["params"].get("pcg_cheb_degree", 0) < 2 and tun.get("pcg_cheb_local") != 4
           else PRECONDITIONERS.get(tun.get("pcg_cheb_local"), "?"))
    return {"value": round(world * len(r["step_ms"]) / (r["total_ms"] * 1e-3), 3),
            "unit": METRIC, "ms_per_step": round(r["total_ms"] / len(r["step_ms"]), 3),
            "pushes_per_s": round(r["pushes"] / (r["total_ms"] * 1e-3), 1),
            "pcg_iters_mean": round(float(st["pcg_iters"].mean()), 1),
            "preconditioner": pre, "steps": len(r["step_ms"])}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    fp64 = args.precision == "fp64"
    K = args.steps
    res = run_gpu(args, rank, world, args.precision, K, max(3, args.warmup),
                  prof_steps=max(5, min(K, 20)))
    roof, kernels = roofline(res, fp64)
    value = world * K / (res["total_ms"] * 1e-3)
    push_rate = res["pushes"] / (res["total_ms"] * 1e-3)
    e2e = run_e2e(res, args.e2e_steps)
    st = res["stats"]
    cfg = {"workload": args.workload, "tets": res["info"]["n_tets"],
           "nodes": res["info"]["n_nodes"], "free_dofs": res["info"]["n_free"],
           "nnz": res["info"]["nnz"], "emitting_faces": res["info"]["n_faces"],
           "sp_in_flight_mean": int(st["alive"].mean()), "target_sp": int(res["n0"]),
           "dt_fs": 4.0, "precision": args.precision, "pcg_rtol": res["params"]["pcg_rtol"],
           "pcg_variant": args.pcg_variant if args.precision == "fp32_ir" else "standard",
           "l2": "flushed before every timed step (256 MB write)",
           "timed_path": ("CUDA graph replays, no per-kernel events" if res["graph"] == 1
                          else "direct launches"),
           "kernel_split": f"a second pass of {len(res['prof_stats'])} steps with per-kernel "
                           f"CUDA events, right after the timed steps",
           "parallelism": f"replicas x{world}"}
    cross = float(st["crossings"].sum())
    tun = res.get("tuning") or {}
    cfg["preconditioner"] = PRECONDITIONERS.get(tun.get("pcg_cheb_local"), "?")
    extra = {"pushes_per_s": round(push_rate, 1),
             "pcg_iters_mean": round(float(st["pcg_iters"].mean()), 1),
             "pcg_outer_mean": round(float(st["pcg_outer"].mean()), 2),
             "crossings_per_sp": round(cross / max(1, res["pushes"]), 1),
             "walk_lane_slots_per_crossing": round(32.0 * float(st["walk_warp_iters"].sum())
                                                   / max(1.0, cross), 3),
             "kernels": kernels}
    pcg_ms_step = kernels.get("pcg", {}).get("ms_total", 0.0) / max(1, len(res["prof_stats"]))
    extra["pcg_ms_per_step"] = round(pcg_ms_step, 4)
    launches, clocks = res["launches"], res["clocks"]
    res["ctx"].close()
    del res
    compare = {}
    if not args.no_fp64_compare and not fp64:
        for form in ("fp64", "fp64_twolevel"):
            r = run_gpu(args, rank, world, form, max(5, K // 3), max(3, args.warmup),
                        prof_steps=5)
            compare[form] = arm_summary(r, world)
            compare[form]["pcg_ms_per_step"] = round(r["prof"]["pcg"][1] / r["prof"]["pcg"][0], 4)
            compare[form]["roofline_step_fused"] = fp64_walk_roofline(r)
            r["ctx"].close()
            del r
        for form, c in compare.items():
            c["fp32_ir_speedup"] = round(value / world / c["value"], 3)
            c["fp32_ir_solver_speedup"] = round(c["pcg_ms_per_step"] / max(pcg_ms_step, 1e-9), 3)
    ens = None
    if rank == 0 and world == 1 and not args.no_ensemble:
        ens = run_ensemble(args.ensemble, steps=10, warmup=10)
    adj = None
    if rank == 0 and world == 1 and args.adjoint_steps > 0:
        adj = run_adjoint_bench(args.workload, args.adjoint_steps, args.adjoint_ckpt)
    large = None
    if rank == 0 and world == 1 and not args.no_large:
        large = run_large("tip_8m", steps=args.large_steps, warmup=5)
    diode = None
    if rank == 0 and world == 1 and not args.no_diode:
        from paper_1906_08125_gb300 import diode as D
        from paper_1906_08125_gb300 import picfem as PF
        t0 = time.perf_counter()
        diode = D.iv_sweep(PF)
        diode["wall_s"] = round(time.perf_counter() - t0, 1)
        diode["paper_rms"] = 0.019
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_oracle(args.workload, args.cpu_steps)
        cpu["all_cores"] = run_oracle(args.workload, args.cpu_steps, parallel=True)
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "PIC cycles/s",
                "n_gpus": world, "steps": K, "warmup": max(3, args.warmup),
                "ms_per_step": round(world * 1e3 / value, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if not fp64 else "f64", "data": "synthetic",
                "config": cfg, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks,
                "fp64_plain": compare.get("fp64"), "fp64_twolevel": compare.get("fp64_twolevel"),
                "ensemble": ens, "adjoint": adj, "diode_iv": diode, "tip_8m": large, **extra}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
