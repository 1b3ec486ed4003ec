"""Derive the superparticle weight w_sp of a workload with the CPU oracle.

TEST/INPUT INFRASTRUCTURE: calls only the oracle and the seeded input
generators.  The paper leaves w_sp to each simulation (Sec. II.B: chosen for a
smooth charge distribution with a feasible SP count).  In the
space-charge-limited regime the charge in flight is set by the physics, so the
number of SPs in flight scales as 1/w_sp: run the oracle for a few transit
times at a trial weight, measure the SPs in flight, and rescale to the
workload's target count.

    python -m oracle.derive_wsp tip_1m --trial 2.0 --steps 12
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def derive(name: str, trial: float, steps: int, tail: int = 4, verbose: bool = True) -> dict:
    from oracle import oracle as O
    from paper_1906_08125_gb300 import configs as K

    mesh, p, _ = K.workload(name)
    target = K.WORKLOADS[name]["target_sp"]
    p = dict(p, w_sp=trial, pcg_rtol=1e-6, capacity=max(p["capacity"], 4 * target))
    t0 = time.time()
    orc = O.Oracle(mesh, p)
    orc.init_potential()
    alive = []
    for k in range(steps):
        st = orc.step(1)[0]
        alive.append(st.alive)
        if verbose:
            print(f"{name} step {k}: injected {st.injected} alive {st.alive} "
                  f"crossings {st.crossings} pcg {st.pcg_iters} ({time.time() - t0:.0f} s)",
                  file=sys.stderr)
    n_ss = sum(alive[-tail:]) / tail
    w = trial * n_ss / target
    return {"workload": name, "trial_w_sp": trial, "steps": steps, "alive_tail_mean": n_ss,
            "target_sp": target, "w_sp": float(f"{w:.3g}")}


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--trial", type=float, default=1.0)
    ap.add_argument("--steps", type=int, default=12)
    a = ap.parse_args()
    print(json.dumps(derive(a.workload, a.trial, a.steps)))
