"""Run a named workload for a few eager steps and exit: the target of a
profiler capture (few launches before the captured one, nothing else
running).

    python -m paper_1003_4548_gb300.profile_case --workload canyon_er_full --steps 4

Seeds the workload's ensemble, estimates its statistics, sets the chosen
form's solve schedule (lagged FE solve under the coarse residual check) and
advances `steps` steps on the default stream, then synchronises.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="canyon_er_full")
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--precision", default=None, help="state/reduction precision (default: the chosen form's)")
    ap.add_argument("--lag-tol", type=float, default=None, help="default: the workload's lag_tol")
    a = ap.parse_args(argv)

    import torch

    from canyon_inputs.configs import WORKLOADS, build_mesh, cfl_dt
    from paper_1003_4548_gb300 import Canyon, canyon_params

    cfg = WORKLOADS[a.workload]
    prec = a.precision or cfg.get("chosen_precision", cfg["precision"])
    mesh = build_mesh(cfg)
    dt = cfl_dt(mesh, cfl=cfg["cfl"], k0=cfg["k0"])
    torch.cuda.set_device(0)
    lagged = cfg["wall_model"] == "er"
    extra = {"cg_tol": cfg["lag_cg_tol"]} if lagged and cfg.get("lag_cg_tol") else {}
    p = canyon_params(mesh, wall_model=cfg["wall_model"], precision=prec, C0=cfg["C0"], bins=cfg["bins"],
                      seed=cfg["seed"], k0=cfg["k0"], **extra)
    g = Canyon(p, mesh, stream=torch.cuda.current_stream().cuda_stream)
    g.seed_particles(cfg["per_element"])
    g.estimate_stats()
    if lagged:
        g.set_surrogate(5, None, None, a.lag_tol if a.lag_tol is not None else cfg.get("lag_tol", 0.03))
    g.step(dt, a.steps)
    g.sync()
    print(f"{a.workload}: {g.num_particles} particles, {a.steps} steps, {prec}")
    g.close()


if __name__ == "__main__":
    main()
