#!/usr/bin/env python3
"""Throughput of the per-particle time step of the canyon PDF method on GB300.

One step = the particle kernel (mixing, frequency, velocity, position, walls,
element walk, source), the element sort, the element moments and velocity
bins, the node/derived fields and the elliptic-relaxation FE solve, on the
full wall-resolved canyon (~40k triangles, 256 particles per element, ~10.3M
particles, FP32 particle state, FP64 statistics and CG). Inputs are synthetic
(seeded mesh and particles), resident in HBM, and larger than L2.

Prints one JSON line (rank 0). ``--impl reference`` times the plain FP64 CPU
oracle on the same workload instead (bounded sample per step).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s & HBM roofline %, chosen vs plain form at stated error"
UNIT = "particle-steps/s"


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="canyon_er_full")
    ap.add_argument("--precision", default=None, help="override the workload precision")
    ap.add_argument("--cg-precision", type=int, default=0, help="elliptic CG: 0 FP64, 1 compensated FP32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def reduce_max(x: float, dist, device: str) -> float:
    """Max of x over the ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, particles_per_rank: int, steps: int, seconds: float) -> float:
    """Particle-steps/s of the whole job: every rank advances its own case of
    the same size, timed by the slowest rank."""
    return world * particles_per_rank * steps / seconds


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows, self.p = [], None
        self.idx = gpu_index

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 8 for i in range(4)
                          if r[4 + i].lower() in ("active", "1", "yes")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            return int(vis.split(",")[local_rank])
        except Exception:
            return local_rank
    return local_rank


def kernel_source_hash() -> str:
    h = hashlib.sha1()
    for f in ("k_particle.cu", "pdf_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1003_4548_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def profiled_traffic(workload: str, precision: str):
    """DRAM bytes per particle of the particle kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "particle_kernel_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[f"{workload}:{precision}"]
        if e.get("source_hash") != kernel_source_hash():
            return None
        return float(e["dram_bytes_per_particle"])
    except Exception:
        return None


# ---------------------------------------------------------------------------
# the CPU oracle on the same workload (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
class OracleRun:
    def __init__(self, cfg, mesh, seed):
        from oracle.oracle import Oracle, default_params
        p = default_params(wall_model=0 if cfg["wall_model"] == "wf" else 1, C0=cfg["C0"], seed=seed,
                           wall_offset=mesh["offset"], x0=mesh["L"] / 2, y0=mesh["y_floor"],
                           period=mesh["L"], y_roof=mesh["H"], k0=cfg["k0"], nb1=cfg["bins"][0],
                           nb2=cfg["bins"][1], nb3=cfg["bins"][2], cg_tol=1e-8, cg_maxit=20000)
        self.o = Oracle(p, mesh)
        self.o.seed(cfg["per_element"])
        self.n = cfg["per_element"] * mesh["tri"].shape[0]
        t0 = time.perf_counter()
        self.o.estimate_stats()
        self.t_stats = time.perf_counter() - t0
        import numpy as np
        self.rng = np.random.default_rng(seed)

    def step(self, dt, m):
        """Advance m random particles; return the time of one particle-step
        share: t(m particles) + (m/N) t(full statistics estimate)."""
        idx = self.rng.choice(self.n, m, replace=False).astype("int32")
        idx.sort()
        t0 = time.perf_counter()
        self.o.advance_subset(dt, idx, check=False)
        t = time.perf_counter() - t0
        return t + self.t_stats * m / self.n


def cpu_baseline(cfg, mesh, dt, budget_s=20.0):
    r = OracleRun(cfg, mesh, cfg["seed"])
    m = max(1000, r.n // 50)
    tt, done = 0.0, 0
    t_start = time.perf_counter()
    while time.perf_counter() - t_start < budget_s or done == 0:
        tt += r.step(dt, m)
        done += m
        if done >= r.n:
            break
    return {"value": done / tt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} particle-steps on the full {cfg['name']} ensemble ({r.n} particles): random "
                      f"subsets of {m} advanced, plus their share of one timed full statistics estimate "
                      f"({r.t_stats:.2f} s: moments, bins, nodes, FE CG); single-threaded FP64 C"}


def run_reference(a, cfg, mesh, dt):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    r = OracleRun(cfg, mesh, cfg["seed"])
    m = max(1000, r.n // 200)
    for _ in range(a.warmup):
        r.step(dt, m)
    ts = [r.step(dt, m) for _ in range(a.steps)]
    total = sum(ts)
    value = a.steps * m / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * total / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_block(cfg, mesh, r.n, "fp64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"per step: {m} of {r.n} particles advanced plus m/N of one full "
                                       f"statistics estimate ({r.t_stats:.2f} s)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_block(cfg, mesh, n, precision):
    return {"workload": cfg["name"], "triangles": int(mesh["tri"].shape[0]), "nodes": int(mesh["xy"].shape[0]),
            "particles": int(n), "per_element": cfg["per_element"],
            "wall_model": "elliptic relaxation (P1 FE, FP64 Jacobi-PCG)" if cfg["wall_model"] == "er"
            else "wall functions", "precision": precision, "bins": list(cfg["bins"]),
            "l2": "inputs larger than L2 (particle state > 0.7 GB)"}


def main():
    a = args_()
    from canyon_inputs.configs import WORKLOADS, build_mesh, cfl_dt
    cfg = dict(WORKLOADS[a.workload])
    cfg["name"] = a.workload
    if a.precision:
        cfg["precision"] = a.precision
    mesh = build_mesh(cfg)
    dt = cfl_dt(mesh, cfl=cfg["cfl"], k0=cfg["k0"])
    if a.impl == "reference":
        run_reference(a, cfg, mesh, dt)
        return

    import numpy as np
    import torch
    from paper_1003_4548_gb300 import Canyon, canyon_params, capi

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    # each rank runs its own canyon case (independent problems, no exchange)
    p = canyon_params(mesh, wall_model=cfg["wall_model"], precision=cfg["precision"], C0=cfg["C0"],
                      bins=cfg["bins"], seed=cfg["seed"], k0=cfg["k0"], case_id=rank, cg_precision=a.cg_precision)
    g = Canyon(p, mesh, stream=stream.cuda_stream)
    g.seed_particles(cfg["per_element"])
    g.estimate_stats()
    g.sync()
    n = g.num_particles
    for _ in range(a.warmup):
        g.step(dt, 1)
    g.sync()
    L = capi.lib()

    clocks = Clocks(gpu_index(local))
    clocks.start()
    time.sleep(0.3)
    g.set_timing(True)
    g.reset_timing()
    launches0 = L.pdf_launch_count(g.handle)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        g.step(dt, 1)
    e1.record(stream)
    st = g.sync(check=False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    time.sleep(0.2)
    ck = clocks.stop()
    launches = L.pdf_launch_count(g.handle) - launches0
    kt = {k: g.kernel_time(k) for k in capi.KERNEL}
    g.set_timing(False)
    ms = reduce_max(ms, dist, "cuda")
    value = whole_job_value(world, n, a.steps, ms / 1e3)

    # end to end through the C ABI with host buffers: load the ensemble from
    # pinned host memory, then per step advance and read the element statistics
    e2e = None
    if not a.no_e2e:
        P = {k: g.field(k) for k in ("x", "y", "u", "v", "w", "om", "psi", "id", "elem")}
        pin = {}
        for k, v in P.items():
            t = torch.empty(v.shape, dtype={np.float64: torch.float64, np.uint32: torch.int32,
                                            np.int32: torch.int32}[v.dtype.type], pin_memory=True)
            t.numpy()[...] = v.view(np.int32) if v.dtype == np.uint32 else v
            pin[k] = t
        host = {k: (pin[k].numpy().view(np.uint32) if k == "id" else pin[k].numpy()) for k in pin}
        out = torch.empty((g.nt, 5), dtype=torch.float64, pin_memory=True)
        h2d = sum(v.nbytes for v in host.values())
        d2h = out.numel() * 8
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set_particles(host, step=g.step_index)
        g.estimate_stats()
        for _ in range(a.steps):
            g.step(dt, 1)
            g.field_into("elem_mean", out.data_ptr(), out.numel() * 8, device=False)
        g.sync(check=False)
        te = reduce_max(time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": whole_job_value(world, n, a.steps, te), "unit": UNIT, "h2d_bytes_per_step": h2d / a.steps,
               "d2h_bytes_per_step": d2h}

    ts = 8 if cfg["precision"] == "fp64" else 4
    bytes_per_particle = 14 * ts + 13  # read 7 state + id + elem + bin, write 7 state + elem
    pk_ms, pk_n = kt["particle"]
    peak, peak_kind = measured_peaks()
    achieved = bytes_per_particle * n / (pk_ms / pk_n / 1e3) / 1e9 if pk_n else None
    traffic_pp = profiled_traffic(a.workload, cfg["precision"])
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None,
            "traffic": traffic_pp * n if traffic_pp else None,
            "kernel": "k_step (per-particle step)", "bytes_per_particle": bytes_per_particle,
            "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
            else "fallback 6.8 TB/s"}
    kernels = {k: {"ms_per_step": v[0] / a.steps, "launches": v[1]} for k, v in kt.items()}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if cfg["precision"] != "fp64" else "f64",
            "data": "synthetic", "config": config_block(cfg, mesh, n, cfg["precision"]),
            "roofline": roof, "e2e": e2e, "gpu_launches": int(launches), "clocks": ck,
            "kernels": kernels, "status": capi.ERRORS.get(st, "ok") if st else "ok",
            "cg_iterations_last": g.cg_iterations}
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, mesh, dt)
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
