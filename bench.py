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
FLT_MIN = 1.1754943508222875e-38  # smallest normal FP32 number


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
    ap.add_argument("--no-surrogate", action="store_true", help="FE solve every step in the timed form")
    ap.add_argument("--chosen", default="lagged", choices=["lagged", "corrected", "surrogate"],
                    help="wp of the timed form: lagged FE under the coarse residual check, the lagged FE plus the "
                         "trained network's change since the last solve, or the trained network alone")
    ap.add_argument("--lag-tol", type=float, default=None,
                    help="coarse residual above which the lagged form solves the FE problem again (default: the "
                         "workload's lag_tol)")
    ap.add_argument("--lag-cg-tol", type=float, default=None,
                    help="relative residual of the lagged form's FE solves (default: the workload's lag_cg_tol)")
    ap.add_argument("--no-forms", action="store_true", help="skip the plain forms and the precision study")
    ap.add_argument("--save-surrogate", default=None, help="write the trained network (npz) here")
    ap.add_argument("--load-surrogate", default=None, help="use this trained network (npz) instead of training")
    ap.add_argument("--sur-epochs", type=int, default=10, help="training epochs of the surrogate")
    ap.add_argument("--pressure", action="store_true",
                    help="add the mean-pressure projection to the timed form (not the published configuration)")
    ap.add_argument("--se-seeds", type=int, default=8,
                    help="independent seeds per form in the standard-error study of the stated error")
    ap.add_argument("--surrogate-mode", type=int, default=1, choices=[1, 3],
                    help="1: network at the nodes; 3: network at every particle inside the particle kernel")
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


KERNEL_SOURCES = {
    "k_step": ("k_particle.cu", "pdf_internal.cuh"),
    "k_moments_w": ("k_stats.cu", "exact_sum.cuh", "pdf_internal.cuh"),
    "k_bins_med": ("k_stats.cu", "exact_sum.cuh", "pdf_internal.cuh"),
    "k_scatter": ("k_sort.cu", "pdf_internal.cuh"),
}


def kernel_source_hash(kernel: str = "k_step") -> str:
    """Hash of the code of a kernel's sources (line comments and blank lines
    left out, so a comment edit does not invalidate a capture)."""
    import re
    h = hashlib.sha1()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1003_4548_gb300", "csrc", f), encoding="utf-8") as fh:
            for line in fh:
                code = re.sub(r"//.*$", "", line).strip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:12]


def profiled_instructions(kernel: str, workload: str, precision: str):
    """Warp instructions of one launch of a kernel (smsp__inst_executed.sum
    from the committed ncu summary), if taken on the current source."""
    path = os.path.join(ROOT, "profiles", "kernel_traffic.json")
    try:
        with open(path) as f:
            e = json.load(f)[f"{kernel}:{workload}:{precision}"]
        if e.get("source_hash") != kernel_source_hash(kernel):
            return None
        return float(e["warp_instructions_per_launch"])
    except Exception:
        return None


def issue_roofline(kernel, ms_per_launch, workload, precision, sm_mhz):
    """A kernel bound by instruction issue rather than by HBM: its warp
    instructions per launch over its event time, against the issue rate of
    one warp instruction per cycle per SM sub-partition (4 per SM) at the SM
    clock seen in the timed region."""
    w = profiled_instructions(kernel, workload, precision)
    if not w or not sm_mhz or not ms_per_launch:
        return None
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 4 * sm_mhz * 1e6
    got = w / (ms_per_launch / 1e3)
    return {"bound": "issue", "warp_instructions_per_launch": w, "achieved_per_s": got, "peak_per_s": peak,
            "frac": got / peak, "peak_source": f"{sms} SMs x 4 schedulers x {sm_mhz:.0f} MHz"}


def profiled_traffic(kernel: str, workload: str, precision: str):
    """DRAM bytes per particle of a kernel from the committed ncu summary, if
    it was taken on the current source of that kernel."""
    path = os.path.join(ROOT, "profiles", "kernel_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[f"{kernel}:{workload}:{precision}"]
        if e.get("source_hash") != kernel_source_hash(kernel):
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
            "data": "synthetic", "config": config_block(cfg, mesh, r.n, "fp64", "plain FP64 CPU oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"per step: {m} of {r.n} particles advanced plus m/N of one full "
                                       f"statistics estimate ({r.t_stats:.2f} s)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_block(cfg, mesh, n, precision, form):
    return {"workload": cfg["name"], "triangles": int(mesh["tri"].shape[0]), "nodes": int(mesh["xy"].shape[0]),
            "particles": int(n), "per_element": cfg["per_element"],
            "wall_model": "elliptic relaxation (P1 FE, FP64 block-Jacobi PCG)" if cfg["wall_model"] == "er"
            else "wall functions", "precision": precision, "bins": list(cfg["bins"]), "form": form,
            "l2": "inputs larger than L2 (particle state > 0.7 GB)"}


# algorithmic bytes per particle of the dominant kernel of each timed class
def algorithmic_bytes(kclass: str, ts: int):
    if kclass == "particle":  # k_step: read 7 state + id + elem + bin, write 7 state + elem
        return 14 * ts + 13, "k_step (per-particle step)"
    if kclass == "moments":   # k_moments_w: read u v w psi omega (12 values per element written)
        return 5 * ts, "k_moments_w (element moments)"
    if kclass == "bins":      # k_bins_med: read u v w psi, write the bin (ids only where values tie)
        return 4 * ts + 1, "k_bins_med (velocity bins and <phi|V>, beside the field chain)"
    if kclass == "sort":      # k_scatter: read and write 7 state + id + elem
        return 2 * (7 * ts + 8), "k_scatter (element re-sort)"
    return None, None


KTRAFFIC = {"particle": "k_step", "moments": "k_moments_w", "bins": "k_bins_med", "sort": "k_scatter"}


def roofline(kclass, kt, n, ts, workload, precision):
    bpp, name = algorithmic_bytes(kclass, ts)
    ms, launches = kt[kclass]
    peak, peak_kind = measured_peaks()
    if bpp is None or not launches:
        return {"bound": "latency", "kernel": kclass, "achieved": None, "peak": peak, "unit": "GB/s", "frac": None,
                "traffic": None, "note": "L2-resident and latency-bound: no HBM roofline applies"}
    achieved = bpp * n / (ms / launches / 1e3) / 1e9
    tpp = profiled_traffic(KTRAFFIC[kclass], workload, precision) if kclass in KTRAFFIC else None
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": tpp * n if tpp else None, "kernel": name, "bytes_per_particle": bpp,
            "ms_per_launch": ms / launches,
            "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs), burst"
            if peak_kind == "measured" else "fallback 6.8 TB/s"}


def fp64_roofline(kt, n, workload):
    """The FP64 form's particle kernel against the GPU's measured FP64 FMA
    rate: FP64 FLOPs per particle (2 per DFMA, 1 per DADD and DMUL, counted
    by ncu on the current source of k_step<double>) times the particles,
    over the kernel's CUDA-event time per launch."""
    from paper_1003_4548_gb300 import capi
    peak = capi.measure_fp64_fma_rate()
    ms, launches = kt["particle"]
    fpp = None
    try:
        with open(os.path.join(ROOT, "profiles", "kernel_traffic.json")) as fh:
            e = json.load(fh)[f"k_step:{workload}:fp64"]
        if e.get("source_hash") == kernel_source_hash("k_step"):
            fpp = float(e["fp64_flops_per_particle"])
    except Exception:
        fpp = None
    out = {"bound": "alu", "kernel": "k_step<double> (per-particle step, FP64 state)", "peak": peak,
           "unit": "TFLOP/s", "peak_source": "measured FP64 FMA rate (pdf_measure_fp64_fma_rate)",
           "ms_per_launch": ms / max(launches, 1), "fp64_flops_per_particle": fpp, "achieved": None, "frac": None}
    if fpp and launches:
        out["achieved"] = fpp * n / (ms / launches / 1e3) / 1e12
        out["frac"] = out["achieved"] / peak
    return out


def cell_stats(g, mesh, nx=12, ny=8):
    """Particle-weighted <U>, <V>, the Reynolds stresses <uu>, <vv>, <ww>,
    <uv>, k, <psi> and the psi variance over an nx x ny grid of cells (element
    means grouped by centroid) for comparing runs."""
    import numpy as np
    cent = mesh["xy"][mesh["tri"]].mean(1)
    cell = (np.clip((cent[:, 0] / mesh["L"] * nx).astype(int), 0, nx - 1) * ny +
            np.clip((cent[:, 1] / mesh["T"] * ny).astype(int), 0, ny - 1))
    n = g.field("elem_n").astype(float)
    M, R, pv = g.field("elem_mean"), g.field("elem_R"), g.field("elem_psivar")
    out = {}
    for name, q in (("U", M[:, 0]), ("V", M[:, 1]), ("uu", R[:, 0]), ("vv", R[:, 1]), ("ww", R[:, 2]),
                    ("uv", R[:, 3]), ("k", 0.5 * (R[:, 0] + R[:, 1] + R[:, 2])), ("psi", M[:, 3]),
                    ("psi_var", pv)):
        w = np.bincount(cell, weights=n, minlength=nx * ny)
        out[name] = np.bincount(cell, weights=n * q, minlength=nx * ny) / np.maximum(w, 1.0)
    return out


def rel_rms(a, b):
    import numpy as np
    return float(np.sqrt(np.mean((a - b) ** 2)) / (np.sqrt(np.mean(b ** 2)) + 1e-300))


class Form:
    """One context of the workload in a given precision, with or without the
    surrogate."""

    def __init__(self, cfg, mesh, stream, *, precision, case_id=0, seed=None, cg_precision=0, sur=None, **extra):
        from paper_1003_4548_gb300 import Canyon, canyon_params
        if sur is not None and sur.get("cg_tol") is not None and "cg_tol" not in extra:
            extra["cg_tol"] = sur["cg_tol"]  # the lagged forms' FE solve tolerance
        p = canyon_params(mesh, wall_model=cfg["wall_model"], precision=precision, C0=cfg["C0"],
                          bins=cfg["bins"], seed=cfg["seed"] if seed is None else seed, k0=cfg["k0"],
                          case_id=case_id, cg_precision=cg_precision, **extra)
        self.g = Canyon(p, mesh, stream=stream.cuda_stream)
        self.g.seed_particles(cfg["per_element"])
        self.g.estimate_stats()
        if sur is not None:
            self.g.set_surrogate(sur.get("mode", 1), sur["params"], sur["norm"], sur["tol"])
        self.stream = stream

    def timed(self, dt, steps, warmup, dist=None, clocks=None):
        import torch
        from paper_1003_4548_gb300 import capi
        g = self.g
        for _ in range(warmup):
            g.step(dt, 1)
        g.sync()
        if clocks:
            clocks.start()
            time.sleep(0.3)
        g.set_timing(True)
        g.reset_timing()
        L = capi.lib()
        launches0 = L.pdf_launch_count(g.handle)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        for _ in range(steps):
            g.step(dt, 1)
        e1.record(self.stream)
        st = g.sync(check=False)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = e0.elapsed_time(e1)
        ck = None
        if clocks:
            time.sleep(0.2)
            ck = clocks.stop()
        kt = {k: g.kernel_time(k) for k in capi.KERNEL}
        g.set_timing(False)
        return {"ms": ms, "kt": kt, "launches": L.pdf_launch_count(g.handle) - launches0, "status": st,
                "clocks": ck, "cg_iterations_last": g.cg_iterations,
                "pressure_iterations_last": g.pressure_iterations}

    def timed_graph(self, dt, steps, warmup, dist=None, clocks=None):
        """The same steps replayed from one CUDA graph of a step pair (the
        public pdf_batch_* calls with this one context): no kernel-class events
        inside, so launch gaps are the graph's. Returns ms for the (even) step
        count, the kernels launched and the clocks."""
        import torch
        from paper_1003_4548_gb300 import capi
        g = self.g
        gs = torch.cuda.Stream(priority=-1)  # the graph's launch stream, distinct from the context's
        for _ in range(max(0, warmup - 2)):
            g.step(dt, 1)
        g.sync()
        b = capi.Batch([g], [dt], gs.cuda_stream)
        b.step(2)
        b.sync()
        steps += steps & 1
        if clocks:
            clocks.start()
            time.sleep(0.3)
        L = capi.lib()
        launches0 = L.pdf_launch_count(g.handle)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(gs)
        b.step(steps)
        e1.record(gs)
        torch.cuda.synchronize()
        status = "ok"
        try:
            b.sync()
        except capi.PdfError as err:
            status = str(err)
        if dist:
            dist.barrier()
        ms = e0.elapsed_time(e1)
        ck = None
        if clocks:
            time.sleep(0.2)
            ck = clocks.stop()
        b.close()
        return {"ms": ms, "steps": steps, "launches": L.pdf_launch_count(g.handle) - launches0, "clocks": ck,
                "status": status}

    def close(self):
        self.g.close()


def prepare_surrogate(cfg, mesh, dt, seed=0, harvest_meshes=None, ratios=(0.5, 0.75, 1.0, 1.5, 2.0), epochs=10):
    """Harvest FE runs at W/H = 0.5 .. 2 (this workload's mesh recipe, or the
    given meshes), train the network with the library's kernels, and
    calibrate the check on a held-out run of this workload: threshold = 1.5 x
    the largest coarse residual seen there."""
    from canyon_inputs.configs import cfl_dt
    from canyon_inputs.mesh import canyon_mesh
    from paper_1003_4548_gb300 import surrogate
    t0 = time.perf_counter()
    meshes = harvest_meshes
    if meshes is None:
        meshes = []
        for i, W in enumerate(ratios):
            m = dict(cfg["mesh"])
            m["W"], m["seed"] = W, 10 + i
            meshes.append(canyon_mesh(**m))
    # the harvest and the calibration span the length of a production run (the
    # C2 recipe's 500 steps): the developed flow differs from the early
    # transient, and a network that never saw it fails the check there
    X, T, counts = surrogate.harvest(meshes, steps=500, every=10, per_element=cfg["per_element"],
                                     dt_of=lambda m: cfl_dt(m, cfl=cfg["cfl"], k0=cfg["k0"]), C0=cfg["C0"],
                                     seed=seed + 1000)
    t1 = time.perf_counter()
    params, norm, hist = surrogate.train(X, T, epochs=epochs, batch=4096, lr=2e-3, lr_final=1e-4, seed=seed)
    t2 = time.perf_counter()
    res = surrogate.calibrate(params, norm, mesh, steps=500, every=10, per_element=cfg["per_element"], dt=dt,
                              seed=seed + 99, C0=cfg["C0"])
    tol = 1.5 * max(r[0] for r in res)
    info = {"samples": int(X.shape[0]), "harvest_and_calibration_steps": 500, "aspect_ratios": [round(float(m["W"]), 3) for m in meshes],
            "harvest_triangles": [int(m["tri"].shape[0]) for m in meshes], "epochs": epochs,
            "final_loss_standardised": hist[-1][1], "harvest_s": t1 - t0, "train_s": t2 - t1,
            "calibration_coarse_residual_max": max(r[0] for r in res), "residual_tol": tol,
            "check": "coarse FE residual (aggregates of 128 Morton-ordered nodes) <= residual_tol"}
    del X, T
    return {"params": params, "norm": norm, "tol": tol}, info


def surrogate_error(form, mesh):
    """wp of the network against the FE solve on the same statistics, at the
    end of a run (relative L2 over the nodes, per component)."""
    import numpy as np
    g = form.g
    solves, falls, res = g.surrogate_stats()
    g.set_surrogate(0)
    g.estimate_stats()
    wfe = g.field("node_wp")
    return {"solves": solves, "fallbacks": falls, "last_residual_coarse": res[0], "last_residual_fine": res[1],
            "wp_rel_l2_vs_fe": [round(float(x), 4) for x in
                                np.linalg.norm(form.last_wp - wfe, axis=0) / np.linalg.norm(wfe, axis=0)]}


def run_batch(a, cfg, emit=True):
    """Many independent cases in one CUDA graph (pdf_batch_*): each case its own
    mesh, particle count, seed and source, autotuned launch shapes, the chosen
    form (FP32 state, compensated-FP32 reductions, surrogate wp with the FE
    solve as checked fallback). value = all cases' particle-steps per second."""
    import torch
    from canyon_inputs.configs import WORKLOADS, batch_cases, build_mesh, cfl_dt
    from canyon_inputs.mesh import canyon_mesh
    from paper_1003_4548_gb300 import Canyon, canyon_params, capi
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prec = a.precision or cfg["chosen_precision"]
    cases = batch_cases(cfg)
    meshes = [canyon_mesh(**c["mesh"]) for c in cases]
    # wp: the lagged FE solve under the coarse check (the chosen form), or the
    # network trained on held-out cases of the same family (another draw of
    # the batch recipe: W/H 0.5 .. 3, spacing 0.017 .. 0.1), calibrated on the
    # wall-resolved W/H = 1 canyon
    sur, sur_info = None, {"form": "lagged FE", "residual_tol": a.lag_tol, "cg_tol": a.lag_cg_tol}
    if a.chosen == "surrogate":
        ref = dict(WORKLOADS["canyon_er_full"])
        ref["name"] = "canyon_er_full"
        ref_mesh = build_mesh(ref)
        held = batch_cases(dict(cfg, seed=cfg["seed"] + 1))[:8]
        sur, sur_info = prepare_surrogate(ref, ref_mesh, cfl_dt(ref_mesh, cfl=ref["cfl"], k0=ref["k0"]),
                                          harvest_meshes=[canyon_mesh(**c["mesh"]) for c in held])
    # torch hands out pooled streams (32 per priority): the cases take the
    # low-priority pool, the batch stream comes from the high-priority one
    streams = [torch.cuda.Stream() for _ in cases]
    bstream = torch.cuda.Stream(priority=-1)
    assert len({s_.cuda_stream for s_ in streams + [bstream]}) == len(cases) + 1, "streams must be distinct"
    ctxs, dts, tunings, tols = [], [], [], []
    t0 = time.perf_counter()
    for c, m, st in zip(cases, meshes, streams):
        p = canyon_params(m, wall_model="er", precision=prec, C0=cfg["C0"], bins=cfg["bins"], seed=c["seed"],
                          k0=cfg["k0"], case_id=rank, **({"cg_tol": a.lag_cg_tol} if sur is None else {}))
        g = Canyon(p, m, stream=st.cuda_stream)
        g.seed_particles(c["per_element"])
        g.estimate_stats()
        dt = cfl_dt(m, cfl=cfg["cfl"], k0=cfg["k0"])
        if sur is not None:
            # the check's threshold per case: 1.5 x the largest coarse residual
            # of the network's wp over this case's first steps (the warm-up)
            g.set_surrogate(2, sur["params"], sur["norm"], 0.0)
            res = []
            for _ in range(3):
                g.step(dt, 2)
                res.append(g.surrogate_stats()[2][0])
            tols.append(1.5 * max(res))
            g.set_surrogate(1, sur["params"], sur["norm"], tols[-1])
        else:
            tols.append(a.lag_tol)
            g.set_surrogate(5, None, None, a.lag_tol)
        tunings.append(g.autotune(dt, 2))
        ctxs.append(g)
        dts.append(dt)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    n_total = sum(g.num_particles for g in ctxs)
    b = capi.Batch(ctxs, dts, bstream.cuda_stream)
    steps = a.steps + (a.steps & 1)
    b.step(2 * max(2, (a.warmup + 1) // 2))
    b.sync()
    L = capi.lib()
    launches0 = sum(L.pdf_launch_count(g.handle) for g in ctxs)
    sur0 = [g.surrogate_stats() for g in ctxs]
    clocks = Clocks(gpu_index(local))
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(bstream)
    b.step(steps)
    e1.record(bstream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    time.sleep(0.2)
    ck = clocks.stop()
    try:
        b.sync()
        status = "ok"
    except capi.PdfError as err:
        status = str(err)
    ms = reduce_max(ms, dist, "cuda")
    value = whole_job_value(world, n_total, steps, ms / 1e3)
    launches = sum(L.pdf_launch_count(g.handle) for g in ctxs) - launches0
    sur1 = [g.surrogate_stats() for g in ctxs]
    solves = sum(x[0] - y[0] for x, y in zip(sur1, sur0))
    falls = sum(x[1] - y[1] for x, y in zip(sur1, sur0))
    # the same cases launched context by context on their streams, without the graph
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k = min(steps, 10)
    f0.record(bstream)
    for s_ in streams:
        s_.wait_event(f0)
    for _ in range(k):
        for g, dt in zip(ctxs, dts):
            g.step(dt, 1)
    for s_ in streams:
        bstream.wait_stream(s_)
    f1.record(bstream)
    torch.cuda.synchronize()
    no_graph = n_total * k / (f0.elapsed_time(f1) / 1e3)
    b.close()
    tri = [int(m["tri"].shape[0]) for m in meshes]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": a.warmup,
            "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg["name"], "cases": len(cases), "particles": int(n_total),
                       "triangles_min_max_total": [min(tri), max(tri), sum(tri)],
                       "per_element_min_max": [min(c["per_element"] for c in cases),
                                               max(c["per_element"] for c in cases)],
                       "W_over_H_min_max": [round(min(c["mesh"]["W"] for c in cases), 3),
                                            round(max(c["mesh"]["W"] for c in cases), 3)],
                       "precision": prec, "form": "one CUDA graph per step pair over all cases; chosen form (" +
                       ("trained network" if sur is not None else "lagged FE") + " wp under the coarse check)",
                       "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "kernel": "whole step, all cases (69 B per particle-step algorithmic)",
                         "achieved": 69 * n_total * steps / (ms / 1e3) / 1e9, "peak": measured_peaks()[0],
                         "unit": "GB/s", "frac": 69 * n_total * steps / (ms / 1e3) / 1e9 / measured_peaks()[0],
                         "traffic": None},
            "gpu_launches": int(launches), "clocks": ck, "status": status,
            "streams_without_graph": {"value": no_graph, "steps": k},
            "autotuned": {"step_blocks_per_sm": sorted({t["step_blocks_per_sm"] for t in tunings}),
                          "scatter_threads": sorted({t["scatter_threads"] for t in tunings}),
                          "cg_rows_per_block": sorted({t["cg_rows_per_block"] for t in tunings}),
                          "bins_blocks_per_sm": sorted({t["bins_blocks_per_sm"] for t in tunings})},
            "wp": dict(sur_info, checked_steps=solves, fe_solves=falls,
                       residual_tol_per_case_min_max=[min(tols), max(tols)],
                       check_calibration=("per case: 1.5 x the largest coarse residual over its first 6 steps "
                                          "(warm-up)") if sur is not None else "the same tolerance for every case"),
            "setup_s": t_setup,
            "e2e": None}
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    for g in ctxs:
        g.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return line


def batch_summary(a):
    """The 32-case batch (canyon_batch32) measured inside the main run: 20
    steps through its graph after 4 warm-up steps, the chosen form."""
    import copy
    from canyon_inputs.configs import WORKLOADS
    b = copy.copy(a)
    b.steps, b.warmup, b.precision, b.chosen = 20, 4, None, "lagged"
    cfg = dict(WORKLOADS["canyon_batch32"])
    cfg["name"] = "canyon_batch32"
    t0 = time.perf_counter()
    line = run_batch(b, cfg, emit=False)
    keep = ("value", "unit", "steps", "warmup", "ms_per_step", "config", "roofline", "gpu_launches", "clocks",
            "status", "streams_without_graph", "autotuned", "wp", "setup_s")
    out = {k: line[k] for k in keep}
    out["wall_s"] = round(time.perf_counter() - t0, 1)
    return out


def small_case_summary(stream):
    """The small wall-function canyon (canyon_wf_small) as its recipe runs
    it: FP64, 100 steps at CFL 0.5, Philox seed 0; the oracle on a bounded
    sample of the same ensemble beside it."""
    from canyon_inputs.configs import WORKLOADS, build_mesh, cfl_dt
    cfg = dict(WORKLOADS["canyon_wf_small"])
    cfg["name"] = "canyon_wf_small"
    mesh = build_mesh(cfg)
    dt = cfl_dt(mesh, cfl=cfg["cfl"], k0=cfg["k0"])
    f = Form(cfg, mesh, stream, precision=cfg["precision"])
    n = f.g.num_particles
    rr = f.timed(dt, cfg["steps"], 3)
    out = {"value": n * cfg["steps"] / (rr["ms"] / 1e3), "unit": UNIT, "steps": cfg["steps"], "warmup": 3,
           "ms_per_step": rr["ms"] / cfg["steps"], "precision": cfg["precision"], "status": rr["status"],
           "config": {"workload": cfg["name"], "triangles": int(mesh["tri"].shape[0]), "particles": int(n),
                      "per_element": cfg["per_element"], "wall_model": "wall functions (SLM)", "C0": cfg["C0"],
                      "bins": list(cfg["bins"])},
           "kernels_ms_per_step": {q: v[0] / cfg["steps"] for q, v in rr["kt"].items()}}
    f.close()
    out["cpu_baseline"] = cpu_baseline(cfg, mesh, dt, budget_s=5.0)
    return out


def main():
    a = args_()
    from canyon_inputs.configs import WORKLOADS, build_mesh, cfl_dt
    cfg = dict(WORKLOADS[a.workload])
    cfg["name"] = a.workload
    # the lagged FE form's schedule: the workload's check and solve tolerances
    if a.lag_tol is None:
        a.lag_tol = cfg.get("lag_tol", 0.03)
    if a.lag_cg_tol is None:
        a.lag_cg_tol = cfg.get("lag_cg_tol")
    if cfg.get("kind") == "batch":
        if a.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batch workload has no oracle arm"}))
            return
        run_batch(a, cfg)
        return
    plain_precision = cfg["precision"]
    if a.precision:
        cfg["precision"] = a.precision
    elif a.impl != "reference" and not a.no_surrogate and cfg.get("chosen_precision"):
        cfg["precision"] = cfg["chosen_precision"]
    mesh = build_mesh(cfg)
    dt = cfl_dt(mesh, cfl=cfg["cfl"], k0=cfg["k0"])
    if a.impl == "reference":
        run_reference(a, cfg, mesh, dt)
        return

    import numpy as np
    import torch

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    # wp of the timed form: the lagged FE solve (the previous solution kept
    # while its coarse FE residual under the current statistics stays below
    # --lag-tol) or the trained network under the same check. The network is
    # trained whenever it is timed or measured beside the chosen form.
    er = cfg["wall_model"] == "er" and not a.no_surrogate
    use_net = er and (a.chosen in ("surrogate", "corrected") or not a.no_forms)
    sur, sur_info = None, None
    if use_net and a.load_surrogate:
        z = np.load(a.load_surrogate)
        sur = {"params": z["params"], "norm": z["norm"], "tol": float(z["tol"])}
        sur_info = {"loaded_from": os.path.basename(a.load_surrogate), "residual_tol": sur["tol"]}
    elif use_net:
        sur, sur_info = prepare_surrogate(cfg, mesh, dt, epochs=a.sur_epochs)
    if sur is not None:
        sur["mode"] = a.surrogate_mode
    if sur is not None and a.save_surrogate:
        np.savez(a.save_surrogate, params=sur["params"], norm=sur["norm"], tol=sur["tol"])
    lagged = {"mode": 5, "params": None, "norm": None, "tol": a.lag_tol, "cg_tol": a.lag_cg_tol}
    corrected = dict(sur, mode=6, tol=a.lag_tol, cg_tol=a.lag_cg_tol) if sur is not None else None
    chosen_wp = ({"surrogate": sur, "corrected": corrected}.get(a.chosen, lagged)) if er else None
    prec = cfg["precision"]
    red = {"fp64": "FP64", "fp32": "FP64-exact", "fp32_kahan": "compensated FP32"}[prec]
    form_name = f"{prec} particle state, {red} statistics, " + (
        "FE solve every step" if chosen_wp is None else
        "surrogate wp with the FE solve as checked fallback" if chosen_wp is sur else
        (f"lagged FE solve plus the trained network's change since the last solve, kept while its coarse FE "
         f"residual stays below {a.lag_tol}") if chosen_wp is corrected else
        f"lagged FE solve: the previous wp kept while its coarse FE residual stays below {a.lag_tol}")
    # each rank runs its own canyon case (independent problems, no exchange)
    extra = {"pressure": 1} if a.pressure else {}
    if a.pressure:
        form_name += ", mean-pressure projection every step"
    # The timed region replays one CUDA graph of a step pair (pdf_batch_* with
    # this context alone). The kernel-class durations behind the rooflines come
    # from CUDA events around every class in an eager pass of the same steps
    # on a second context of the same seed (events cannot sit inside the graph).
    chosen = Form(cfg, mesh, stream, precision=prec, case_id=rank, cg_precision=a.cg_precision, sur=chosen_wp,
                  **extra)
    n = chosen.g.num_particles
    graph_form = Form(cfg, mesh, torch.cuda.Stream(), precision=prec, case_id=rank, cg_precision=a.cg_precision,
                      sur=chosen_wp, **extra)  # a graph's contexts need their own (non-default) streams
    rg = graph_form.timed_graph(dt, a.steps, a.warmup, dist, Clocks(gpu_index(local)))
    r = chosen.timed(dt, a.steps, a.warmup, dist)
    steps_timed = rg["steps"]
    ms = reduce_max(rg["ms"], dist, "cuda")
    value = whole_job_value(world, n, steps_timed, ms / 1e3)
    eager_ms = reduce_max(r["ms"], dist, "cuda")
    kt = r["kt"]
    ts = 8 if prec == "fp64" else 4
    dominant = max((k for k in kt if kt[k][1]), key=lambda k: kt[k][0])
    roof = roofline(dominant, kt, n, ts, a.workload, prec)
    rooflines = {k: roofline(k, kt, n, ts, a.workload, prec) for k in ("particle", "moments", "bins", "sort")
                 if k in kt and kt[k][1]}
    kernels = {k: {"ms_per_step": v[0] / a.steps, "launches": v[1]} for k, v in kt.items()}
    stated = {}
    if chosen_wp is not None:
        solves, falls, _ = chosen.g.surrogate_stats()
        stated["wp_fe_solves_in_timed_steps"] = {"steps": int(solves), "fe_solves": int(falls)}
    if chosen_wp is not None and chosen_wp is sur:
        chosen.last_wp = chosen.g.field("node_wp")
        stated["surrogate"] = surrogate_error(chosen, mesh)
        chosen.g.set_surrogate(sur["mode"], sur["params"], sur["norm"], sur["tol"])

    # end to end through the C ABI with host buffers, on the graph context:
    # load the ensemble from pinned host memory and estimate its statistics,
    # then replay the step-pair graph, which copies each step's element means
    # into one of two device buffers (pdf_batch_create_out); after every
    # replay the two steps' means go to their own pinned host buffers
    # (asynchronous copies on the graph's stream, so the host keeps queueing
    # replays). One sync at the end; then the host checks the copied results
    # (finite, distinct per step, the last equal to the context's own field). The graph is captured inside the timed region, after the
    # upload: loading an ensemble re-sorts it, which moves the state between
    # the context's two buffers, and a graph holds the buffers it was captured
    # with.
    e2e = None
    if not a.no_e2e:
        from paper_1003_4548_gb300 import capi
        g = graph_form.g
        e2e_steps = a.steps + (a.steps & 1)
        P = {k: g.field(k) for k in ("x", "y", "u", "v", "w", "om", "psi", "id", "elem")}
        pin = {}
        for k, v in P.items():
            t = torch.empty(v.shape, dtype={np.float64: torch.float64, np.uint32: torch.int32,
                                            np.int32: torch.int32}[v.dtype.type], pin_memory=True)
            t.numpy()[...] = v.view(np.int32) if v.dtype == np.uint32 else v
            pin[k] = t
        host = {k: (pin[k].numpy().view(np.uint32) if k == "id" else pin[k].numpy()) for k in pin}
        out = torch.empty((e2e_steps, g.nt, 5), dtype=torch.float64, pin_memory=True)
        h2d = sum(v.nbytes for v in host.values())
        d2h = g.nt * 5 * 8
        snaps = [torch.empty((g.nt, 5), dtype=torch.float64, device="cuda") for _ in range(2)]
        gs = torch.cuda.Stream(priority=-1)
        ready = torch.cuda.Event()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set_particles(host, step=g.step_index)
        g.estimate_stats()
        eb = capi.Batch([g], [dt], gs.cuda_stream, outputs=("elem_mean", [t.data_ptr() for t in snaps], [d2h]))
        ready.record(graph_form.stream)
        gs.wait_event(ready)
        for j in range(e2e_steps // 2):
            eb.step(2)
            with torch.cuda.stream(gs):
                out[2 * j].copy_(snaps[0], non_blocking=True)
                out[2 * j + 1].copy_(snaps[1], non_blocking=True)
        eb.sync()
        te = reduce_max(time.perf_counter() - t0, dist, "cuda")
        eb.close()
        # after the timed region: the last copied result is the context's own
        # final state bit for bit, and every step's result differs from the
        # step before (a stale buffer or a wrong one wired into the graph shows)
        res = out.numpy()
        results_finite = bool(np.isfinite(res).all())
        last_equals_context = bool(np.array_equal(res[-1], g.field("elem_mean")))
        steps_distinct = bool(all(not np.array_equal(res[k], res[k - 1]) for k in range(1, e2e_steps)))
        e2e = {"value": whole_job_value(world, n, e2e_steps, te), "unit": UNIT, "h2d_bytes_per_step": h2d / e2e_steps,
               "d2h_bytes_per_step": d2h, "results_finite": results_finite,
               "last_result_equals_context": last_equals_context, "results_distinct_per_step": steps_distinct,
               "steps": e2e_steps,
               "path": "pdf_set_particles + pdf_estimate_stats from pinned host buffers, then the step-pair graph "
                       "(pdf_batch_create_out) with each step's element means copied to pinned host memory"}
    graph_form.close()
    chosen.close()

    # a whole production run of the chosen form from its seeded start (the C2
    # recipe's 500 steps): the per-element counts spread and the flow leaves
    # the early transient, so the rate and the surrogate's fallbacks over the
    # full run are stated beside the 100-step window above
    def sustained_run(wp):
        f = Form(cfg, mesh, stream, precision=prec, sur=wp, **extra)
        s0 = f.g.surrogate_stats()
        rr = f.timed(dt, 500, 0)
        s1 = f.g.surrogate_stats()
        out = {"steps": 500, "value": f.g.num_particles * 500 / (rr["ms"] / 1e3), "ms_per_step": rr["ms"] / 500,
               "checked_steps": s1[0] - s0[0], "fe_solves": s1[1] - s0[1],
               "kernels_ms_per_step": {q: v[0] / 500 for q, v in rr["kt"].items()}}
        f.close()
        return out

    sustained = None
    sustained_other = {}
    if not a.no_forms and rank == 0 and chosen_wp is not None:
        sustained = sustained_run(chosen_wp)
        # the other checked forms over the same 500 steps: FE solves and rate
        for nm, wp in (("lagged_fe", lagged), ("lagged_fe_with_network_correction", corrected)):
            if wp is not None and wp is not chosen_wp:
                sustained_other[nm] = sustained_run(wp)

    # the plain forms on the same workload (fewer steps), and the stated error
    forms = {}
    if not a.no_forms and rank == 0:
        k = max(10, a.steps // 5)
        for name, fp, cgp in (("plain_fp64_fe", "fp64", 0), (f"{plain_precision}_fe", plain_precision, 0)):
            f = Form(cfg, mesh, stream, precision=fp, cg_precision=cgp)
            rr = f.timed(dt, k, 3)
            forms[name] = {"value": f.g.num_particles * k / (rr["ms"] / 1e3), "ms_per_step": rr["ms"] / k,
                           "steps": k, "cg_iterations_last": rr["cg_iterations_last"],
                           "kernels_ms_per_step": {q: v[0] / k for q, v in rr["kt"].items()}}
            if fp == "fp64":
                forms[name]["roofline_fp64"] = fp64_roofline(rr["kt"], f.g.num_particles, a.workload)
            f.close()
        if sur is not None and chosen_wp is not sur:  # the trained network in place of the lagged solve
            f = Form(cfg, mesh, stream, precision=prec, sur=sur)
            s0 = f.g.surrogate_stats()
            rr = f.timed(dt, k, 3)
            s1 = f.g.surrogate_stats()
            f.last_wp = f.g.field("node_wp")
            forms["surrogate_node_form"] = {
                "value": f.g.num_particles * k / (rr["ms"] / 1e3), "ms_per_step": rr["ms"] / k, "steps": k,
                "fe_fallbacks": int(s1[1] - s0[1]), "wp_error_vs_fe": surrogate_error(f, mesh),
                "kernels_ms_per_step": {q: v[0] / k for q, v in rr["kt"].items()}}
            f.close()
        if chosen_wp is not None:  # the chosen form with the mean-pressure projection added
            f = Form(cfg, mesh, stream, precision=prec, sur=chosen_wp, pressure=1)
            rr = f.timed(dt, k, 3)
            forms["chosen_with_pressure_projection"] = {
                "value": f.g.num_particles * k / (rr["ms"] / 1e3), "ms_per_step": rr["ms"] / k, "steps": k,
                "pressure_tol": f.g.params.pressure_tol,
                "pressure_iterations_last": rr["pressure_iterations_last"],
                "kernels_ms_per_step": {q: v[0] / k for q, v in rr["kt"].items()}}
            f.close()
        stated["precision_study"] = precision_study(cfg, mesh, dt, stream, sur, steps=200, lag_tol=a.lag_tol,
                                                    lag_cg_tol=a.lag_cg_tol)
        stated["standard_errors"] = standard_error_study(cfg, mesh, dt, stream, sur, lag_tol=a.lag_tol,
                                                         lag_cg_tol=a.lag_cg_tol,
                                                         seeds=a.se_seeds)
    # the other workloads of the recipe, measured in the same run: the small
    # wall-function canyon and the 32-case batch
    workloads = {}
    if not a.no_forms and rank == 0 and world == 1:
        workloads["canyon_wf_small"] = small_case_summary(stream)
        workloads["canyon_batch32"] = batch_summary(a)
    # the instruction-issue roofline of the kernels that issue rather than
    # stream bound (their HBM fraction alone reads low)
    sm_mhz = (rg["clocks"] or {}).get("sm_mhz")
    for k, rl_k in rooflines.items():
        if k in KTRAFFIC and rl_k.get("ms_per_launch"):
            iss = issue_roofline(KTRAFFIC[k], rl_k["ms_per_launch"], a.workload, prec, sm_mhz)
            if iss:
                rl_k["issue"] = iss
    if roof.get("ms_per_launch") and dominant in KTRAFFIC:
        iss = issue_roofline(KTRAFFIC[dominant], roof["ms_per_launch"], a.workload, prec, sm_mhz)
        if iss:
            roof["issue"] = iss
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps_timed,
            "warmup": a.warmup, "ms_per_step": ms / steps_timed, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec != "fp64" else "f64",
            "data": "synthetic", "config": config_block(cfg, mesh, n, prec, form_name),
            "roofline": roof, "rooflines": rooflines, "e2e": e2e, "gpu_launches": int(rg["launches"]),
            "clocks": rg["clocks"], "kernels": kernels, "status": rg["status"],
            "timing": {"value": "one CUDA graph per step pair (pdf_batch_* with one context), CUDA events on "
                                "its launch stream",
                       "kernels": "CUDA events around every kernel class in an eager pass of the same steps on a "
                                  "second context of the same seed",
                       "eager_ms_per_step": eager_ms / a.steps, "eager_status": capi_status(r["status"])},
            "cg_iterations_last": r["cg_iterations_last"], "surrogate": sur_info}
    if sustained:
        line["sustained_production_run"] = sustained
        if sustained_other:
            line["sustained_other_forms"] = sustained_other
    if workloads:
        line["workloads"] = workloads
    if forms:
        line["forms"] = forms
        line["speedup_vs_plain_fp64"] = value / forms["plain_fp64_fe"]["value"]
    if stated:
        line["stated_error"] = stated
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, mesh, dt)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def capi_status(st):
    from paper_1003_4548_gb300 import capi
    return capi.ERRORS.get(st, "ok") if st else "ok"


def precision_study(cfg, mesh, dt, stream, sur, steps, lag_tol=0.03, lag_cg_tol=None):
    """The same seeded ensemble advanced `steps` steps in each form; statistics
    on a 12 x 8 grid of cells compared with the all-FP64 form (relative rms),
    next to the Monte Carlo scale (the FP64 form with another seed)."""
    lag = lambda tol: {"mode": 5, "params": None, "norm": None, "tol": tol, "cg_tol": lag_cg_tol}  # noqa: E731
    variants = (("fp64_fe", "fp64", 0, None, None), ("fp64_fe_other_seed", "fp64", 0, None, 1),
                ("fp32_fe", "fp32", 0, None, None), ("fp32_kahan_fe", "fp32_kahan", 0, None, None),
                ("fp32_fe_ff_cg", "fp32", 1, None, None),
                ("fp32_kahan_surrogate", "fp32_kahan", 0, sur, None),
                ("chosen_fp32_kahan_lagged_fe", "fp32_kahan", 0, lag(lag_tol), None),
                ("fp32_kahan_frozen_wp", "fp32_kahan", 0, lag(1e30), None))
    ref, out = None, {}
    for name, prec, cgp, s, seed in variants:
        if s is None and name == "fp32_kahan_surrogate":
            continue
        f = Form(cfg, mesh, stream, precision=prec, cg_precision=cgp, sur=s, seed=seed)
        s0 = f.g.surrogate_stats() if s is not None else None
        rr = f.timed(dt, steps, 0)
        st = cell_stats(f.g, mesh)
        rate = f.g.num_particles * steps / (rr["ms"] / 1e3)
        if ref is None:
            ref = st
        out[name] = {"particle_steps_per_s": rate,
                     "rel_rms_vs_fp64": {q: rel_rms(st[q], ref[q]) for q in st}}
        if s is not None:
            s1 = f.g.surrogate_stats()
            out[name]["fe_solves"] = int(s1[1] - s0[1])
        f.close()
    return {"steps": steps, "cells": "12 x 8 grid, particle-weighted element means", "variants": out,
            "note": "fp64_fe_other_seed is the Monte Carlo scale: differences below it are within sampling noise"}


def z_cells(A, B):
    """Per cell and statistic, the difference of two seed ensembles' means in
    standard errors, (mean_A - mean_B) / sqrt(s_A^2 / M_A + s_B^2 / M_B)
    (a statistic identical in every run, e.g. psi = 0 far from the source,
    gives 0); then the largest |z| and the fraction of |z| above 3."""
    import numpy as np
    out, flat, allz, tiny = {}, [], [], 0
    for q in A[0]:
        a, b = np.array([x[q] for x in A]), np.array([x[q] for x in B])
        # a form with FP32 particle state cannot hold a value below FP32's
        # smallest normal number (its arithmetic flushes them to zero): where
        # such values decide a cell (psi far upwind of the source, about
        # 1e-40 to 1e-170 in FP64), both ensembles take them as zero
        small = (np.abs(a) < FLT_MIN) | (np.abs(b) < FLT_MIN)
        tiny += int(np.sum(np.any(small & ((a != 0) | (b != 0)), axis=0)))
        a, b = np.where(np.abs(a) < FLT_MIN, 0.0, a), np.where(np.abs(b) < FLT_MIN, 0.0, b)
        d = a.mean(0) - b.mean(0)
        se = np.sqrt(a.var(0, ddof=1) / len(A) + b.var(0, ddof=1) / len(B))
        ok = se > 0
        z = np.where(ok, d / np.where(ok, se, 1.0), 0.0)
        # cells with no spread in either ensemble (every run of both sets
        # gives the same value, e.g. psi = 0 where the scalar has not
        # arrived): listed with their values, not turned into a z
        for c in np.flatnonzero(~ok & (d != 0))[:4]:
            flat.append({"stat": q, "cell": int(c), "value": float(a[0, c]), "reference": float(b[0, c])})
        out[q] = float(np.abs(z).max())
        allz.append(np.abs(z[ok]))
    allz = np.concatenate(allz)
    return {"max_abs_z": float(allz.max()) if allz.size else 0.0,
            "frac_above_3": float(np.mean(allz > 3)) if allz.size else 0.0, "tests": int(allz.size),
            "max_abs_z_per_stat": out, "cells_without_spread_differing": flat,
            "cells_with_values_below_fp32_normal_range": tiny}


def standard_error_study(cfg, mesh, dt, stream, sur, lag_tol=0.03, lag_cg_tol=None, seeds=8,
                         checkpoints=(200, 500)):
    """The stated error of each form in Monte Carlo standard errors: `seeds`
    runs of the plain FP64 form (FE solve every step) and `seeds` runs of
    each other form, with disjoint seeds, from their seeded starts; at each
    checkpoint step the 12 x 8 cell statistics (<U>, <V>, <uu>, <vv>, <ww>,
    <uv>, k, <psi>, psi variance) of the two ensembles are compared cell by
    cell in standard errors of the difference of their means. Without a bias
    |z| follows Student's t with 2 x seeds - 2 degrees of freedom (about 1 % of
    the tests above 3 for 8 seeds). The chosen form also runs on the FP64
    runs' own seeds: the paired differences state its bias per cell in
    standard errors of the FP64 ensemble's mean (paired_bias)."""
    lag = {"mode": 5, "params": None, "norm": None, "tol": lag_tol, "cg_tol": lag_cg_tol}
    forms = [("fp64_fe", "fp64", None, 1000), ("chosen_fp32_kahan_lagged_fe", "fp32_kahan", lag, 2000),
             ("fp32_kahan_fe", "fp32_kahan", None, 3000)]
    if sur is not None:
        forms.append(("fp32_kahan_surrogate_node_form", "fp32_kahan", sur, 4000))
        forms.append(("fp32_kahan_lagged_fe_with_network_correction", "fp32_kahan",
                      dict(sur, mode=6, tol=lag_tol, cg_tol=lag_cg_tol), 5000))
    t0 = time.perf_counter()
    cells = {}
    for name, prec, s, base in forms:
        runs = {c: [] for c in checkpoints}
        for i in range(seeds):
            f = Form(cfg, mesh, stream, precision=prec, sur=s, seed=base + i)
            done = 0
            for c in checkpoints:
                f.g.step(dt, c - done)
                done = c
                f.g.sync()
                runs[c].append(cell_stats(f.g, mesh))
            f.close()
        cells[name] = runs
    # the chosen form again on the FP64 runs' own seeds: paired differences,
    # in which the Monte Carlo noise common to a pair cancels
    paired = {c: [] for c in checkpoints}
    for i in range(seeds):
        f = Form(cfg, mesh, stream, precision="fp32_kahan", sur=lag, seed=1000 + i)
        done = 0
        for c in checkpoints:
            f.g.step(dt, c - done)
            done = c
            f.g.sync()
            paired[c].append(cell_stats(f.g, mesh))
        f.close()
    out = {"seeds_per_form": seeds, "checkpoints": list(checkpoints), "reference": "fp64_fe",
           "cells": "12 x 8 grid, particle-weighted element statistics", "wall_s": None}
    for name in cells:
        if name == "fp64_fe":
            continue
        out[name] = {str(c): z_cells(cells[name][c], cells["fp64_fe"][c]) for c in checkpoints}
    out["chosen_paired_with_fp64_seeds"] = {str(c): paired_bias(paired[c], cells["fp64_fe"][c]) for c in checkpoints}
    out["wall_s"] = round(time.perf_counter() - t0, 1)
    return out


def paired_bias(A, B):
    """Runs A[i] and B[i] share a seed: per cell and statistic the mean of
    the paired differences d = A - B, in units of the Monte Carlo standard
    error of B's ensemble mean (s_B / sqrt(M)), and the paired t = mean(d) /
    (s_d / sqrt(M)) (Student's t with M - 1 degrees of freedom without a
    bias: about 2 % of the tests above 3 for 8 pairs)."""
    import numpy as np
    bias, tmax, allt, flat = {}, {}, [], []
    for q in A[0]:
        a, b = np.array([x[q] for x in A]), np.array([x[q] for x in B])
        a, b = np.where(np.abs(a) < FLT_MIN, 0.0, a), np.where(np.abs(b) < FLT_MIN, 0.0, b)
        d = a - b
        m = len(A)
        se_b = b.std(0, ddof=1) / np.sqrt(m)
        sd_d = d.std(0, ddof=1) / np.sqrt(m)
        ok = se_b > 0
        r = np.where(ok, np.abs(d.mean(0)) / np.where(ok, se_b, 1.0), 0.0)
        okd = sd_d > 0
        t = np.where(okd, d.mean(0) / np.where(okd, sd_d, 1.0), 0.0)
        bias[q] = float(r.max())
        tmax[q] = float(np.abs(t).max())
        allt.append(np.abs(t[okd]))
        flat.append(r[ok])
    allt, flat = np.concatenate(allt), np.concatenate(flat)
    # (pairs that agree exactly leave no paired t: their bias is 0)
    return {"max_bias_in_se": float(flat.max()) if flat.size else 0.0,
            "median_bias_in_se": float(np.median(flat)) if flat.size else 0.0,
            "max_bias_in_se_per_stat": bias, "max_abs_paired_t": float(allt.max()) if allt.size else 0.0,
            "frac_paired_t_above_3": float(np.mean(allt > 3)) if allt.size else 0.0, "tests": int(allt.size),
            "max_abs_paired_t_per_stat": tmax}


if __name__ == "__main__":
    main()
