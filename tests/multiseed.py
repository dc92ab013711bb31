"""Independent-seed ensembles and their per-cell comparison in Monte Carlo
standard errors (test infrastructure).

The statistics of a run are taken per cell of an nx x ny grid over the
domain: particle-weighted means of the element statistics whose centroid lies
in the cell (<U>, <V>, the Reynolds stresses <uu>, <vv>, <ww>, <uv>, k, <psi>
and the psi variance). Two sets of runs with disjoint seeds estimate the same
expected statistics; per cell and statistic,
    z = (mean_A - mean_B) / sqrt(s_A^2 / M_A + s_B^2 / M_B)
with s^2 the sample variance over the seeds of a set. Without a bias z
follows Student's t with about M_A + M_B - 2 degrees of freedom.
"""
from __future__ import annotations

import numpy as np

STATS = ("U", "V", "uu", "vv", "ww", "uv", "k", "psi", "psi_var")


def cell_stats(field, mesh, nx: int, ny: int) -> dict:
    """field(name) -> element field of a run (elem_n, elem_mean, elem_R, elem_psivar)."""
    cent = mesh["xy"][mesh["tri"]].mean(1)
    cell = (np.clip((cent[:, 0] / mesh["L"] * nx).astype(int), 0, nx - 1) * ny +
            np.clip((cent[:, 1] / mesh["T"] * ny).astype(int), 0, ny - 1))
    n = np.asarray(field("elem_n"), float)
    M, R, pv = field("elem_mean"), field("elem_R"), field("elem_psivar")
    w = np.bincount(cell, weights=n, minlength=nx * ny)
    out = {}
    for name, q in (("U", M[:, 0]), ("V", M[:, 1]), ("uu", R[:, 0]), ("vv", R[:, 1]), ("ww", R[:, 2]),
                    ("uv", R[:, 3]), ("k", 0.5 * (R[:, 0] + R[:, 1] + R[:, 2])), ("psi", M[:, 3]),
                    ("psi_var", pv)):
        out[name] = np.bincount(cell, weights=n * q, minlength=nx * ny) / np.maximum(w, 1.0)
    out["_w"] = w
    return out


def z_scores(A: list, B: list) -> dict:
    """Per-cell z of every statistic between two lists of cell_stats (cells
    holding particles in every run; a statistic identical in every run of
    both sets, e.g. psi = 0 far from the source, gives z = 0)."""
    keep = np.all([a["_w"] > 0 for a in A + B], axis=0)
    out = {}
    for q in STATS:
        a = np.array([x[q][keep] for x in A])
        b = np.array([x[q][keep] for x in B])
        d = a.mean(0) - b.mean(0)
        se = np.sqrt(a.var(0, ddof=1) / len(A) + b.var(0, ddof=1) / len(B))
        z = np.where(se > 0, d / np.where(se > 0, se, 1.0), np.where(d == 0, 0.0, np.inf))
        out[q] = z
    return out


def summary(z: dict) -> dict:
    allz = np.concatenate([np.abs(v) for v in z.values()])
    return {"max_abs_z": float(allz.max()), "frac_above_3": float(np.mean(allz > 3)), "tests": int(allz.size),
            "max_abs_z_per_stat": {q: float(np.abs(v).max()) for q, v in z.items()}}


def oracle_run(args) -> dict:
    """One oracle run (a process of a spawn pool): mesh recipe, oracle
    parameters, particles per element, dt, steps, grid -> cell_stats."""
    mesh_kw, params, ppe, dt, steps, nx, ny = args
    from canyon_inputs.mesh import canyon_mesh
    from oracle.oracle import Oracle
    mesh = canyon_mesh(**mesh_kw)
    o = Oracle(params, mesh)
    o.seed(ppe)
    o.estimate_stats()
    o.step(dt, steps)
    return cell_stats(o.field, mesh, nx, ny)
