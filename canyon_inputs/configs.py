"""Named synthetic workloads (input generation only; none of the method's arithmetic).

Each workload fixes the mesh recipe, the particle count per element, the wall
treatment, the precision mode and the run length. The numbers follow the
paper's street-canyon set-up (Section 3: Re ~ 12,000 on U0 and H, so
nu = 1/12000 with U0 = H = 1; log-law inflow; source at street level in the
canyon centre) and the workload sizes of this project:

  canyon_wf_small   ~1,600 triangles, wall functions (walls moved y_p = 0.05H
                    into the fluid), 64 particles per element (~100k), 2x2x2
                    velocity bins, C0 = 2.1, 100 steps at CFL 0.5, FP64.
  canyon_batch32    32 independent wall-resolved canyons: W/H uniform in [0.5, 3],
                    meshes of ~6k-61k triangles (spacing log-uniform in
                    [0.017, 0.1], growth 1.3), 32-256 particles per element
                    (~105M particles in all), each case with its own seed and its
                    source at its own canyon centre.
  canyon_er_full    ~40k triangles graded to a first-cell height nu/u* at the
                    walls, elliptic relaxation solved by P1 finite elements every
                    step, 256 particles per element (~10.3M), FP32 particle state
                    with FP64 statistics and CG, 500 steps. The chosen form
                    keeps the FP32 state, reduces in compensated FP32 and
                    keeps the previous step's wp while its coarse FE residual
                    under the current statistics stays below lag_tol = 0.03
                    (the FE solve, to a relative residual of lag_cg_tol =
                    1e-6, runs when it does not).

The time step follows a CFL rule that depends on the mesh and the initial
condition only: dt = CFL * min_e(2 r_e) / U_ref, with r_e the inradius and
U_ref the largest mean speed of the initial log-law profile plus five standard
deviations of the initial velocity fluctuation.
"""
from __future__ import annotations

import math

import numpy as np

from .mesh import canyon_mesh, inradius

NU = 1.0 / 12000.0
USTAR = 0.05


def yplus30(nu: float = NU, ustar: float = USTAR) -> float:
    """Wall distance at y+ = 30 (Section 3: first point of the wall-function grid)."""
    return 30.0 * nu / ustar


WORKLOADS = {
    "canyon_wf_small": dict(
        mesh=dict(H=1.0, W=1.0, B=2.0, T=2.0, offset=yplus30(), h=0.071, y1=None, seed=0),
        wall_model="wf", per_element=64, bins=(2, 2, 2), C0=2.1, steps=100, cfl=0.5,
        precision="fp64", seed=0, k0=1e-3),
    "canyon_er_full": dict(
        mesh=dict(H=1.0, W=1.0, B=2.0, T=2.0, offset=0.0, h=0.017, y1=NU / USTAR,
                  growth=1.2, seed=0),
        wall_model="er", per_element=256, bins=(2, 2, 2), C0=2.1, steps=500, cfl=0.5,
        precision="fp32", chosen_precision="fp32_kahan", seed=0, k0=1e-3, lag_tol=0.03, lag_cg_tol=1e-6),
}


WORKLOADS["canyon_batch32"] = dict(kind="batch", cases=32, seed=0, wall_model="er", bins=(2, 2, 2), C0=2.1,
                                   cfl=0.5, k0=1e-3, precision="fp32", chosen_precision="fp32_kahan",
                                   mesh=WORKLOADS["canyon_er_full"]["mesh"], per_element=256, lag_tol=0.03,
                                   lag_cg_tol=1e-6)


def batch_cases(cfg: dict) -> list[dict]:
    """The seeded case list of a batch workload: mesh recipe, particles per
    element and seed of every case."""
    rng = np.random.default_rng(cfg["seed"])
    out = []
    for i in range(cfg["cases"]):
        W = float(rng.uniform(0.5, 3.0))
        h = float(np.exp(rng.uniform(np.log(0.017), np.log(0.1))))
        ppe = int(rng.integers(4, 33)) * 8  # 32 .. 256
        out.append(dict(mesh=dict(H=1.0, W=W, B=2.0, T=2.0, offset=0.0, h=h, y1=NU / USTAR, growth=1.3,
                                  seed=1000 + i),
                        per_element=ppe, seed=cfg["seed"] * 1000 + 17 * i + 1))
    return out


def build_mesh(name_or_cfg) -> dict:
    cfg = WORKLOADS[name_or_cfg] if isinstance(name_or_cfg, str) else name_or_cfg
    return canyon_mesh(**cfg["mesh"])


def reference_speed(mesh: dict, *, k0: float, ustar: float = USTAR, kappa: float = 0.41,
                    E: float = 8.5, nu: float = NU) -> float:
    """Largest initial mean speed plus five initial standard deviations."""
    d_top = mesh["T"] - mesh["H"]
    u_top = ustar / kappa * math.log(E * d_top * ustar / nu)
    return u_top + 5.0 * math.sqrt(2.0 / 3.0 * k0)


def cfl_dt(mesh: dict, *, cfl: float, k0: float) -> float:
    return float(cfl * np.min(2.0 * inradius(mesh)) / reference_speed(mesh, k0=k0))


# Sampling locations of Section 3's Table 1 (building walls and roofs) in the
# paper's coordinates (building height 2, canyon between x = 2 and x = 4),
# mapped to these canyons (H = 1, canyon between 1 and 2): x' = (x - 2)/2 + 1,
# y' = y / 2. Entry 10 of the first row prints x = 2.5 in the middle of the
# x = 2 wall sequence and is read as x = 2.
_TABLE1 = ((0.5, 2.0), (1.0, 2.0), (1.5, 2.0), (2.0, 2.0), (2.0, 1.93), (2.0, 1.5), (2.0, 1.33), (2.0, 1.0),
           (2.0, 0.67), (2.0, 0.5), (2.0, 0.33), (2.0, 0.17), (4.0, 0.17), (4.0, 0.33), (4.0, 0.5), (4.0, 0.67),
           (4.0, 1.0), (4.0, 1.33), (4.0, 1.5), (4.0, 1.93), (4.0, 2.0), (4.5, 2.0), (5.0, 2.0), (5.5, 2.0))
# Fig. 7's scalar CDF points (3, 0.2) and (3, 2), mapped the same way
_CDF_POINTS = ((3.0, 0.2), (3.0, 2.0))


def _map(pts, W: float = 1.0):
    return np.array([((x - 2.0) / 2.0 * W + 1.0, y / 2.0) for x, y in pts])


def table1_points(W: float = 1.0) -> np.ndarray:
    """The 24 wall and roof sampling points, shape (24, 2)."""
    return _map(_TABLE1, W)


def cdf_points(W: float = 1.0) -> np.ndarray:
    return _map(_CDF_POINTS, W)
