"""The per-cell standard-error comparison (tests/multiseed.py) on the CPU:
two oracle ensembles with disjoint seeds agree, and an ensemble run with a
wrong Langevin constant (C0 = 3.5 instead of 2.1, Eq. wall-GandC) is told
apart, so the test that compares the GPU with the oracle this way has the
power to see a bias of that size. The small wall-function canyon runs with
the frequency reflection of Section 4: with Eq. wall-omega most seeds blow
up within fifteen steps (particles of the roof-level shear layer that
impinge on the windward wall get their frequency multiplied by
exp(beta V_I / (y_p <omega>)), about 10^3 for V_I near the free-stream
velocity, and the explicit drift of Eq. wall-GandC then diverges)."""
import multiprocessing as mp
import os

from canyon_inputs.configs import WORKLOADS, cfl_dt
from canyon_inputs.mesh import canyon_mesh
from tests import multiseed
from tests.conftest import oracle_params_for

MESH = dict(WORKLOADS["canyon_wf_small"]["mesh"])  # 1,594 triangles


def ensembles(C0_b):
    mesh = canyon_mesh(**MESH)
    dt = cfl_dt(mesh, cfl=0.5, k0=1e-3)
    M, steps, nx, ny = 8, 12, 4, 2
    jobs = [(MESH, oracle_params_for(mesh, C0=2.1, seed=300 + i, omega_wall=1), 64, dt, steps, nx, ny) for i in range(M)]
    jobs += [(MESH, oracle_params_for(mesh, C0=C0_b, seed=400 + i, omega_wall=1), 64, dt, steps, nx, ny) for i in range(M)]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        runs = pool.map(multiseed.oracle_run, jobs)
    return multiseed.summary(multiseed.z_scores(runs[:M], runs[M:]))


def test_same_model_within_standard_errors():
    s = ensembles(2.1)
    assert s["frac_above_3"] <= 0.05 and s["max_abs_z"] < 6.0, s


def test_wrong_constant_is_seen():
    s = ensembles(3.5)
    assert s["max_abs_z"] > 6.0 and s["frac_above_3"] > 0.1, s
