"""Error paths of the C ABI, reached without a GPU fault or hang.

Each failure is made on the host (a parameter cap, a value loaded through
pdf_set_particles, a low limit on the solver's bounded waits); the kernels
record it in the context's status word and carry on, and pdf_sync maps the
status to its PDF_ERR_* code, clears it and leaves the context usable:
  * PDF_ERR_CG_NOCONV: one CG iteration allowed (cg_maxit = 1);
  * PDF_ERR_WALL: no boundary reflection allowed (reflect_max = 0) while
    particles move toward the walls;
  * PDF_ERR_NONFINITE: a NaN velocity loaded with the particles;
  * PDF_ERR_LOST_PARTICLE: a particle crossing thousands of elements in one
    step (the element walk is capped);
  * the grid barrier of the cooperative elliptic CG polling once before it
    gives up (pdf_set_wait_limit): PDF_ERR_CUDA "timed out", and with the
    default limit the next solve passes.
"""
import math

import numpy as np
import pytest

from canyon_inputs.configs import cfl_dt

pytestmark = pytest.mark.gpu

ERR_CUDA, ERR_NONFINITE, ERR_LOST, ERR_WALL, ERR_CG = -3, -4, -5, -6, -7


def make(mesh, **kw):
    from paper_1003_4548_gb300 import Canyon, canyon_params
    return Canyon(canyon_params(mesh, **kw), mesh)


def test_cg_not_converged(tiny_er_mesh):
    g = make(tiny_er_mesh, wall_model="er", precision="fp64", cg_maxit=1, cg_tol=1e-14, seed=2)
    g.seed_particles(16)
    g.estimate_stats()  # the elliptic-relaxation solve of the seeded statistics
    assert g.sync(check=False) == ERR_CG
    assert "CG" in g.last_error
    assert g.sync(check=False) == 0  # cleared
    g.close()


def test_wall_reflection_cap(tiny_wf_mesh):
    g = make(tiny_wf_mesh, wall_model="wf", precision="fp64", reflect_max=0, seed=3)
    g.seed_particles(16)
    g.estimate_stats()
    g.sync()
    P = g.particles()
    P["v"] = np.full_like(P["v"], -5.0)  # everything heads for the canyon floor and the roofs
    g.set_particles(P)
    g.estimate_stats()
    g.step(cfl_dt(tiny_wf_mesh, cfl=0.5, k0=1e-3), 1)
    assert g.sync(check=False) == ERR_WALL
    assert g.sync(check=False) == 0
    assert g.particles()["x"].size == P["x"].size
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_kahan"])
def test_nonfinite_state(tiny_wf_mesh, precision):
    g = make(tiny_wf_mesh, wall_model="wf", precision=precision, seed=4)
    g.seed_particles(16)
    g.estimate_stats()
    g.sync()
    P = g.particles()
    P["u"] = P["u"].copy()
    P["u"][P["u"].size // 2] = math.nan
    g.set_particles(P)
    g.estimate_stats()
    g.step(cfl_dt(tiny_wf_mesh, cfl=0.5, k0=1e-3), 1)
    assert g.sync(check=False) == ERR_NONFINITE
    assert g.sync(check=False) == 0
    g.close()


def test_lost_particle(tiny_wf_mesh):
    g = make(tiny_wf_mesh, wall_model="wf", precision="fp64", seed=5)
    g.seed_particles(16)
    g.estimate_stats()
    g.sync()
    P = g.particles()
    # one particle above the roofs, moving along x fast enough to cross
    # thousands of elements (and the periodic seam many times) in one step
    i = int(np.argmax(P["y"]))
    P["u"] = P["u"].copy()
    P["v"] = P["v"].copy()
    P["u"][i], P["v"][i] = 1e5, 0.0
    g.set_particles(P)
    g.estimate_stats()
    g.step(cfl_dt(tiny_wf_mesh, cfl=0.5, k0=1e-3), 1)
    assert g.sync(check=False) == ERR_LOST
    assert g.sync(check=False) == 0
    Q = g.particles()
    assert Q["x"].size == P["x"].size and np.all(Q["elem"] >= 0) and np.all(Q["elem"] < tiny_wf_mesh["tri"].shape[0])
    g.close()


def test_grid_barrier_gives_up(tiny_er_mesh):
    g = make(tiny_er_mesh, wall_model="er", precision="fp64", seed=6)
    g.seed_particles(16)
    g.set_wait_limit(1)  # every waiting block polls once, then proceeds
    g.estimate_stats()
    assert g.sync(check=False) == ERR_CUDA
    assert "timed out" in g.last_error
    g.set_wait_limit(0)  # the default bound: the barriers complete again (the
    g.estimate_stats()   # warm start may hold the undefined solution: no assertion on it)
    assert g.sync(check=False) == 0
    g.close()
    with pytest.raises(Exception):
        g2 = make(tiny_er_mesh, wall_model="er", precision="fp64", seed=6)
        try:
            g2.set_wait_limit(-1)
        finally:
            g2.close()
