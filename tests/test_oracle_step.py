"""Pins of the oracle's whole time step (Section 2 equations + Section 3 set-up).

Invariants the method fixes: the particle count and the set of particle ids
are conserved (periodic x, reflecting walls); every particle lies in its host
element afterwards; with the source switched off the mixing substep conserves
the total scalar and keeps it within [0, 1]; a particle leaving through the
outflow is re-injected at the inflow (Section 3); the Euler mixing ratio above
one is an error.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from tests.conftest import oracle_params_for
from tests.test_oracle_geometry import brute_locate


def run(mesh, ppe, nsteps, dt, **over):
    o = Oracle(oracle_params_for(mesh, **over), mesh)
    o.seed(ppe)
    o.estimate_stats()
    o.step(dt, nsteps)
    return o


@pytest.mark.parametrize("wall_model", [0, 1])
def test_conservation_and_host_elements(tiny_wf_mesh, tiny_er_mesh, wall_model):
    mesh = tiny_wf_mesh if wall_model == 0 else tiny_er_mesh
    o = Oracle(oracle_params_for(mesh, wall_model=wall_model, r0=0.0, seed=2), mesh)
    o.seed(32)
    P0 = o.particles()
    # give the scalar a non-trivial field to mix
    P0["psi"] = np.clip(0.5 + 0.5 * np.sin(4 * P0["x"]) * np.cos(3 * P0["y"]), 0, 1)
    o.set_particles(P0)
    o.estimate_stats()
    s0 = P0["psi"].sum()
    o.step(0.005, 5)
    P = o.particles()
    assert P["x"].size == P0["x"].size
    assert np.array_equal(np.sort(P["id"]), np.sort(P0["id"]))
    assert np.all((P["x"] >= 0) & (P["x"] < mesh["L"]))
    assert np.all((P["psi"] >= 0) & (P["psi"] <= 1))
    assert abs(P["psi"].sum() - s0) < 1e-10 * P["x"].size
    sub = np.random.default_rng(0).choice(P["x"].size, 1500, replace=False)
    loc, margin = brute_locate(mesh, np.stack([P["x"][sub], P["y"][sub]], 1))
    ok = np.all((margin < -1e-9) | (margin > 1e-9), axis=1)
    assert np.array_equal(loc[ok], P["elem"][sub][ok])
    assert np.all(loc >= 0)
    assert np.all(P["om"] >= 0)


def test_periodic_reinjection(tiny_wf_mesh):
    m = tiny_wf_mesh
    o = Oracle(oracle_params_for(m, seed=4), m)
    o.seed(16)
    P = o.particles()
    i = 0
    P["x"][i], P["y"][i], P["u"][i], P["v"][i] = m["L"] - 1e-3, 1.5, 0.5, 0.0
    P["elem"][i] = o.locate(P["x"][i], P["y"][i])
    o.set_particles(P)
    o.estimate_stats()
    o.step(0.01, 1)
    Q = o.particles()
    j = np.nonzero(Q["id"] == P["id"][i])[0][0]
    assert 0.0 <= Q["x"][j] < 0.05
    assert abs(Q["y"][j] - 1.5) < 0.01
    assert Q["elem"][j] == o.locate(Q["x"][j], Q["y"][j])


def test_euler_mixing_ratio_above_one_is_an_error(tiny_wf_mesh):
    o = Oracle(oracle_params_for(tiny_wf_mesh), tiny_wf_mesh)
    o.seed(16)
    o.estimate_stats()
    st = o.step(50.0, 1, check=False)
    assert st == -8


def test_walls_reflect_inside_domain(tiny_wf_mesh):
    """Velocities pushed toward the floor: every particle stays in the fluid."""
    m = tiny_wf_mesh
    o = Oracle(oracle_params_for(m, seed=8, mix_exp=1), m)
    o.seed(16)
    P = o.particles()
    P["v"] -= 0.5
    o.set_particles(P)
    o.estimate_stats()
    o.step(0.01, 3)
    Q = o.particles()
    for part in np.array_split(np.arange(Q["x"].size), 8):
        loc, _ = brute_locate(m, np.stack([Q["x"][part], Q["y"][part]], 1))
        assert np.all(loc >= 0)
