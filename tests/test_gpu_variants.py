"""Parity of the two model variants of Section 4 with the FP64 oracle, through
the C ABI:

 - the frequency reflection for general GLM closures at wall-function walls,
   omega_R = omega_I exp(-2 V_I <omega v>_p / <omega v^2>_p): the
   frequency-weighted moments in the elements around the walls and at the wall
   nodes (rtol 1e-12 for FP64 and FP32 state, whose reductions are FP64), then
   one full step (the bars of the main parity suite);
 - the Rotta / simplified Langevin model inside the elliptic relaxation (the
   H_ijkl term dropped): the relaxed wp_ij and one full step.
"""
import numpy as np
import pytest

from canyon_inputs.configs import cfl_dt
from tests.test_gpu_parity import assert_state_close, both, by_id, edge_distance, small_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wf_mesh():
    return small_mesh()


@pytest.fixture(scope="module")
def er_mesh():
    from canyon_inputs.mesh import canyon_mesh
    return canyon_mesh(offset=0.0, h=0.06, y1=2e-3, growth=1.25, seed=2)


def wall_sets(mesh):
    """Wall nodes (periodic partners included) and the elements holding one."""
    tri, tag, pair = mesh["tri"], mesh["edge_tag"], mesh["periodic_pair"]
    wall = np.zeros(mesh["xy"].shape[0], bool)
    for k in range(3):
        on = tag[:, k] == 1
        wall[tri[on, (k + 1) % 3]] = True
        wall[tri[on, (k + 2) % 3]] = True
    has_pair = pair >= 0
    wall[pair[has_pair & wall]] = True
    wall[has_pair] |= wall[pair[has_pair]]
    elems = wall[tri].any(axis=1)
    return wall, elems


def step_parity(mesh, g, o, precision):
    dt = cfl_dt(mesh, cfl=0.5, k0=1e-3)
    g.seed_particles(32)
    g.estimate_stats()
    g.step(dt, 3)
    g.sync()
    P0 = g.particles()
    o.set_particles(P0, step=g.step_index)
    o.estimate_stats()
    g.step(dt, 1)
    g.sync()
    o.advance(dt)
    G, O = by_id(g.particles()), by_id(o.particles())
    assert np.array_equal(G["id"], O["id"])
    edge_tol = 1e-9 if precision == "fp64" else 1e-6
    near = np.abs(edge_distance(mesh, O)) < edge_tol
    assert np.all((G["elem"] == O["elem"]) | near)
    if precision == "fp64":
        assert_state_close(G, O, 1e-12)
    else:  # the FP32 bar of the main parity suite, boundary-grazing particles aside
        assert_state_close(G, O, 1e-5, skip=near)
    return G, O


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_frequency_weighted_wall_moments(wf_mesh, precision):
    # (with compensated FP32 reductions the same kernel centres on element
    # means that carry the 2e-6 bar of those reductions; the centring is
    # checked in the main statistics parity)
    g, o = both(wf_mesh, precision=precision, seed=13, omega_wall=1)
    g.seed_particles(24)
    g.estimate_stats()
    g.step(cfl_dt(wf_mesh, cfl=0.5, k0=1e-3), 2)
    g.sync()
    P = g.particles()
    o.set_particles(P, step=g.step_index)
    o.estimate_stats()
    wall, elems = wall_sets(wf_mesh)
    rt = 1e-12
    for name, rows in (("elem_omw", elems), ("node_omw", wall)):
        a, b = g.field(name), o.field(name)
        assert np.all(a[~rows] == 0.0)
        a, b = a[rows], b[rows]
        scale = np.sqrt(np.mean(b ** 2, axis=0)) + 1e-300
        assert np.all(np.abs(a - b) <= rt * (np.abs(b) + scale)), (name, float(np.max(np.abs(a - b) / scale)))
        assert np.all(scale[2:] > 0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_frequency_reflection_one_step(wf_mesh, precision):
    g, o = both(wf_mesh, precision=precision, seed=17, omega_wall=1)
    G, O = step_parity(wf_mesh, g, o, precision)
    # the variant changes omega after a wall hit: the same step under Eq. wall-omega differs
    g0, o0 = both(wf_mesh, precision="fp64", seed=17)
    G0, _ = step_parity(wf_mesh, g0, o0, "fp64")
    assert np.any(np.abs(G0["om"] - O["om"]) > 1e-6 * np.abs(O["om"]))


def test_omega_wall_fields_need_the_flag(wf_mesh):
    from paper_1003_4548_gb300 import PdfError
    g, _ = both(wf_mesh, seed=1)
    g.seed_particles(8)
    g.estimate_stats()
    with pytest.raises(PdfError):
        g.field("node_omw")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rotta_elliptic_relaxation(er_mesh, precision):
    g, o = both(er_mesh, precision=precision, wall_model="er", seed=19, rotta=1)
    g.seed_particles(24)
    g.estimate_stats()
    g.step(cfl_dt(er_mesh, cfl=0.5, k0=1e-3), 2)
    g.sync()
    P = g.particles()
    o.set_particles(P, step=g.step_index)
    o.estimate_stats()
    a, b = g.field("node_wp"), o.field("node_wp")
    scale = np.sqrt(np.mean(b ** 2, axis=0))
    assert np.all(np.abs(a - b) <= 1e-8 * (np.abs(b) + scale))
    # without H_ijkl the off-diagonal sources vanish, so wp12 = wp21 and both
    # come from the wall values alone
    np.testing.assert_allclose(a[:, 1], a[:, 2], rtol=1e-9, atol=1e-12 * scale[0])
    g, o = both(er_mesh, precision=precision, wall_model="er", seed=23, rotta=1)
    step_parity(er_mesh, g, o, precision)
