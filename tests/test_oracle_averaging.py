"""Pins of the oracle's time averages, probes and scalar CDFs (Section 3:
statistics averaged in time over the stationary steps; Table 1 wall points;
Fig. 7 cumulative distributions of the scalar).

  * the time average is the plain mean of the per-step fields read after
    each averaged step (and steps outside the averaging window do not count);
  * a probe of a node field is its P1 interpolant: exact for a node field
    that is linear in x and y, so a probe anywhere in the domain returns the
    linear function itself;
  * a probe inside the domain takes the element that contains it (the
    oracle's own element walk finds the same one), and a point outside the
    fluid domain takes the element whose smallest barycentric coordinate is
    largest (checked by brute force in numpy);
  * the CDF of a point is the cumulative histogram of the psi values of the
    particles in its element, pooled over the averaged steps.
"""
import numpy as np

from canyon_inputs.configs import cdf_points, cfl_dt, table1_points
from oracle.oracle import Oracle
from tests.conftest import oracle_params_for


def seeded(mesh, **over):
    o = Oracle(oracle_params_for(mesh, C0=2.1, mix_exp=1, **over), mesh)
    o.seed(12)
    o.estimate_stats()
    return o


def test_time_averages_are_means_of_the_steps(tiny_wf_mesh):
    o = seeded(tiny_wf_mesh, seed=31)
    dt = cfl_dt(tiny_wf_mesh, cfl=0.5, k0=1e-3)
    o.step(dt, 1)
    o.set_averaging(True, reset=True)
    sums = {k: 0.0 for k in ("elem_mean", "elem_R", "elem_psivar", "node_mean")}
    for _ in range(4):
        o.step(dt, 1)
        for k in sums:
            sums[k] = sums[k] + o.field(k)
    o.set_averaging(False)
    o.step(dt, 1)
    assert o.averaging_count == 4
    for k, s in sums.items():
        np.testing.assert_allclose(o.averages(k), s / 4, rtol=1e-14, atol=1e-300, err_msg=k)


def barycentric(mesh, e, x, y):
    xy, tri = mesh["xy"], mesh["tri"]
    P = xy[tri[e]]
    T = np.array([[P[0, 0] - P[2, 0], P[1, 0] - P[2, 0]], [P[0, 1] - P[2, 1], P[1, 1] - P[2, 1]]])
    l01 = np.linalg.solve(T, [x - P[2, 0], y - P[2, 1]])
    return np.array([l01[0], l01[1], 1 - l01.sum()])


def test_probes_interpolate_and_locate(tiny_wf_mesh):
    mesh = tiny_wf_mesh
    o = seeded(mesh, seed=32)
    xy, tri = mesh["xy"], mesh["tri"]
    nn = xy.shape[0]
    # a node field linear in x and y: its P1 interpolant is itself
    a, b, c = 0.3, -1.7, 0.25
    nmean = np.zeros((nn, 4))
    nmean[:, 0] = a * xy[:, 0] + b * xy[:, 1] + c
    nR = np.tile([1e-3, 1e-3, 1e-3, 0, 0, 0], (nn, 1))
    nke = np.tile([1.5e-3, 1e-3], (nn, 1))
    o.set_node_fields(nmean, nR, nke)
    rng = np.random.default_rng(5)
    es = rng.choice(tri.shape[0], 40, replace=False)
    lam = rng.dirichlet([2, 2, 2], size=40)
    pts = np.einsum("km,kmd->kd", lam, xy[tri[es]])
    v, el = o.probe("node_mean", 0, pts[:, 0], pts[:, 1])
    np.testing.assert_allclose(v, a * pts[:, 0] + b * pts[:, 1] + c, rtol=1e-13, atol=1e-14)
    assert np.array_equal(el, es)
    assert all(o.locate(x, y) == e for (x, y), e in zip(pts, es))
    # element fields are taken as they are
    v1, _ = o.probe("elem_mean", 3, pts[:, 0], pts[:, 1])
    assert np.array_equal(v1, o.field("elem_mean")[es, 3])
    # points on the physical walls and roofs lie outside the offset fluid
    # domain of the wall-function mesh: the element with the largest
    # smallest barycentric coordinate, by brute force
    wp = table1_points()
    _, elw = o.probe("node_mean", 2, wp[:, 0], wp[:, 1])
    for (x, y), e in zip(wp, elw):
        x = x - mesh["L"] * np.floor(x / mesh["L"])
        m = np.array([barycentric(mesh, q, x, y).min() for q in range(tri.shape[0])])
        assert m[e] >= m.max() - 1e-12, (x, y, e, int(np.argmax(m)))


def test_cdf_is_the_pooled_histogram(tiny_wf_mesh):
    o = seeded(tiny_wf_mesh, seed=33)
    dt = cfl_dt(tiny_wf_mesh, cfl=0.5, k0=1e-3)
    cp = cdf_points()
    o.set_cdf_probes(cp[:, 0], cp[:, 1], 16)
    o.set_averaging(True, reset=True)
    _, pel = o.cdf()
    hist = np.zeros((len(cp), 16))
    for _ in range(3):
        o.step(dt, 1)
        P = o.particles()
        for j, e in enumerate(pel):
            v = P["psi"][P["elem"] == e]
            hist[j] += np.bincount(np.clip((v * 16).astype(int), 0, 15), minlength=16)
    F, el = o.cdf()
    assert np.array_equal(el, pel)
    tot = hist.sum(1, keepdims=True)
    np.testing.assert_allclose(F, np.cumsum(hist, 1) / np.maximum(tot, 1), rtol=0, atol=1e-15)
