"""Pins of the oracle's mean-pressure projection (a first-principles P1
fractional step; the scheme the paper cites is not given in it):

 - after a projection the element mean velocities are weakly divergence-free,
   sum_e A_e grad N_i . <U>_e = 0 at every node class (checked from the
   mesh geometry here, not by the oracle);
 - a mean field that is the P1 gradient of a periodic q is removed entirely,
   and the pressure is (q - q(pin)) / dt;
 - the curl of a P1 stream function that vanishes on the whole boundary is
   weakly divergence-free and passes unchanged (zero pressure gradient);
 - projecting twice changes nothing the second time;
 - every particle of an element moves by the same velocity shift, so the
   Reynolds stresses and the velocity bins stay as they were.
"""
import math

import numpy as np

from oracle.oracle import Oracle
from tests.conftest import oracle_params_for


def geometry(mesh):
    """Element areas and the gradients of the three barycentric coordinates."""
    xy, tri = mesh["xy"], mesh["tri"]
    P = xy[tri]  # nt x 3 x 2
    d1, d2 = P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]
    A2 = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    g = np.empty((tri.shape[0], 3, 2))
    for k in range(3):
        a, b = P[:, (k + 1) % 3], P[:, (k + 2) % 3]
        g[:, k, 0] = (a[:, 1] - b[:, 1]) / A2
        g[:, k, 1] = (b[:, 0] - a[:, 0]) / A2
    return 0.5 * A2, g


def node_classes(mesh):
    pair = mesh["periodic_pair"]
    n = pair.size
    rep = np.arange(n)
    has = pair >= 0
    rep[has] = np.minimum(np.arange(n)[has], pair[has])
    return rep


def weak_divergence(mesh, Umean):
    A, g = geometry(mesh)
    rep = node_classes(mesh)
    D = np.zeros(mesh["xy"].shape[0])
    S = np.zeros_like(D)
    for k in range(3):
        t = A * (g[:, k, 0] * Umean[:, 0] + g[:, k, 1] * Umean[:, 1])
        np.add.at(D, rep[mesh["tri"][:, k]], t)
        np.add.at(S, rep[mesh["tri"][:, k]], np.abs(t))
    return D, S


def seeded(mesh, **over):
    kw = dict(pressure=1, cg_tol=1e-13, seed=3)
    kw.update(over)
    o = Oracle(oracle_params_for(mesh, **kw), mesh)
    o.seed(16)
    o.estimate_stats()
    return o


def with_element_means(o, mesh, Ue):
    """Replace each element's mean in-plane velocity by Ue[e], keeping every
    particle's fluctuation."""
    P = o.particles()
    m = o.field("elem_mean")
    e = P["elem"]
    P["u"] = P["u"] - m[e, 0] + Ue[e, 0]
    P["v"] = P["v"] - m[e, 1] + Ue[e, 1]
    o.set_particles(P, step=o.step_index)
    o.estimate_stats()
    return P


def test_projection_is_weakly_divergence_free(tiny_wf_mesh):
    o = seeded(tiny_wf_mesh)
    rng = np.random.default_rng(1)
    Ue = rng.normal(0.0, 0.3, (tiny_wf_mesh["tri"].shape[0], 2)) + [1.0, 0.0]
    with_element_means(o, tiny_wf_mesh, Ue)
    D0, S0 = weak_divergence(tiny_wf_mesh, o.field("elem_mean"))
    assert np.max(np.abs(D0)) > 0.1 * np.max(S0)
    o.project(0.01)
    D, S = weak_divergence(tiny_wf_mesh, o.field("elem_mean"))
    assert np.max(np.abs(D)) < 1e-10 * np.max(S0)


def test_gradient_field_is_removed(tiny_wf_mesh):
    m = tiny_wf_mesh
    o = seeded(m)
    L = m["L"]
    x, y = m["xy"][:, 0], m["xy"][:, 1]
    q = np.sin(2 * math.pi * x / L) * (0.3 + y) + 0.2 * y * y
    A, g = geometry(m)
    gq = np.einsum("ek,ekd->ed", q[m["tri"]], g)
    with_element_means(o, m, gq)
    dt = 0.02
    o.project(dt)
    Um = o.field("elem_mean")[:, :2]
    assert np.max(np.abs(Um)) < 1e-9 * np.max(np.abs(gq))
    pin = int(np.flatnonzero(node_classes(m) == np.arange(q.size))[0])
    np.testing.assert_allclose(o.field("node_p"), (q - q[pin]) / dt, rtol=0, atol=1e-8 * np.max(np.abs(q)) / dt)


def test_discrete_solenoidal_field_passes(tiny_wf_mesh):
    m = tiny_wf_mesh
    o = seeded(m)
    rng = np.random.default_rng(2)
    rep = node_classes(m)
    tag, tri = m["edge_tag"], m["tri"]
    bnd = np.zeros(rep.size, bool)
    for k in range(3):
        on = (tag[:, k] == 1) | (tag[:, k] == 2)
        bnd[rep[tri[on, (k + 1) % 3]]] = True
        bnd[rep[tri[on, (k + 2) % 3]]] = True
    psi = rng.normal(size=rep.size)[rep]  # one value per periodic class
    psi[bnd[rep]] = 0.0
    A, g = geometry(m)
    gpsi = np.einsum("ek,ekd->ed", psi[tri], g)
    curl = np.stack([gpsi[:, 1], -gpsi[:, 0]], 1)
    D, S = weak_divergence(m, curl)
    assert np.max(np.abs(D)) < 1e-12 * np.max(S)  # the field is discretely solenoidal
    with_element_means(o, m, curl)
    before = o.field("elem_mean")[:, :2].copy()
    o.project(0.01)
    np.testing.assert_allclose(o.field("elem_mean")[:, :2], before, rtol=0, atol=1e-10 * np.max(np.abs(curl)))


def test_idempotent_and_uniform_shift(tiny_wf_mesh):
    m = tiny_wf_mesh
    o = seeded(m)
    rng = np.random.default_rng(3)
    with_element_means(o, m, rng.normal(0.0, 0.2, (m["tri"].shape[0], 2)))
    P0 = o.particles()
    R0, bins0 = o.field("elem_R"), P0["bin"].copy()
    o.project(0.01)
    P1 = o.particles()
    assert np.array_equal(P1["id"], P0["id"])
    du, dv = P1["u"] - P0["u"], P1["v"] - P0["v"]
    for e in range(0, m["tri"].shape[0], 7):
        sel = P0["elem"] == e
        assert np.ptp(du[sel]) < 1e-12 and np.ptp(dv[sel]) < 1e-12
    np.testing.assert_allclose(o.field("elem_R"), R0, rtol=1e-9, atol=1e-15)
    assert np.array_equal(P1["bin"], bins0)
    o.project(0.01)
    P2 = o.particles()
    assert np.max(np.abs(P2["u"] - P1["u"])) < 1e-10 and np.max(np.abs(P2["v"] - P1["v"])) < 1e-10


def test_steps_with_projection(tiny_wf_mesh):
    o = seeded(tiny_wf_mesh, seed=9)
    n0 = o.particles()["x"].size
    o.step(0.004, 4)
    P = o.particles()
    assert P["x"].size == n0
    assert all(np.all(np.isfinite(P[k])) for k in ("u", "v", "om", "psi"))
    assert np.all(np.abs(o.field("node_p")) < 1e3)
