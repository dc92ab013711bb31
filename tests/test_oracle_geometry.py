"""Pins of the oracle's mesh, location, seeding and wall conditions.

Location: brute force over all elements (vectorised here, independently of the
oracle's bucket grid) on the lowest-id rule. Wall conditions
(Eqs. wall-normal-velocity .. wall-omega): the reflection is an involution in
the wall frame, V_R = -V_I exactly, the frame rotation is an isometry, and at
log-law equilibrium alpha reduces to 2 u_hat^2 / <v^2>.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from tests.conftest import oracle_params_for


def brute_locate(mesh, pts):
    xy, tri = mesh["xy"], mesh["tri"]
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]

    def orient(p, q, r):
        return (q[..., 0] - p[..., 0]) * (r[..., 1] - p[..., 1]) - (q[..., 1] - p[..., 1]) * (r[..., 0] - p[..., 0])

    area2 = orient(a, b, c)
    P = pts[:, None, :]
    l0 = orient(b[None], c[None], P) / area2
    l1 = orient(c[None], a[None], P) / area2
    l2 = orient(a[None], b[None], P) / area2
    inside = (l0 >= 0) & (l1 >= 0) & (l2 >= 0)
    first = np.where(inside.any(axis=1), inside.argmax(axis=1), -1)
    margin = np.minimum(np.minimum(l0, l1), l2)
    return first, margin


def test_locate_matches_brute_force(tiny_wf_mesh):
    m = tiny_wf_mesh
    o = Oracle(oracle_params_for(m), m)
    rng = np.random.default_rng(0)
    pts = np.stack([rng.uniform(0, m["L"], 3000), rng.uniform(0, m["T"], 3000)], axis=1)
    want, margin = brute_locate(m, pts)
    # stay away from exact ties on edges (measure zero)
    near = np.array([np.any((mg > -1e-12) & (mg < 1e-12)) for mg in margin])
    got = np.array([o.locate(x, y) for x, y in pts])
    assert np.array_equal(got[~near], want[~near])
    assert np.sum(want >= 0) > 1000 and np.sum(want < 0) > 100  # inside and outside cases


def test_wall_distance_brute_force(tiny_wf_mesh):
    m = tiny_wf_mesh
    o = Oracle(oracle_params_for(m), m)
    xy, tri, tag = m["xy"], m["tri"], m["edge_tag"]
    segs = []
    for e in range(tri.shape[0]):
        for k in range(3):
            if tag[e, k] == 1:
                segs.append((xy[tri[e, (k + 1) % 3]], xy[tri[e, (k + 2) % 3]]))
    A = np.array([s[0] for s in segs])
    B = np.array([s[1] for s in segs])
    best = np.full(xy.shape[0], np.inf)
    for shift in (-m["L"], 0.0, m["L"]):
        a = A + [shift, 0]
        b = B + [shift, 0]
        d = b - a
        t = np.clip(np.einsum("snk,sk->sn", xy[None] - a[:, None], d) / np.sum(d * d, axis=1)[:, None], 0, 1)
        proj = a[:, None] + t[..., None] * d[:, None]
        best = np.minimum(best, np.min(np.linalg.norm(xy[None] - proj, axis=2), axis=0))
    np.testing.assert_allclose(o.field("node_wdist"), best + m["offset"], rtol=0, atol=1e-13)


def test_seeding_law(wf_small_mesh):
    m = wf_small_mesh
    p = oracle_params_for(m, seed=11)
    o = Oracle(p, m)
    ppe = 16
    o.seed(ppe)
    P = o.particles()
    n = P["x"].size
    assert n == ppe * m["tri"].shape[0]
    assert np.array_equal(P["id"], np.arange(n, dtype=np.uint32))
    assert np.array_equal(P["elem"], np.repeat(np.arange(m["tri"].shape[0]), ppe))
    # positions are inside their birth element (uniformly: P(l0 > 1/2) = 1/4)
    xy, tri = m["xy"], m["tri"][P["elem"]]
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    X = np.stack([P["x"], P["y"]], axis=1)
    area2 = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    l0 = ((b[:, 0] - X[:, 0]) * (c[:, 1] - X[:, 1]) - (b[:, 1] - X[:, 1]) * (c[:, 0] - X[:, 0])) / area2
    l1 = ((c[:, 0] - X[:, 0]) * (a[:, 1] - X[:, 1]) - (c[:, 1] - X[:, 1]) * (a[:, 0] - X[:, 0])) / area2
    l2 = 1 - l0 - l1
    assert np.all(np.minimum(np.minimum(l0, l1), l2) > -1e-12)
    for lam in (l0, l1, l2):
        frac = np.mean(lam > 0.5)
        assert abs(frac - 0.25) < 5 * np.sqrt(0.25 * 0.75 / n)
    # velocity: Gaussian about the log law with variance 2/3 k0 per component
    sig = math.sqrt(2 / 3 * p["k0"])
    dy = P["y"] - p["y_roof"]
    ulog = np.where(dy >= p["yp"], p["ustar"] / p["kappa"] * np.log(np.maximum(p["E"] * dy * p["ustar"] / p["nu"], 1e-300)), 0.0)
    for r in ((P["u"] - ulog) / sig, P["v"] / sig, P["w"] / sig):
        assert abs(r.mean()) < 5 / math.sqrt(n)
        assert abs(r.var() - 1) < 5 * math.sqrt(2 / n)
    # omega / omega0 ~ Gamma(4, 1/4) with omega0 from the interpolated wall distance
    wd = o.field("node_wdist")
    dw = l0 * wd[tri[:, 0]] + l1 * wd[tri[:, 1]] + l2 * wd[tri[:, 2]]
    om0 = math.sqrt(p["Cmu"]) * p["ustar"] / (p["kappa"] * np.maximum(dw, p["yp"]))
    g = P["om"] / om0
    assert abs(g.mean() - 1) < 5 * math.sqrt(0.25 / n)
    assert abs(g.var() - 0.25) < 5 * math.sqrt((3 * 4 * 6 / 256 - 1 / 16) / n)
    # scalar: unit inside the source disc
    d = np.hypot(P["x"] - p["x0"], P["y"] - p["y0"])
    assert np.array_equal(P["psi"] == 1.0, d < p["r0"])
    assert np.all((P["psi"] == 0) | (P["psi"] == 1))


def rot(t):
    return np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])


def wall_case(rng):
    n = rng.standard_normal(2)
    n /= np.linalg.norm(n)
    Um = rng.standard_normal(2) * 0.3
    Lc = rng.standard_normal((2, 2)) * 0.1
    R2 = Lc @ Lc.T + 0.01 * np.eye(2)
    stat = np.array([Um[0], Um[1], R2[0, 0], R2[1, 1], 0.02, R2[0, 1], 0.8])
    U = rng.standard_normal(3) * 0.2
    return n, stat, U


@pytest.mark.parametrize("wall_model", [0, 1])
def test_wall_reflection_involution_and_normal_flip(tiny_wf_mesh, wall_model):
    o = Oracle(oracle_params_for(tiny_wf_mesh, wall_model=wall_model), tiny_wf_mesh)
    rng = np.random.default_rng(1)
    for _ in range(50):
        n, stat, U = wall_case(rng)
        u1, v1, w1, om1 = o.reflect(1, n, stat, U[0], U[1], U[2], 1.3)
        Vi, Vr = U[0] * n[0] + U[1] * n[1], u1 * n[0] + v1 * n[1]
        assert abs(Vr + Vi) < 1e-14
        u2, v2, w2, om2 = o.reflect(1, n, stat, u1, v1, w1, om1)
        np.testing.assert_allclose([u2, v2, w2, om2], [U[0], U[1], U[2], 1.3], rtol=1e-12, atol=1e-14)
        if wall_model == 0:
            assert w1 == U[2]
            assert (om1 > 1.3) == (Vi < 0)  # beta < 0: incident particles gain frequency
        else:
            np.testing.assert_allclose([u1, v1, w1, om1], [-U[0], -U[1], -U[2], 1.3])


def test_wall_reflection_rotation_isometry(tiny_wf_mesh):
    p = oracle_params_for(tiny_wf_mesh, fx=0.0, fy=0.0)  # no pressure gradient to rotate
    o = Oracle(p, tiny_wf_mesh)
    rng = np.random.default_rng(2)
    for _ in range(30):
        n, stat, U = wall_case(rng)
        Q = rot(rng.uniform(0, 2 * math.pi))
        R2 = np.array([[stat[2], stat[5]], [stat[5], stat[3]]])
        R2r = Q @ R2 @ Q.T
        Umr = Q @ stat[:2]
        statr = np.array([Umr[0], Umr[1], R2r[0, 0], R2r[1, 1], stat[4], R2r[0, 1], stat[6]])
        Ur = Q @ U[:2]
        a = o.reflect(1, n, stat, U[0], U[1], U[2], 0.9)
        b = o.reflect(1, Q @ n, statr, Ur[0], Ur[1], U[2], 0.9)
        np.testing.assert_allclose(Q @ np.array(a[:2]), b[:2], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(a[2:], b[2:], rtol=1e-12)


def test_wall_function_equilibrium_alpha(tiny_wf_mesh):
    """At log-law equilibrium (<U>_p = U_e with u* = u_hat) alpha = 2 u_hat^2/<v^2>."""
    p = oracle_params_for(tiny_wf_mesh, fx=0.0, fy=0.0)
    o = Oracle(p, tiny_wf_mesh)
    us = 0.04
    k = us ** 2 / math.sqrt(p["Cmu"])  # u_hat = Cmu^1/4 k^1/2 = u*
    Ue = us / p["kappa"] * math.log(p["E"] * p["yp"] * us / p["nu"])
    v2 = 0.7 * k
    n = np.array([0.0, 1.0])  # floor: t = (1, 0)
    stat = np.array([Ue, 0.0, 2 * k - v2 - 0.3 * k, v2, 0.3 * k, -us ** 2, 1.0])
    Vi = -0.05
    u, v, w, om = o.reflect(1, n, stat, 0.4, Vi, 0.0, 1.0)
    alpha = (u - 0.4) / Vi
    assert abs(alpha - 2 * us ** 2 / v2) < 1e-12 * alpha
    assert v == -Vi
    # alpha scales with <U>_p |<U>_p| and with 1/<v^2>
    stat2 = stat.copy()
    stat2[0] = -2 * Ue
    u2, *_ = o.reflect(1, n, stat2, 0.4, Vi, 0.0, 1.0)
    assert abs((u2 - 0.4) / Vi + 4 * alpha) < 1e-12 * alpha


def test_symmetry_reflection(tiny_wf_mesh):
    o = Oracle(oracle_params_for(tiny_wf_mesh), tiny_wf_mesh)
    n = np.array([0.0, -1.0])  # top boundary, normal into the fluid
    u, v, w, om = o.reflect(2, n, np.zeros(7), 0.9, 0.2, -0.1, 2.0)
    assert (u, v, w, om) == (0.9, -0.2, -0.1, 2.0)
