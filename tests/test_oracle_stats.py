"""Pins of the oracle's Eulerian estimation and elliptic relaxation.

Element moments are the plain ensemble averages of Section 2 (checked against
numpy's own reductions); <phi|V> bins are equal-population groups in
(U, id) -> (V, id) -> (W, id) order (checked against a numpy lexsort
construction, including exact ties); node values are count-weighted means
over incident elements with periodic partners merged; the P1 gradient is exact
for linear fields and the recovered Laplacian tends to the true one;
Eq. H contracted by the oracle equals the explicit fourth-order tensor; the P1
finite-element solve of Eq. elliptic-relaxation converges at O(h^2) to a
manufactured solution.
"""
import math

import numpy as np
import pytest

from canyon_inputs.mesh import canyon_mesh
from oracle import oracle as orc
from oracle.oracle import Oracle
from tests.conftest import oracle_params_for


def seeded(mesh, ppe=24, **over):
    o = Oracle(oracle_params_for(mesh, **over), mesh)
    o.seed(ppe)
    o.estimate_stats()
    return o


def test_element_moments_match_numpy(wf_small_mesh):
    o = seeded(wf_small_mesh, ppe=20, seed=3)
    o.step(0.004, 2)  # mixes particles across elements
    P = o.particles()
    nt = wf_small_mesh["tri"].shape[0]
    e = P["elem"]
    cnt = np.bincount(e, minlength=nt)
    np.testing.assert_array_equal(o.field("elem_n"), cnt)
    mean = o.field("elem_mean")
    R = o.field("elem_R")
    for j, k in enumerate(("u", "v", "w", "psi", "om")):
        want = np.bincount(e, weights=P[k], minlength=nt) / np.maximum(cnt, 1)
        np.testing.assert_allclose(mean[:, j], want, rtol=1e-12, atol=1e-15)
    for j, (a, b) in enumerate((("u", "u"), ("v", "v"), ("w", "w"), ("u", "v"), ("u", "w"), ("v", "w"))):
        for el in range(0, nt, 97):
            sel = e == el
            if sel.sum() < 2:
                continue
            C = np.cov(np.stack([P[a][sel], P[b][sel]]), bias=True)
            assert abs(R[el, j] - C[0, 1]) < 1e-12 * (abs(C[0, 0]) + abs(C[1, 1])) + 1e-17
    pv = o.field("elem_psivar")
    for el in range(0, nt, 97):
        sel = e == el
        if sel.sum():
            assert abs(pv[el] - P["psi"][sel].var()) < 1e-13


def numpy_bins(G, u, v, w, ids):
    n = len(u)
    B = G[0] * G[1] * G[2]
    if n < B:
        return np.zeros(n, int)
    out = np.zeros(n, int)
    groups = [np.arange(n)]
    for d, comp in enumerate((u, v, w)):
        new = []
        for g in groups:
            order = g[np.lexsort((ids[g], comp[g]))]
            sizes = [len(g) // G[d] + (h < len(g) % G[d]) for h in range(G[d])]
            pos = 0
            for h, s in enumerate(sizes):
                sub = order[pos:pos + s]
                out[sub] = out[sub] * G[d] + h
                new.append(sub)
                pos += s
        groups = new
    return out


@pytest.mark.parametrize("G,n", [((2, 2, 2), 64), ((5, 5, 5), 300), ((3, 1, 2), 17), ((2, 2, 2), 5), ((1, 1, 1), 9)])
def test_bins_match_lexsort(G, n):
    p = orc.default_params(nb1=G[0], nb2=G[1], nb3=G[2])
    rng = np.random.default_rng(n)
    u = np.round(rng.standard_normal(n), 1)  # many exact ties -> id decides
    v = np.round(rng.standard_normal(n), 1)
    w = rng.standard_normal(n)
    ids = rng.permutation(10 * n)[:n].astype(np.uint32)
    got = orc.bins(p, u, v, w, ids)
    want = numpy_bins(G, u, v, w, ids)
    np.testing.assert_array_equal(got, want)
    if n >= np.prod(G):
        cnt = np.bincount(got, minlength=np.prod(G))
        assert cnt.max() - cnt.min() <= 3  # equal population up to the split remainders


def test_conditional_means_and_iem_fallback(wf_small_mesh):
    o = seeded(wf_small_mesh, ppe=20, seed=5)
    o.step(0.004, 1)
    P = o.particles()
    cm = o.field("elem_cm")
    n = o.field("elem_n")
    mean = o.field("elem_mean")
    for el in range(0, wf_small_mesh["tri"].shape[0], 53):
        sel = P["elem"] == el
        if n[el] >= 8:
            for b in range(8):
                sb = sel & (P["bin"] == b)
                assert abs(cm[el, b] - P["psi"][sb].mean()) < 1e-14
        else:
            np.testing.assert_allclose(cm[el], mean[el, 3])


def node_incidence(mesh):
    nn = mesh["xy"].shape[0]
    pair = mesh["periodic_pair"]
    inc = [set() for _ in range(nn)]
    for e, t in enumerate(mesh["tri"]):
        for a in t:
            inc[a].add(e)
            if pair[a] >= 0:
                inc[pair[a]].add(e)
    return inc


def test_node_count_weighted_means(wf_small_mesh):
    o = seeded(wf_small_mesh, ppe=20, seed=6)
    o.step(0.004, 1)
    n = o.field("elem_n")
    em = o.field("elem_mean")
    eR = o.field("elem_R")
    nm = o.field("node_mean")
    nR = o.field("node_R")
    inc = node_incidence(wf_small_mesh)
    for i in range(0, wf_small_mesh["xy"].shape[0], 7):
        es = np.array(sorted(inc[i]))
        w = n[es]
        np.testing.assert_allclose(nm[i, 0], np.sum(w * em[es, 0]) / w.sum(), rtol=1e-12, atol=1e-16)
        np.testing.assert_allclose(nm[i, 3], np.sum(w * em[es, 4]) / w.sum(), rtol=1e-12)
        np.testing.assert_allclose(nR[i], (w[:, None] * eR[es]).sum(0) / w.sum(), rtol=1e-12, atol=1e-18)
    pair = wf_small_mesh["periodic_pair"]
    for i in np.nonzero(pair >= 0)[0]:
        np.testing.assert_array_equal(nm[i], nm[pair[i]])
    # constant particle field -> the same constant at every node
    P = o.particles()
    P["u"][:] = 0.625
    o.set_particles(P, step=o.step_index)
    o.estimate_stats()
    np.testing.assert_allclose(o.field("node_mean")[:, 0], 0.625, rtol=1e-14)


def structured(h, jitter=0.0):
    return canyon_mesh(offset=0.0, h=h, y1=None, jitter=jitter, seed=1)


def interior_elements(mesh):
    tag = mesh["edge_tag"]
    tri = mesh["tri"]
    bnode = np.zeros(mesh["xy"].shape[0], bool)
    for e in range(tri.shape[0]):
        for k in range(3):
            if tag[e, k] in (1, 2):
                bnode[tri[e, (k + 1) % 3]] = bnode[tri[e, (k + 2) % 3]] = True
    # also away from the periodic seam images of boundaries: keep it simple
    return ~np.any(bnode[tri], axis=1)


def test_gradient_exact_for_linear_and_laplacian_of_quadratic():
    # linear node field on the jittered periodic canyon: exact P1 gradient, zero Laplacian
    m = structured(0.1, jitter=0.2)
    o = Oracle(oracle_params_for(m), m)
    xy = m["xy"]
    nn = xy.shape[0]
    nR = np.zeros((nn, 6))
    nR[:, 0] = nR[:, 1] = nR[:, 2] = 0.01
    nke = np.tile([0.015, 0.01], (nn, 1))
    nmean = np.zeros((nn, 4))
    nmean[:, 0] = 0.3 + 0.7 * xy[:, 1]     # linear in y (x is periodic)
    nmean[:, 1] = -0.2 * xy[:, 1]
    nmean[:, 3] = 1.0
    o.set_node_fields(nmean, nR, nke)
    d = o.field("elem_der")
    np.testing.assert_allclose(d[:, 0], 0.0, atol=1e-12)
    np.testing.assert_allclose(d[:, 1], 0.7, rtol=1e-12)
    np.testing.assert_allclose(d[:, 3], -0.2, rtol=1e-12)
    np.testing.assert_allclose(d[:, 4:6], 0.0, atol=1e-9)
    # quadratic field on a uniform mesh: point-symmetric node patches make the
    # area-weighted recovered gradient exact, so the Laplacian is exact inside
    sq = square_mesh(12)
    o2 = Oracle(orc.default_params(period=10.0), sq)
    xy = sq["xy"]
    nn = xy.shape[0]
    nm = np.zeros((nn, 4))
    nm[:, 0] = xy[:, 0] ** 2 + 3 * xy[:, 1] ** 2 - xy[:, 0] * xy[:, 1]
    nm[:, 1] = 0.5 * xy[:, 0] ** 2
    nm[:, 3] = 1.0
    o2.set_node_fields(nm, np.tile([0.01, 0.01, 0.01, 0, 0, 0], (nn, 1)), np.tile([0.015, 0.01], (nn, 1)))
    d = o2.field("elem_der")
    edge = (xy[:, 0] < 1.5 / 12) | (xy[:, 0] > 1 - 1.5 / 12) | (xy[:, 1] < 1.5 / 12) | (xy[:, 1] > 1 - 1.5 / 12)
    inner = ~np.any(edge[sq["tri"]], axis=1)
    assert inner.sum() > 50
    np.testing.assert_allclose(d[inner, 4], 8.0, rtol=1e-9)
    np.testing.assert_allclose(d[inner, 5], 1.0, rtol=1e-9)


def test_h_contract_equals_explicit_tensor():
    p = orc.default_params()
    rng = np.random.default_rng(9)
    for _ in range(20):
        A = rng.standard_normal((2, 2)) * 0.1
        R2 = A @ A.T + 0.002 * np.eye(2)
        R33 = 0.003 + 0.001 * rng.random()
        R = np.array([R2[0, 0], R2[1, 1], R33, R2[0, 1], 0.0, 0.0])
        g = rng.standard_normal(4)
        k = 0.5 * (R[0] + R[1] + R[2])
        om = 1.7
        got = orc.h_contract(p, R, g, k, om)
        Rm = np.array([[R[0], R[3], 0], [R[3], R[1], 0], [0, 0, R[2]]])
        b = Rm / np.trace(Rm) - np.eye(3) / 3
        Av = min(1.0, p["Cv"] * np.linalg.det(Rm) / (2 / 3 * k) ** 3)
        d = np.eye(3)
        g5 = p["gamma5"]
        H = ((p["C2"] * Av + g5 / 3) * np.einsum("ik,jl->ijkl", d, d) - g5 / 3 * np.einsum("il,jk->ijkl", d, d)
             + g5 * np.einsum("ik,jl->ijkl", b, d) - g5 * np.einsum("il,jk->ijkl", b, d))
        gradU = np.zeros((3, 3))
        gradU[:2, :2] = g.reshape(2, 2)
        f = 0.5 * (1 - p["C1"]) * k * om * d + k * np.einsum("ijkl,kl->ij", H, gradU)
        np.testing.assert_allclose(got, [f[0, 0], f[0, 1], f[1, 0], f[1, 1], f[2, 2]], rtol=1e-12, atol=1e-15)
        assert abs(f[0, 2]) < 1e-15 and abs(f[2, 1]) < 1e-15
    # Rotta / SLM variant drops the H term
    pr = orc.default_params(rotta=1)
    f2 = orc.h_contract(pr, R, g, k, om)
    iso = 0.5 * (1 - p["C1"]) * k * om
    np.testing.assert_allclose(f2, [iso, 0, 0, iso, iso])


def square_mesh(n):
    xs = np.linspace(0, 1, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    xy = np.stack([X.ravel(), Y.ravel()], 1)
    gid = np.arange((n + 1) ** 2).reshape(n + 1, n + 1)
    tris = []
    for i in range(n):
        for j in range(n):
            a, b, c, d = gid[i, j], gid[i + 1, j], gid[i + 1, j + 1], gid[i, j + 1]
            tris += [(a, b, c), (a, c, d)]
    tri = np.array(tris, np.int32)
    tag = np.zeros_like(tri)
    for e, t in enumerate(tri):
        for k in range(3):
            p, q = xy[t[(k + 1) % 3]], xy[t[(k + 2) % 3]]
            if (p[0] == q[0] and p[0] in (0, 1)) or (p[1] == q[1] and p[1] in (0, 1)):
                tag[e, k] = 1
    return dict(xy=xy, tri=tri, edge_tag=tag, periodic_pair=-np.ones(len(xy), np.int32))


def test_fe_manufactured_solution_second_order():
    Lc = 0.3
    errs = []
    for n in (8, 16, 32):
        m = square_mesh(n)
        o = Oracle(orc.default_params(period=10.0), m)
        xy = m["xy"]
        ex = np.sin(np.pi * xy[:, 0]) * np.sin(np.pi * xy[:, 1])
        f = ((1 + 2 * np.pi ** 2 * Lc ** 2) * ex)[:, None]
        bnd = (xy[:, 0] == 0) | (xy[:, 0] == 1) | (xy[:, 1] == 0) | (xy[:, 1] == 1)
        x = o.fe_solve(np.full(m["tri"].shape[0], Lc), f, np.zeros_like(f), bnd.astype(np.uint8))
        errs.append(np.sqrt(np.mean((x[:, 0] - ex) ** 2)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.8 and 3.3 < r2 < 4.8, errs


def test_fe_solve_matches_direct_solver(tiny_er_mesh):
    """The oracle's CG reaches the discrete solution of the periodic canyon system."""
    sp = pytest.importorskip("scipy.sparse")
    spl = pytest.importorskip("scipy.sparse.linalg")
    m = tiny_er_mesh
    o = Oracle(oracle_params_for(m, wall_model=1), m)
    xy, tri = m["xy"], m["tri"]
    nn, nt = xy.shape[0], tri.shape[0]
    rng = np.random.default_rng(4)
    Le = 0.02 + 0.05 * rng.random(nt)
    pair = m["periodic_pair"]
    rep = np.where((pair >= 0) & (pair < np.arange(nn)), pair, np.arange(nn))
    f = np.cos(2 * np.pi * xy[:, 0] / m["L"])[:, None] * (1 + xy[:, 1][:, None])
    tag = m["edge_tag"]
    wall = np.zeros(nn, bool)
    for e in range(nt):
        for k in range(3):
            if tag[e, k] == 1:
                wall[tri[e, (k + 1) % 3]] = wall[tri[e, (k + 2) % 3]] = True
    wall = wall | wall[rep] | (wall[np.where(pair >= 0, pair, np.arange(nn))])
    g = (0.1 * xy[:, 1])[:, None]
    x = o.fe_solve(Le, f, g, wall.astype(np.uint8))
    # independent assembly on the merged unknowns and a direct solve
    rows, cols, vals = [], [], []
    b = np.zeros(nn)
    for e in range(nt):
        P = xy[tri[e]]
        A2 = (P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[1, 1] - P[0, 1]) * (P[2, 0] - P[0, 0])
        gr = np.array([[-(P[(k + 2) % 3, 1] - P[(k + 1) % 3, 1]), P[(k + 2) % 3, 0] - P[(k + 1) % 3, 0]] for k in range(3)]) / A2
        Me = A2 / 2 / 12 * (np.ones((3, 3)) + np.eye(3))
        Ke = Le[e] ** 2 * A2 / 2 * gr @ gr.T
        for k in range(3):
            for l in range(3):
                rows.append(rep[tri[e, k]]); cols.append(rep[tri[e, l]]); vals.append(Me[k, l] + Ke[k, l])
                b[rep[tri[e, k]]] += Me[k, l] * f[tri[e, l], 0]
    A = sp.csr_matrix((vals, (rows, cols)), shape=(nn, nn))
    free = (rep == np.arange(nn)) & ~wall
    dirn = (rep == np.arange(nn)) & wall
    xs = np.zeros(nn)
    xs[dirn] = g[dirn, 0]
    rhs = b[free] - A[free][:, dirn] @ xs[dirn]
    xs[free] = spl.spsolve(A[free][:, free].tocsc(), rhs)
    np.testing.assert_allclose(x[:, 0], xs[rep], rtol=1e-9, atol=1e-11)
