"""Pins of the Section 4 frequency reflection at wall-function walls,
omega_R = omega_I exp(-2 V_I <omega v>_p / <omega v^2>_p), and of the
frequency-weighted moments it reads.

 - When <omega v>/<omega v^2> takes the value -beta / (2 y_p <omega>) the
   condition reduces exactly to Eq. wall-omega, whatever the wall normal (the
   tangential part of <omega u_i> must not enter).
 - Reflecting twice gives back the incident frequency (V_R = -V_I).
 - Rotating the wall, the velocities and every statistic together leaves
   omega_R unchanged (the wall-frame projections are tensorial).
 - For a particle field with omega = c + s v' exactly (v' the fluctuation about
   the element mean), <omega u> = s <uv>, <omega v> = s <vv>; for s = 0 the
   second moments are c times the Reynolds stresses, in the elements and at
   the nodes.
"""
import math

import numpy as np

from oracle.oracle import Oracle
from tests.conftest import oracle_params_for


def rot(a):
    return np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])


def spd(rng, scale):
    L = rng.standard_normal((2, 2)) * scale
    return L @ L.T + 0.1 * scale * scale * np.eye(2)


def wall_stats(rng, Om):
    Um = rng.standard_normal(2) * 0.3
    R2 = spd(rng, 0.1)
    return np.array([Um[0], Um[1], R2[0, 0], R2[1, 1], 0.02, R2[0, 1], Om])


def beta_of(p):
    return -2.0 / (0.5 + 0.75 * p["C0"] + p["C3"] + p["Comega2"] - p["Comega1"])


def test_reduces_to_wall_omega_condition(tiny_wf_mesh):
    p0 = oracle_params_for(tiny_wf_mesh)
    o0 = Oracle(p0, tiny_wf_mesh)
    o1 = Oracle(oracle_params_for(tiny_wf_mesh, omega_wall=1), tiny_wf_mesh)
    rng = np.random.default_rng(11)
    ratio_coef = -beta_of(p0) / (2.0 * p0["yp"])
    for _ in range(40):
        n = rng.standard_normal(2)
        n /= np.linalg.norm(n)
        t = np.array([n[1], -n[0]])
        Om = rng.uniform(0.5, 5.0)
        stat = wall_stats(rng, Om)
        Wt = spd(rng, 0.2)
        d = n @ Wt @ n
        Wv = (ratio_coef / Om) * d * n + rng.standard_normal() * t  # tangential part is arbitrary
        full = np.concatenate([stat, Wv, [Wt[0, 0], Wt[0, 1], Wt[1, 1]]])
        U = rng.standard_normal(3) * 0.2
        a = o0.reflect(1, n, stat, U[0], U[1], U[2], 1.7)
        b = o1.reflect(1, n, full, U[0], U[1], U[2], 1.7)
        np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-15)


def test_involution_and_rotation(tiny_wf_mesh):
    o = Oracle(oracle_params_for(tiny_wf_mesh, omega_wall=1, fx=0.0, fy=0.0), tiny_wf_mesh)
    rng = np.random.default_rng(12)
    for _ in range(30):
        n = rng.standard_normal(2)
        n /= np.linalg.norm(n)
        stat = wall_stats(rng, 1.2)
        Wv = rng.standard_normal(2) * 0.05
        Wt = spd(rng, 0.2)
        full = np.concatenate([stat, Wv, [Wt[0, 0], Wt[0, 1], Wt[1, 1]]])
        U = rng.standard_normal(3) * 0.2
        r1 = o.reflect(1, n, full, U[0], U[1], U[2], 0.9)
        r2 = o.reflect(1, n, full, *r1)
        np.testing.assert_allclose(r2, [U[0], U[1], U[2], 0.9], rtol=1e-12, atol=1e-14)
        Vi = U[0] * n[0] + U[1] * n[1]
        wv = Wv @ n
        assert (r1[3] > 0.9) == (Vi * wv < 0)
        Q = rot(rng.uniform(0, 2 * math.pi))
        R2 = Q @ np.array([[stat[2], stat[5]], [stat[5], stat[3]]]) @ Q.T
        Um = Q @ stat[:2]
        Wvr = Q @ Wv
        Wtr = Q @ Wt @ Q.T
        fr = np.array([Um[0], Um[1], R2[0, 0], R2[1, 1], stat[4], R2[0, 1], stat[6], Wvr[0], Wvr[1],
                       Wtr[0, 0], Wtr[0, 1], Wtr[1, 1]])
        Ur = Q @ U[:2]
        rr = o.reflect(1, Q @ n, fr, Ur[0], Ur[1], U[2], 0.9)
        np.testing.assert_allclose(Q @ np.array(r1[:2]), rr[:2], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(rr[2:], r1[2:], rtol=1e-12)


def linear_omega_field(mesh, c, s):
    o = Oracle(oracle_params_for(mesh, omega_wall=1, seed=5), mesh)
    o.seed(16)
    o.estimate_stats()
    o.step(0.004, 2)
    P = o.particles()
    nt = mesh["tri"].shape[0]
    cnt = np.maximum(np.bincount(P["elem"], minlength=nt), 1)
    vbar = np.bincount(P["elem"], weights=P["v"], minlength=nt) / cnt
    P["om"] = c + s * (P["v"] - vbar[P["elem"]])
    o.set_particles(P, step=o.step_index)
    o.estimate_stats()
    return o


def test_frequency_weighted_moments(tiny_wf_mesh):
    o = linear_omega_field(tiny_wf_mesh, 2.0, 0.7)
    W, R = o.field("elem_omw"), o.field("elem_R")
    occupied = o.field("elem_n") > 0
    np.testing.assert_allclose(W[occupied, 0], 0.7 * R[occupied, 3], rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(W[occupied, 1], 0.7 * R[occupied, 1], rtol=1e-9, atol=1e-15)
    o = linear_omega_field(tiny_wf_mesh, 2.0, 0.0)
    W, R = o.field("elem_omw"), o.field("elem_R")
    np.testing.assert_allclose(W[:, :2], 0.0, atol=1e-14)
    np.testing.assert_allclose(W[:, 2:], 2.0 * R[:, [0, 3, 1]], rtol=1e-12, atol=1e-17)
    Wn, Rn = o.field("node_omw"), o.field("node_R")
    np.testing.assert_allclose(Wn[:, 2:], 2.0 * Rn[:, [0, 3, 1]], rtol=1e-12, atol=1e-17)


def test_run_conserves_particles_and_differs(tiny_wf_mesh):
    runs = []
    for ow in (0, 1):
        o = Oracle(oracle_params_for(tiny_wf_mesh, omega_wall=ow, seed=9), tiny_wf_mesh)
        o.seed(16)
        o.estimate_stats()
        n0 = o.particles()["x"].size
        o.step(0.004, 4)
        P = o.particles()
        assert P["x"].size == n0
        assert np.all(np.isfinite(P["om"])) and np.all(P["om"] > 0)
        runs.append(P)
    order = [np.argsort(P["id"]) for P in runs]
    om0, om1 = runs[0]["om"][order[0]], runs[1]["om"][order[1]]
    changed = om0 != om1
    assert 0 < changed.sum() < om0.size  # only particles at or near the walls differ
