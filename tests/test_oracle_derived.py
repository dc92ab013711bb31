"""Pins of the oracle's derived fields against hand-evaluated values of the
paper's formulas and against the kinetic-energy budget they must satisfy.

Bakosi, Franzese & Boybeyi, Section 2:
  Eq. dissipation-from-frequency   eps = <omega>(k + nu C_T^2 <omega>)
  Eq. frequency_source             S_omega = C_omega2 - C_omega1 P/eps,
                                   P = -<u_i u_j> d<U_i>/dx_j
  Eq. micromixing-timescale        t_m (all three branches and U_c = 0)
  Eq. L                            L (turbulent and Kolmogorov branches)
  Eqs. Gij, C0                     G_ij and C0 eps from wp_ij
  Eq. wall-GandC                   G_ij and C0 eps of the simplified Langevin model

The expected numbers are in tests/golden/derived_fields_hand.txt with their
arithmetic. Two further pins do not depend on any chosen number:
  * Eqs. Gij and C0 make the GLM conserve the kinetic-energy budget of
    homogeneous turbulence without production: the velocity SDE gives
    dk/dt = G_ij<u_i u_j> + (3/2) C0 eps, and substituting Eqs. Gij, C0 gives
    -eps exactly, for any wp and any Reynolds stress (while C0 > 0);
  * Eq. wall-GandC gives the same budget, -eps, when eps = <omega> k (nu -> 0).
The last test plants one-symbol mistakes in copies of the oracle source and
checks that every one of them breaks at least one of these pins.
"""
import os
import re

import numpy as np
import pytest

from oracle import oracle as orc
from oracle.oracle import Oracle, default_params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "derived_fields_hand.txt")
NU = 1.0 / 12000.0


def expected():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            m = re.match(r"expect\s+(\w+)\s*=\s*(\S+)", line)
            if m:
                out[m.group(1)] = float(m.group(2))
    return out


E = expected()


def hand_mesh():
    """[0,3] x [0,1], three unit squares split by their rising diagonals;
    periodic in x, wall at y = 0, symmetry top at y = 1."""
    xy = np.array([(ix, j) for j in (0, 1) for ix in range(4)], np.float64)
    tri, tag = [], []
    for ix in range(3):
        a, b, c, d = ix, ix + 1, 4 + ix + 1, 4 + ix
        tri.append((a, b, c))                      # lower: (ix,0), (ix+1,0), (ix+1,1)
        tag.append((3 if ix + 1 == 3 else 0, 0, 1))
        tri.append((a, c, d))                      # upper: (ix,0), (ix+1,1), (ix,1)
        tag.append((2, 3 if ix == 0 else 0, 0))
    pair = np.full(8, -1, np.int32)
    pair[0], pair[3], pair[4], pair[7] = 3, 0, 7, 4
    return dict(xy=xy, tri=np.array(tri, np.int32), edge_tag=np.array(tag, np.int32),
                periodic_pair=pair)


def hand_params(**over):
    p = default_params(period=3.0, x0=2.0 / 3.0 + 0.3, y0=1.0 / 3.0 + 0.4, r0=0.05, C0=2.1,
                       wall_model=0, nu=NU)
    p.update(over)
    return p


def node_fields(nn, U=(0.0, 0.0), om=1.0, R=(0.01, 0.01, 0.01, 0.0), k=0.015, eps=0.01, xy=None,
                lin=None):
    nmean = np.zeros((nn, 4))
    nmean[:, 0], nmean[:, 1], nmean[:, 3] = U[0], U[1], om
    if lin is not None:  # <U> = U0 + a x + b y, <V> = V0 + c x + d y
        (u0, a, b), (v0, c, d) = lin
        nmean[:, 0] = u0 + a * xy[:, 0] + b * xy[:, 1]
        nmean[:, 1] = v0 + c * xy[:, 0] + d * xy[:, 1]
    nR = np.zeros((nn, 6))
    nR[:, 0], nR[:, 1], nR[:, 2], nR[:, 3] = R
    nke = np.zeros((nn, 2))
    nke[:, 0], nke[:, 1] = k, eps
    return nmean, nR, nke


def close(a, b, rtol=1e-12):
    assert abs(a - b) <= rtol * abs(b) + 1e-300, (a, b)


# --- pins, each taking the oracle library to check (None: the real one) -----

def pin_dissipation(L=None):
    mesh = hand_mesh()
    o = Oracle(hand_params(), mesh, library=L)
    nt = mesh["tri"].shape[0]
    cen = mesh["xy"][mesh["tri"]].mean(axis=1)
    s = np.array([(1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)], np.float64)
    fl = s * np.array([0.1, 0.2, 0.1])
    for om, key in ((2.0, "D1_eps"), (100.0, "D2_eps")):
        n = 4 * nt
        st = dict(x=np.repeat(cen[:, 0], 4), y=np.repeat(cen[:, 1], 4),
                  u=1.0 + np.tile(fl[:, 0], nt), v=np.tile(fl[:, 1], nt), w=np.tile(fl[:, 2], nt),
                  om=np.full(n, om), psi=np.zeros(n), id=np.arange(n, dtype=np.uint32),
                  elem=np.repeat(np.arange(nt, dtype=np.int32), 4))
        o.set_particles(st)
        o.estimate_stats()
        ke = o.field("node_ke")
        for i in range(ke.shape[0]):
            close(ke[i, 0], E["D1_k"])
            close(ke[i, 1], E[key])


def pin_production_source(L=None):
    mesh = hand_mesh()
    o = Oracle(hand_params(), mesh, library=L)
    nn = mesh["xy"].shape[0]
    f = node_fields(nn, R=(0.02, 0.01, 0.015, -0.004), k=0.0225, eps=0.011, xy=mesh["xy"],
                    lin=((1.0, 0.3, -0.2), (0.0, 0.5, 0.4)))
    o.set_node_fields(*f)
    der = o.field("elem_der")
    for e in range(der.shape[0]):
        close(der[e, 0], E["S_dUdx"], 1e-12)
        close(der[e, 1], E["S_dUdy"], 1e-12)
        close(der[e, 2], E["S_dVdx"], 1e-12)
        close(der[e, 3], E["S_dVdy"], 1e-12)
        close(der[e, 6], E["S_Somega"], 1e-12)


def pin_timescale(L=None):
    mesh = hand_mesh()
    o = Oracle(hand_params(), mesh, library=L)
    nn = mesh["xy"].shape[0]
    U = (0.84, 1.12)
    o.set_node_fields(*node_fields(nn, U=U, k=1.25, eps=0.3125))
    close(o.field("elem_der")[0, 7], E["T1_tm_elem0"])
    for k, key, Uk in ((0.05, "T2_tm", U), (0.01, "T3_tm", U), (1.25, "T4_tm", (0.0, 0.0))):
        o.set_node_fields(*node_fields(nn, U=Uk, k=k, eps=0.3125))
        for v in o.field("elem_der")[:, 7]:
            close(v, E[key])


def pin_length(L=None):
    mesh = hand_mesh()
    o = Oracle(hand_params(), mesh, library=L)
    nn = mesh["xy"].shape[0]
    for k, key in ((0.01, "L1"), (0.001, "L2")):
        o.set_node_fields(*node_fields(nn, k=k, eps=0.01))
        for v in o.field("elem_der")[:, 8]:
            close(v, E[key])


def pin_G_C0_hand(L=None):
    mesh = hand_mesh()
    o = Oracle(hand_params(wall_model=1), mesh, library=L)
    nn = mesh["xy"].shape[0]
    o.set_node_fields(*node_fields(nn, R=(0.016, 0.008, 0.016, -0.005), k=0.02, eps=0.01))
    wp = np.tile([-0.004, 0.003, -0.001, -0.002, -0.003], (nn, 1))
    o.set_node_wp(wp)
    pk = o.field("node_pack")
    for i in range(nn):
        for col, key in ((4, "G_G11"), (5, "G_G12"), (6, "G_G21"), (7, "G_G22"), (8, "G_G33"),
                         (3, "G_C0eps")):
            close(pk[i, col], E[key])
    o.set_node_wp(np.tile([0.01, 0.0, 0.0, 0.01, 0.01], (nn, 1)))
    assert np.all(o.field("node_pack")[:, 3] == E["G2_C0eps"])


def pin_G_C0_energy_budget(L=None):
    """Eqs. Gij, C0: G_ij<u_i u_j> + (3/2) C0 eps = -eps at every node whose
    C0 eps is not clamped, with wp from the oracle's own FE solve under
    random statistics; where it is clamped, wp_ij<u_i u_j> >= 0."""
    from canyon_inputs.mesh import canyon_mesh
    mesh = canyon_mesh(offset=0.0, h=0.12, y1=0.01, growth=1.3, seed=5)
    o = Oracle(default_params(wall_model=1, period=mesh["L"], x0=mesh["L"] / 2), mesh, library=L)
    rng = np.random.default_rng(11)
    nn = mesh["xy"].shape[0]
    uu, vv, ww = (rng.uniform(0.002, 0.03, nn) for _ in range(3))
    uv = rng.uniform(-0.9, 0.9, nn) * np.sqrt(uu * vv)
    nmean = np.stack([rng.normal(0.5, 0.3, nn), rng.normal(0.0, 0.2, nn), np.zeros(nn),
                      rng.uniform(0.5, 5.0, nn)], axis=1)
    nR = np.stack([uu, vv, ww, uv, np.zeros(nn), np.zeros(nn)], axis=1)
    k = 0.5 * (uu + vv + ww)
    eps = rng.uniform(0.002, 0.05, nn)
    o.set_node_fields(nmean, nR, np.stack([k, eps], axis=1))
    wp, pk = o.field("node_wp"), o.field("node_pack")
    G = pk[:, 4:9]
    GR = G[:, 0] * uu + G[:, 1] * uv + G[:, 2] * uv + G[:, 3] * vv + G[:, 4] * ww
    wR = wp[:, 0] * uu + wp[:, 1] * uv + wp[:, 2] * uv + wp[:, 3] * vv + wp[:, 4] * ww
    free = pk[:, 3] > 0
    assert free.sum() > nn // 4 and (~free).sum() > 0, (free.sum(), nn)
    resid = GR[free] + 1.5 * pk[free, 3] + eps[free]
    assert np.all(np.abs(resid) <= 1e-12 * (np.abs(GR[free]) + eps[free])), np.abs(resid).max()
    assert np.all(wR[~free] >= 0.0)


def pin_slm(L=None):
    mesh = hand_mesh()
    o = Oracle(hand_params(wall_model=0, C0=2.1), mesh, library=L)
    nn = mesh["xy"].shape[0]
    R = (0.03, 0.02, 0.01, -0.01)        # anisotropic, tr R = 2k = 0.06
    o.set_node_fields(*node_fields(nn, om=2.0, R=R, k=0.03, eps=0.06))
    pk = o.field("node_pack")
    for i in range(nn):
        for col in (4, 7, 8):
            close(pk[i, col], E["W_Gii"])
        assert pk[i, 5] == 0.0 and pk[i, 6] == 0.0
        close(pk[i, 3], E["W_C0eps"])
        GR = pk[i, 4] * R[0] + pk[i, 7] * R[1] + pk[i, 8] * R[2] + (pk[i, 5] + pk[i, 6]) * R[3]
        close(GR + 1.5 * pk[i, 3], -0.06, 1e-12)


PINS = [pin_dissipation, pin_production_source, pin_timescale, pin_length, pin_G_C0_hand,
        pin_G_C0_energy_budget, pin_slm]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin()


# One-symbol mistakes a transcription could make in the derived-field code:
# (original text, replacement). Each must occur exactly once in the source.
MUTATIONS = [
    ("double eps = Om * (kk + p->nu * p->CT * p->CT * Om);", "double eps = Om * (kk + p->nu * p->CT * Om);"),
    ("double eps = Om * (kk + p->nu * p->CT * p->CT * Om);", "double eps = Om * (kk - p->nu * p->CT * p->CT * Om);"),
    ("double P = -(Rc[0] * Ux", "double P = (Rc[0] * Ux"),
    ("Rc[3] * Uy + Rc[3] * Vx", "Rc[1] * Uy + Rc[3] * Vx"),
    ("d[6] = p->Comega2 - p->Comega1 * P / ec;", "d[6] = p->Comega2 + p->Comega1 * P / ec;"),
    ("cbrt(p->r0 * p->r0 / ec)", "cbrt(p->r0 / ec)"),
    ("p->Ct * dist_source(p, xc, yc) / Ucn", "p->Cs * dist_source(p, xc, yc) / Ucn"),
    ("double t2 = maxd(kc / ec, p->CT * sqrt(p->nu / ec));", "double t2 = mind(kc / ec, p->CT * sqrt(p->nu / ec));"),
    ("double Cxi = 1.0 + 1.3 * 1.0;", "double Cxi = 1.0 + 1.3 * 0.0;"),
    ("maxd(Cxi * pow(kc, 1.5) / ec,", "maxd(Cxi * pow(kc, 0.5) / ec,"),
    ("pow(p->nu * p->nu * p->nu / ec, 0.25)", "pow(p->nu * p->nu / ec, 0.25)"),
    ("q[4] = (2.0 * w[0] - eps) / (2.0 * kk);", "q[4] = (w[0] - eps) / (2.0 * kk);"),
    ("q[5] = w[1] / kk;", "q[5] = w[2] / kk;"),
    ("q[8] = (2.0 * w[4] - eps) / (2.0 * kk);", "q[8] = (2.0 * w[4] + eps) / (2.0 * kk);"),
    ("double c0eps = -2.0 * s / (3.0 * kk);", "double c0eps = -2.0 * s / (2.0 * kk);"),
    ("w[3] * R[1] + w[4] * R[2]", "w[3] * R[1] + w[4] * R[1]"),
    ("double a = -(0.5 + 0.75 * p->C0) * Om;", "double a = -(0.5 + 0.5 * p->C0) * Om;"),
    ("q[3] = p->C0 * eps;", "q[3] = p->C0 * Om;"),
]


def test_pins_catch_planted_mistakes(tmp_path):
    src = open(orc.SRC).read()
    caught = []
    for i, (old, new) in enumerate(MUTATIONS):
        assert src.count(old) == 1, old
        path = tmp_path / f"mut{i}.c"
        path.write_text(src.replace(old, new))
        L = orc.load(orc.compile_source(str(path), str(tmp_path / f"libmut{i}.so")))
        failed = []
        for pin in PINS:
            try:
                pin(L)
            except (AssertionError, RuntimeError):
                failed.append(pin.__name__)
        assert failed, f"no pin catches: {old!r} -> {new!r}"
        caught.append((new, failed))
    assert len(caught) == len(MUTATIONS)
