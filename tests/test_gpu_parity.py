"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Both sides start from the same seeded mesh, the same particle state and the
same Philox streams. Bars:
  * host element ids: bit-exact except particles within 1e-9 (FP64) or 1e-5
    (FP32) of an element edge in barycentric terms, where the GPU's element
    must still contain the GPU's position;
  * one-step particle state: |gpu - oracle| <= rtol (|oracle| + rms) with
    rtol = 1e-12 (FP64) and 1e-5 (FP32), rms the root mean square of that
    component over the ensemble; in FP32, particles that end within 1e-6 of
    an element edge are left out of the state bar (a boundary crossing by
    less than the FP32 resolution of the position can be taken or not; their
    host element is still checked);
  * statistics from the same particles: rtol 1e-12 (FP64 reductions) or
    2e-6 (compensated FP32 reductions); bins bit-exact;
  * multi-step statistics of independent runs: within 3 Monte Carlo standard
    errors (domain averages).
"""
import numpy as np
import pytest

from canyon_inputs.configs import WORKLOADS, build_mesh, cfl_dt
from canyon_inputs.mesh import canyon_mesh
from oracle.oracle import Oracle
from tests.conftest import oracle_params_for

pytestmark = pytest.mark.gpu

STATE = ("x", "y", "u", "v", "w", "om", "psi")


def gpu_params(mesh, **kw):
    from paper_1003_4548_gb300 import canyon_params
    return canyon_params(mesh, **kw)


def both(mesh, *, precision="fp64", wall_model="wf", C0=2.1, seed=0, cg_tol=1e-14, cg_precision=0, **over):
    """A GPU context and an oracle on the same mesh and parameters. Both FE
    solves of the elliptic relaxation converge to a relative residual of
    1e-14 by default, so the drift tensor they give agrees far below the
    1e-12 bar of the one-step state."""
    from paper_1003_4548_gb300 import Canyon
    gp = gpu_params(mesh, wall_model=wall_model, precision=precision, C0=C0, seed=seed, cg_tol=cg_tol,
                    cg_maxit=20000, cg_precision=cg_precision, **over)
    op = oracle_params_for(mesh, wall_model=0 if wall_model == "wf" else 1, C0=C0, seed=seed,
                           cg_tol=min(cg_tol, 1e-14), **over)
    return Canyon(gp, mesh), Oracle(op, mesh)


def by_id(P):
    order = np.argsort(P["id"], kind="stable")
    return {k: v[order] for k, v in P.items()}


def bary_margin(mesh, P):
    """Smallest barycentric coordinate of each particle in its element."""
    xy, tri = mesh["xy"], mesh["tri"][P["elem"]]
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    X = np.stack([P["x"], P["y"]], 1)

    def orient(p, q, r):
        return (q[:, 0] - p[:, 0]) * (r[:, 1] - p[:, 1]) - (q[:, 1] - p[:, 1]) * (r[:, 0] - p[:, 0])

    A = orient(a, b, c)
    return np.minimum(np.minimum(orient(b, c, X) / A, orient(c, a, X) / A), orient(a, b, X) / A)


def edge_distance(mesh, P):
    """Signed distance of each particle to the nearest edge of its element
    (negative outside): barycentric coordinate times the matching height."""
    xy, tri = mesh["xy"], mesh["tri"][P["elem"]]
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    X = np.stack([P["x"], P["y"]], 1)

    def orient(p, q, r):
        return (q[:, 0] - p[:, 0]) * (r[:, 1] - p[:, 1]) - (q[:, 1] - p[:, 1]) * (r[:, 0] - p[:, 0])

    d0 = orient(b, c, X) / np.hypot(*(c - b).T)
    d1 = orient(c, a, X) / np.hypot(*(a - c).T)
    d2 = orient(a, b, X) / np.hypot(*(b - a).T)
    return np.minimum(np.minimum(d0, d1), d2)


def assert_state_close(g, o, rtol, skip=None, velocity="component"):
    """Relative error per particle and component: each of x, y, u, v, w,
    omega, psi against its own magnitude plus the ensemble rms of that
    component (a small v beside a large u is judged against the spread of v,
    not against |U|). velocity="vector" judges u, v, w against the velocity
    vector's magnitude plus its ensemble rms instead: for the mean-pressure
    projection, whose correction -dt grad p is a vector from an iterative
    solve, its error is of the size of |grad p| in every component.
    Particles flagged in skip are left out."""
    if skip is not None:
        keep = ~skip
        g = {k: v[keep] for k, v in g.items()}
        o = {k: v[keep] for k, v in o.items()}
    speed = np.sqrt(o["u"] ** 2 + o["v"] ** 2 + o["w"] ** 2)
    for k in ("x", "y", "u", "v", "w", "om", "psi"):
        ref = speed if (velocity == "vector" and k in ("u", "v", "w")) else np.abs(o[k])
        scale = ref + np.sqrt(np.mean(ref ** 2)) + 1e-300
        d = np.abs(g[k] - o[k])
        lim = rtol * scale
        bad = d > lim
        if bad.any():
            w = np.argsort(-(d / lim))[:5]
            detail = [{q: float(o[q][i]) for q in STATE} | {"gpu": float(g[k][i]), "elem": int(o["elem"][i])}
                      for i in w]
            raise AssertionError(f"{k}: {int(bad.sum())} of {d.size} beyond rtol {rtol}; worst ratio "
                                 f"{float(np.max(d / lim)):.2f}; worst: {detail}")


def small_mesh():
    return build_mesh(WORKLOADS["canyon_wf_small"])


@pytest.fixture(scope="module")
def wf_mesh():
    return small_mesh()


@pytest.fixture(scope="module")
def er_mesh():
    return canyon_mesh(offset=0.0, h=0.06, y1=2e-3, growth=1.25, seed=2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_seeding_matches_oracle(wf_mesh, precision):
    g, o = both(wf_mesh, precision=precision, seed=5)
    g.seed_particles(24)
    o.seed(24)
    G, O = by_id(g.particles()), by_id(o.particles())
    assert np.array_equal(G["id"], O["id"])
    assert np.array_equal(G["elem"], O["elem"])
    rtol = 1e-13 if precision == "fp64" else 1e-7
    assert_state_close(G, O, rtol)
    # the library keeps its particles sorted by element
    assert np.all(np.diff(g.field("elem")) >= 0)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_kahan"])
@pytest.mark.parametrize("wall_model", ["wf", "er"])
def test_statistics_match_oracle(wf_mesh, er_mesh, precision, wall_model):
    mesh = wf_mesh if wall_model == "wf" else er_mesh
    g, o = both(mesh, precision=precision, wall_model=wall_model, seed=7)
    g.seed_particles(24)
    g.estimate_stats()
    g.step(cfl_dt(mesh, cfl=0.5, k0=1e-3), 2)  # move the particles across elements
    g.sync()
    P = g.particles()
    o.set_particles(P, step=g.step_index)
    o.estimate_stats()
    rt = 1e-12 if precision in ("fp64", "fp32") else 2e-6
    assert np.array_equal(g.field("elem_n"), o.field("elem_n").astype(np.int32))
    for name in ("elem_mean", "elem_R", "elem_psivar", "elem_cm", "node_mean", "node_R", "node_ke",
                 "elem_der", "node_pack", "node_grad"):
        a, b = g.field(name), o.field(name)
        scale = np.sqrt(np.mean(b ** 2, axis=0)) + 1e-300
        tol = rt * (np.abs(b) + scale)
        if wall_model == "er" and name in ("node_pack",):
            tol = tol + 1e-8 * scale  # CG tolerance of the drift tensor
        assert np.all(np.abs(a - b) <= tol), (name, float(np.max(np.abs(a - b) / scale)))
    if wall_model == "er":
        a, b = g.field("node_wp"), o.field("node_wp")
        scale = np.sqrt(np.mean(b ** 2, axis=0))
        assert np.all(np.abs(a - b) <= max(rt, 1e-8) * (np.abs(b) + scale))
    # bins: identical assignment per particle
    gb = by_id({"id": P["id"], "bin": P["bin"]})
    ob = by_id({"id": o.particles()["id"], "bin": o.particles()["bin"]})
    assert np.array_equal(gb["bin"], ob["bin"])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("wall_model", ["wf", "er"])
def test_one_step_matches_oracle(wf_mesh, er_mesh, precision, wall_model):
    mesh = wf_mesh if wall_model == "wf" else er_mesh
    g, o = both(mesh, precision=precision, wall_model=wall_model, seed=11)
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
    G, O, S = by_id(g.particles()), by_id(o.particles()), by_id(P0)
    assert np.array_equal(G["id"], O["id"])
    edge_tol = 1e-9 if precision == "fp64" else 1e-6  # absolute distance to an element edge
    near = np.abs(edge_distance(mesh, O)) < edge_tol
    same = G["elem"] == O["elem"]
    if not np.all(same | near):
        bad = np.nonzero(~same & ~near)[0]
        info = [{"id": int(O["id"][i]), "oracle": (float(O["x"][i]), float(O["y"][i]), int(O["elem"][i])),
                 "gpu": (float(G["x"][i]), float(G["y"][i]), int(G["elem"][i])),
                 "start": (float(S["x"][i]), float(S["y"][i]), float(S["u"][i]), float(S["v"][i]), int(S["elem"][i]))}
                for i in bad[:5]]
        raise AssertionError(f"{len(bad)} host elements differ away from edges: {info}")
    if (~same).any():  # near an edge: the GPU element holds the GPU position
        Gs = {k: v[~same] for k, v in G.items()}
        assert np.all(edge_distance(mesh, Gs) > -10 * edge_tol)
    rtol = 1e-12 if precision == "fp64" else 1e-5
    assert_state_close(G, O, rtol, skip=None if precision == "fp64" else near)
    assert np.array_equal(np.sort(G["elem"]), g.field("elem"))


def test_full_size_sampled_parity():
    """The bench configuration (~40k triangles, 256 per element, FP32 state,
    elliptic relaxation): sampled particles against the oracle one by one."""
    cfg = WORKLOADS["canyon_er_full"]
    mesh = build_mesh(cfg)
    g, o = both(mesh, precision="fp32", wall_model="er", C0=cfg["C0"], seed=cfg["seed"], cg_tol=1e-10)
    dt = cfl_dt(mesh, cfl=cfg["cfl"], k0=cfg["k0"])
    g.seed_particles(cfg["per_element"])
    g.estimate_stats()
    g.step(dt, 1)
    g.sync()
    P0 = g.particles()
    n = P0["x"].size
    assert n == cfg["per_element"] * mesh["tri"].shape[0]
    # properties that hold at any size
    assert np.array_equal(np.bincount(P0["elem"], minlength=mesh["tri"].shape[0]), g.field("elem_n"))
    assert np.all((P0["psi"] >= 0) & (P0["psi"] <= 1))
    assert np.array_equal(np.sort(P0["id"]), np.arange(n, dtype=np.uint32))
    o.set_particles(P0, step=g.step_index)
    o.estimate_stats()
    g.step(dt, 1)
    g.sync()
    G = g.particles()
    rng = np.random.default_rng(0)
    sample = rng.choice(n, 4000, replace=False)  # indices into the oracle's (= P0) order
    o.advance_subset(dt, sample)
    O = o.particles()
    Os = {k: v[sample] for k, v in O.items()}
    pos = np.argsort(G["id"])
    Gs = {k: v[pos[Os["id"]]] for k, v in G.items()}
    near = np.abs(edge_distance(mesh, Os)) < 1e-6
    same = Gs["elem"] == Os["elem"]
    assert np.all(same | near)
    assert_state_close(Gs, Os, 1e-5)


@pytest.mark.parametrize("case", ["wf", "er", "er-chosen"])
def test_multistep_cells_within_standard_errors_of_oracle(case):
    """Eight GPU runs (FP64) and eight oracle runs with disjoint seeds, 50
    forward Euler-Maruyama steps each (end of Section 2) from the seeded
    initial state: the small wall-function canyon (1,594 triangles, 64 per
    element; the frequency reflection of Section 4) and a wall-resolved one with the elliptic relaxation solved
    every step (3,928 triangles, 32 per element). "er-chosen" runs the
    chosen form on the GPU instead (FP32 state, compensated FP32 statistics,
    the lagged FE solve under the coarse check at the wall-resolved
    workload's lag_tol, solved to its lag_cg_tol) against the same
    FP64 oracle with the FE solve every step. Per cell of a 6 x 4 grid
    and per statistic (<U>, <V>, <uu>, <vv>, <ww>, <uv>, k, <psi>, psi
    variance) z is the difference of the two ensemble means in standard
    errors (tests/multiseed.py): |z| > 3 in at most 5 % of the tests (about 1 %
    is the chance rate of Student's t with 14 degrees of freedom) and nowhere
    above 6."""
    import multiprocessing as mp
    import os

    from tests import multiseed
    chosen = case == "er-chosen"
    if case == "wf":
        mesh_kw, ppe, wm = dict(WORKLOADS["canyon_wf_small"]["mesh"]), 64, "wf"
    else:
        mesh_kw = dict(H=1.0, W=1.0, B=2.0, T=2.0, offset=0.0, h=0.1, y1=5e-3, growth=1.3, seed=2)
        ppe, wm = 32, "er"
    mesh = canyon_mesh(**mesh_kw)
    dt = cfl_dt(mesh, cfl=0.5, k0=1e-3)
    steps, M, nx, ny = 50, 8, 6, 4
    # the wall-function canyon with the frequency reflection of Section 4
    # (omega_wall = 1): Eq. wall-omega blows up within fifteen steps for most
    # seeds of this canyon (see tests/test_oracle_multiseed.py)
    ow = 1 if wm == "wf" else 0
    oparams = [oracle_params_for(mesh, wall_model=0 if wm == "wf" else 1, C0=2.1, seed=200 + i, cg_tol=1e-10,
                                 omega_wall=ow) for i in range(M)]
    # the oracle runs in processes of a spawn pool while the GPU runs here
    with mp.get_context("spawn").Pool(min(M, os.cpu_count() or 1)) as pool:
        pending = pool.map_async(multiseed.oracle_run, [(mesh_kw, p, ppe, dt, steps, nx, ny) for p in oparams])
        from paper_1003_4548_gb300 import Canyon
        gpu = []
        for i in range(M):
            er_full = WORKLOADS["canyon_er_full"]
            g = Canyon(gpu_params(mesh, wall_model=wm, precision="fp32_kahan" if chosen else "fp64", C0=2.1,
                                  seed=100 + i, cg_tol=er_full["lag_cg_tol"] if chosen else 1e-10, cg_maxit=20000,
                                  omega_wall=ow), mesh)
            g.seed_particles(ppe)
            g.estimate_stats()
            if chosen:
                g.set_surrogate(5, None, None, er_full["lag_tol"])
            g.step(dt, steps)
            g.sync()
            gpu.append(multiseed.cell_stats(g.field, mesh, nx, ny))
            g.close()
        orc = pending.get(timeout=900)
    z = multiseed.z_scores(gpu, orc)
    s = multiseed.summary(z)
    assert s["frac_above_3"] <= 0.05 and s["max_abs_z"] < 6.0, s


def test_errors_are_reported_not_fatal(wf_mesh):
    g, _ = both(wf_mesh, seed=3, Cs=1e-9, Ct=1e-9)  # tiny t_m: dt/t_m far above one
    g.seed_particles(8)
    g.estimate_stats()
    g.step(1e-3, 1)
    assert g.sync(check=False) == -8
    assert g.sync(check=False) == 0  # the status word is reset, the context stays usable
    P = g.particles()
    assert P["x"].size == 8 * wf_mesh["tri"].shape[0]


@pytest.mark.parametrize("cg_tol", [1e-8, 1e-10])
def test_compensated_fp32_cg_matches_fp64_oracle(er_mesh, cg_tol):
    """The float-float elliptic-relaxation CG reaches the FP64 oracle's
    discrete solution to the requested relative residual."""
    g, o = both(er_mesh, precision="fp32", wall_model="er", seed=9, cg_tol=cg_tol, cg_precision=1)
    g.seed_particles(24)
    g.estimate_stats()
    g.step(cfl_dt(er_mesh, cfl=0.5, k0=1e-3), 2)
    g.sync()
    P = g.particles()
    o.set_particles(P, step=g.step_index)
    o.estimate_stats()
    a, b = g.field("node_wp"), o.field("node_wp")
    scale = np.sqrt(np.mean(b ** 2, axis=0))
    err = np.max(np.abs(a - b) / (np.abs(b) + scale), axis=0)
    assert np.all(err < 100 * cg_tol), err
    assert g.cg_iterations > 0


@pytest.mark.parametrize("precision", ["fp32", "fp32_kahan", "fp64"])
def test_crowded_elements_statistics(wf_mesh, precision):
    """Elements far above the mean count (the density drifts during long runs)
    go through the larger size classes of the moments kernel: 700, 3000 and
    5000 particles in three elements, against the oracle."""
    g, o = both(wf_mesh, precision=precision, seed=13)
    o.seed(16)
    P = o.particles()
    rng = np.random.default_rng(3)
    xy, tri = wf_mesh["xy"], wf_mesh["tri"]
    extra = []
    for e, m in ((5, 700), (77, 3000), (301, 5000)):
        s = np.sqrt(rng.random(m))
        t = rng.random(m)
        lam = np.stack([1 - s, s * (1 - t), s * t], 1)
        X = lam @ xy[tri[e]]
        extra.append(dict(x=X[:, 0], y=X[:, 1], u=1.0 + 0.05 * rng.standard_normal(m),
                          v=0.05 * rng.standard_normal(m), w=0.05 * rng.standard_normal(m),
                          om=rng.gamma(4.0, 0.25, m), psi=rng.random(m), elem=np.full(m, e, np.int32)))
    n0 = P["x"].size
    Q = {k: np.concatenate([P[k]] + [ex[k] for ex in extra]) for k in ("x", "y", "u", "v", "w", "om", "psi", "elem")}
    Q["id"] = np.arange(Q["x"].size, dtype=np.uint32)
    g.set_particles(Q)
    g.estimate_stats()
    g.sync()
    G = g.particles()
    o.set_particles(G)
    o.estimate_stats()
    rt = 2e-6 if precision == "fp32_kahan" else 1e-12
    cnt = g.field("elem_n")
    assert cnt[77] == 3000 + 16 and cnt[301] == 5000 + 16 and cnt[5] == 716
    for name in ("elem_mean", "elem_R", "elem_psivar", "elem_cm"):
        a, b = g.field(name), o.field(name)
        scale = np.sqrt(np.mean(b ** 2, axis=0)) + 1e-300
        assert np.all(np.abs(a - b) <= rt * (np.abs(b) + scale)), name
    gb = by_id({"id": G["id"], "bin": G["bin"]})
    ob = by_id({"id": o.particles()["id"], "bin": o.particles()["bin"]})
    assert np.array_equal(gb["bin"], ob["bin"])


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_kahan"])
def test_ragged_empty_and_tied_elements(wf_mesh, precision):
    """Degenerate element populations against the oracle: empty elements,
    elements with fewer particles than bins (the IEM fallback), exactly as
    many as bins, and elements whose particles share one velocity (bins then
    split by particle id); then one step from that state (FP64)."""
    g, o = both(wf_mesh, precision=precision, seed=17)
    o.seed(12)
    P = o.particles()
    keep = np.zeros(P["x"].size, bool)
    nt = wf_mesh["tri"].shape[0]
    for e in range(nt):
        idx = np.flatnonzero(P["elem"] == e)
        keep[idx[: e % 11]] = True  # 0 .. 10 particles: empty, < 8 bins, = 8, > 8
    Q = {k: v[keep].copy() for k, v in P.items() if k != "bin"}
    tied = np.isin(Q["elem"], np.arange(9, nt, 22))  # elements holding 9 particles
    Q["u"][tied] = 0.75
    Q["v"][tied] = -0.25
    Q["w"][tied] = 0.125
    g.set_particles(Q)
    g.estimate_stats()
    g.sync()
    G = g.particles()
    o.set_particles(G)
    o.estimate_stats()
    cnt = g.field("elem_n")
    assert np.array_equal(cnt, np.arange(nt) % 11)
    assert np.array_equal(cnt, o.field("elem_n").astype(np.int32))
    rt = 2e-6 if precision == "fp32_kahan" else 1e-12
    for name in ("elem_mean", "elem_R", "elem_psivar", "elem_cm", "node_mean", "node_R"):
        a, b = g.field(name), o.field(name)
        scale = np.sqrt(np.mean(b ** 2, axis=0)) + 1e-300
        assert np.all(np.abs(a - b) <= rt * (np.abs(b) + scale)), name
    assert np.all(g.field("elem_mean")[cnt == 0] == 0.0)
    gb = by_id({"id": G["id"], "bin": G["bin"]})
    ob = by_id({"id": o.particles()["id"], "bin": o.particles()["bin"]})
    assert np.array_equal(gb["bin"], ob["bin"])
    if precision == "fp64":
        dt = cfl_dt(wf_mesh, cfl=0.5, k0=1e-3)
        g.step(dt, 1)
        g.sync()
        o.advance(dt)
        Gs, Os = by_id(g.particles()), by_id(o.particles())
        near = np.abs(edge_distance(wf_mesh, Os)) < 1e-9
        assert np.all((Gs["elem"] == Os["elem"]) | near)
        assert_state_close(Gs, Os, 1e-12)


@pytest.mark.parametrize("precision", ["fp32_kahan", "fp32"])
def test_warp_class_sizes_and_crowded_buckets(wf_mesh, precision):
    """Every particle count from 0 to 519 per element (the warp kernels take
    up to 512 particles: the bins kernel nine keys per lane in registers and
    the rest in shared memory, the moments kernel blocks of eight keys per
    lane; larger elements go to the block kernels), against the oracle. Some
    elements make a boundary bucket crowded or tie the boundary value:
    one velocity component constant over the element (every key in one
    bucket: bisection over the value bits, then the ids), half the
    particles sharing a value, values on a coarse grid (many equal values
    near each median)."""
    rng = np.random.default_rng(23)
    xy, tri = wf_mesh["xy"], wf_mesh["tri"]
    nt = tri.shape[0]
    parts = []
    for e in range(nt):
        m = e % 520
        if m == 0:
            continue
        s = np.sqrt(rng.random(m))
        t = rng.random(m)
        X = np.stack([1 - s, s * (1 - t), s * t], 1) @ xy[tri[e]]
        u = 1.0 + 0.05 * rng.standard_normal(m)
        v = 0.05 * rng.standard_normal(m)
        w = 0.05 * rng.standard_normal(m)
        kind = e % 7
        if kind == 1:
            u[:] = 0.8125                       # level 0 bucket holds every key
        elif kind == 2:
            v[: m // 2] = -0.03125              # half the keys share the level-1 value
        elif kind == 3:
            w = np.round(w / 0.02) * 0.02       # a few distinct values at level 2
        elif kind == 4:
            u = np.round(u / 0.01) * 0.01
            v = np.round(v / 0.01) * 0.01
        parts.append(dict(x=X[:, 0], y=X[:, 1], u=u, v=v, w=w, om=rng.gamma(4.0, 0.25, m),
                          psi=rng.random(m), elem=np.full(m, e, np.int32)))
    Q = {k: np.concatenate([p[k] for p in parts]) for k in ("x", "y", "u", "v", "w", "om", "psi", "elem")}
    Q["id"] = rng.permutation(Q["x"].size).astype(np.uint32)
    g, o = both(wf_mesh, precision=precision, seed=29)
    g.set_particles(Q)
    g.estimate_stats()
    g.sync()
    G = g.particles()
    o.set_particles(G)
    o.estimate_stats()
    cnt = g.field("elem_n")
    assert np.array_equal(cnt, np.arange(nt) % 520)
    rt = 2e-6 if precision == "fp32_kahan" else 1e-12
    for name in ("elem_mean", "elem_R", "elem_psivar", "elem_cm"):
        a, b = g.field(name), o.field(name)
        scale = np.sqrt(np.mean(b ** 2, axis=0)) + 1e-300
        assert np.all(np.abs(a - b) <= rt * (np.abs(b) + scale)), name
    gb = by_id({"id": G["id"], "bin": G["bin"]})
    ob = by_id({"id": o.particles()["id"], "bin": o.particles()["bin"]})
    assert np.array_equal(gb["bin"], ob["bin"])


def test_empty_ensemble(wf_mesh):
    """No particles at all: statistics are zero, a step is a no-op."""
    g, _ = both(wf_mesh, seed=19)
    empty = {k: np.zeros(0) for k in ("x", "y", "u", "v", "w", "om", "psi")}
    empty["id"] = np.zeros(0, np.uint32)
    empty["elem"] = np.zeros(0, np.int32)
    g.set_particles(empty)
    g.estimate_stats()
    g.step(1e-3, 2)
    g.sync()
    assert g.num_particles == 0
    assert not g.field("elem_n").any() and not g.field("elem_mean").any()


def test_asynchronous_host_copy(wf_mesh):
    """pdf_get_fields with an asynchronous host destination delivers, after
    pdf_sync, the same bytes as the synchronous copy, for a statistics field
    and a converted particle field."""
    import torch
    g, _ = both(wf_mesh, precision="fp32", seed=3)
    g.seed_particles(16)
    g.estimate_stats()
    g.step(cfl_dt(wf_mesh, cfl=0.5, k0=1e-3), 2)
    for name in ("elem_mean", "u"):
        ref = g.field(name)
        buf = torch.empty(ref.shape, dtype=torch.float64, pin_memory=True)
        g.field_into(name, buf.data_ptr(), ref.nbytes, device=False, asynchronous=True)
        g.sync()
        assert np.array_equal(buf.numpy(), ref)
