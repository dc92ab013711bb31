"""Batched cases in one CUDA graph, and the autotuner.

A batch replays one captured step of several contexts; every case must end
exactly where the same case stepped on its own ends (same kernels in the same
order per case; FP64 reductions, so the particle order inside an element
does not matter). The autotuner changes launch shapes only: a tuned FP64
wall-function context must match an untuned twin stepped as often.
"""
import numpy as np
import pytest

from canyon_inputs.configs import cfl_dt, yplus30
from canyon_inputs.mesh import canyon_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("needs a GPU")
    return t


def cases():
    out = []
    for k, (W, ppe, wm) in enumerate(((0.75, 16, "wf"), (1.0, 24, "er"), (1.5, 32, "wf"))):
        if wm == "wf":
            mesh = canyon_mesh(W=W, offset=yplus30(), h=0.12, seed=20 + k)
        else:
            mesh = canyon_mesh(W=W, offset=0.0, h=0.1, y1=3e-3, growth=1.3, seed=20 + k)
        out.append((mesh, ppe, wm, k))
    return out


def make(torch, mesh, ppe, wm, k, stream, **over):
    from paper_1003_4548_gb300 import Canyon, canyon_params
    precision = over.pop("precision", "fp64")
    cg_tol = over.pop("cg_tol", 1e-10)
    p = canyon_params(mesh, wall_model=wm, precision=precision, C0=2.1, seed=100 + k, case_id=k, cg_tol=cg_tol,
                      cg_maxit=20000, **over)
    g = Canyon(p, mesh, stream=stream.cuda_stream)
    g.seed_particles(ppe)
    g.estimate_stats()
    return g


def by_id(g):
    P = g.particles()
    o = np.argsort(P["id"])
    return {k: v[o] for k, v in P.items()}


def test_batch_graph_matches_individual_steps(torch):
    from paper_1003_4548_gb300 import capi
    cs = cases()
    streams = [torch.cuda.Stream() for _ in range(2 * len(cs) + 1)]
    batched = [make(torch, m, ppe, wm, k, streams[k]) for m, ppe, wm, k in cs]
    alone = [make(torch, m, ppe, wm, k, streams[len(cs) + k]) for m, ppe, wm, k in cs]
    dts = [cfl_dt(m, cfl=0.5, k0=1e-3) for m, _, _, _ in cs]
    b = capi.Batch(batched, dts, streams[-1].cuda_stream)
    for g, dt in zip(alone, dts):
        g.step(dt, 4)
        g.sync()
    b.step(2)
    b.step(2)
    b.sync()
    with pytest.raises(capi.PdfError):
        b.step(3)
    for ga, gb in zip(alone, batched):
        assert gb.step_index == ga.step_index == 4
        A, B = by_id(ga), by_id(gb)
        for k in ("x", "y", "u", "v", "w", "om", "psi", "elem"):
            assert np.array_equal(A[k], B[k]), k
        assert np.array_equal(ga.field("elem_mean"), gb.field("elem_mean"))
    b.close()
    for g in batched + alone:
        g.close()


def test_batch_rejects_shared_streams(torch):
    from paper_1003_4548_gb300 import capi
    m, ppe, wm, k = cases()[0]
    s = torch.cuda.Stream()
    g1 = make(torch, m, ppe, wm, 0, s)
    g2 = make(torch, m, ppe, wm, 1, s)
    with pytest.raises(capi.PdfError):
        capi.Batch([g1, g2], [1e-3, 1e-3], torch.cuda.Stream().cuda_stream)
    g1.close()
    g2.close()


def test_autotune_changes_shapes_not_results(torch):
    from paper_1003_4548_gb300 import capi
    m, ppe, wm, k = cases()[0]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    tuned = make(torch, m, ppe, wm, k, s1, mix_exp=1)
    twin = make(torch, m, ppe, wm, k, s2, mix_exp=1)
    dt = cfl_dt(m, cfl=0.25, k0=1e-3)
    t = tuned.autotune(dt, 1)
    assert 1 <= t["step_blocks_per_sm"] <= 8 and t["scatter_threads"] in (128, 256, 512)
    assert t["cg_rows_per_block"] == 0 and t["ms_particle"] > 0
    twin.step(dt, tuned.step_index)
    tuned.sync()
    twin.sync()
    A, B = by_id(tuned), by_id(twin)
    for key in ("x", "u", "om", "psi", "elem"):
        assert np.array_equal(A[key], B[key]), key
    # the same shapes applied to the twin without timing: the next steps of
    # both stay identical; a shape outside the tuned sets is refused
    twin.apply_tuning(t)
    tuned.step(dt, 2)
    twin.step(dt, 2)
    tuned.sync()
    twin.sync()
    A, B = by_id(tuned), by_id(twin)
    for key in ("x", "u", "om", "psi", "elem"):
        assert np.array_equal(A[key], B[key]), key
    with pytest.raises(capi.PdfError):
        twin.apply_tuning(dict(t, scatter_threads=300))
    tuned.close()
    twin.close()


def test_batch_graph_fp32_lagged_and_pressure(torch):
    """The FP32 path in the graph: the warp-per-element moments on the side
    stream and the bins on the third, the lagged FE solve (mode 5; in the
    graph the CG sits in a conditional node opened by the residual check:
    tolerance 0 solves every step, 1e30 never, 0.05 as the check decides)
    and the pressure projection's cooperative solve. With exact FP32
    reductions (order-independent) a batched case ends exactly where the
    same case stepped on its own ends, with the same solve count."""
    from paper_1003_4548_gb300 import capi
    specs = (("er", dict(), 5, 0.05), ("er", dict(pressure=1, pressure_tol=1e-10), 5, 0.05), ("wf", dict(), 0, 0),
             ("er", dict(), 5, 0.0), ("er", dict(), 5, 1e30))
    cs = cases()
    er_mesh = cs[1][0]
    wf_mesh = cs[0][0]
    streams = [torch.cuda.Stream() for _ in range(2 * len(specs) + 1)]
    batched, alone, dts = [], [], []
    for k, (wm, over, mode, tol) in enumerate(specs):
        mesh = er_mesh if wm == "er" else wf_mesh
        for lst, st in ((batched, streams[k]), (alone, streams[len(specs) + k])):
            g = make(torch, mesh, 24, wm, k, st, **dict(over, precision="fp32"))
            if mode:
                g.set_surrogate(mode, None, None, tol)
            lst.append(g)
        dts.append(cfl_dt(mesh, cfl=0.5, k0=1e-3))
    b = capi.Batch(batched, dts, streams[-1].cuda_stream)
    for g, dt in zip(alone, dts):
        g.step(dt, 4)
        g.sync()
    b.step(4)
    b.sync()
    for ga, gb in zip(alone, batched):
        A, B = by_id(ga), by_id(gb)
        for k in ("x", "y", "u", "v", "w", "om", "psi", "elem", "bin"):
            assert np.array_equal(A[k], B[k]), k
        assert np.array_equal(ga.field("elem_mean"), gb.field("elem_mean"))
        assert np.array_equal(ga.field("node_pack"), gb.field("node_pack"))
    assert np.array_equal(alone[1].field("node_p"), batched[1].field("node_p"))
    for k, (wm, _, mode, tol) in enumerate(specs):
        if mode:
            (sa, fa, _), (sb, fb, _) = alone[k].surrogate_stats(), batched[k].surrogate_stats()
            assert (sa, fa) == (sb, fb), k
            if tol == 0.0:
                assert fa == sa == 4  # every check rejects: the CG runs in every step
            if tol == 1e30:
                assert fa == 0 and sa == 4
    b.close()
    for g in batched + alone:
        g.close()


def test_batch_outputs_per_step(torch):
    """pdf_batch_create_out: the graph copies the element means after each of
    its two steps into the caller's device buffers, overwritten by every
    replay. They equal the means of the same cases stepped one step at a time
    (FP64 reductions, deterministic)."""
    from paper_1003_4548_gb300 import capi
    cs = cases()[:2]
    streams = [torch.cuda.Stream() for _ in range(2 * len(cs) + 1)]
    batched = [make(torch, m, ppe, wm, k, streams[k]) for m, ppe, wm, k in cs]
    alone = [make(torch, m, ppe, wm, k, streams[len(cs) + k]) for m, ppe, wm, k in cs]
    dts = [cfl_dt(m, cfl=0.5, k0=1e-3) for m, _, _, _ in cs]
    bufs = [torch.zeros((g.nt, 5), dtype=torch.float64, device="cuda") for g in batched for _ in range(2)]
    nbytes = [g.nt * 5 * 8 for g in batched]
    with pytest.raises(capi.PdfError):  # a byte count that is not the field's size
        capi.Batch(batched, dts, streams[-1].cuda_stream,
                   outputs=("elem_mean", [t.data_ptr() for t in bufs], [b + 8 for b in nbytes]))
    b = capi.Batch(batched, dts, streams[-1].cuda_stream,
                   outputs=("elem_mean", [t.data_ptr() for t in bufs], nbytes))
    expect = []
    for g, dt in zip(alone, dts):
        per = []
        for _ in range(4):
            g.step(dt, 1)
            g.sync()
            per.append(g.field("elem_mean"))
        expect.append(per)
    for pair in range(2):
        b.step(2)
        b.sync()
        for j in range(len(batched)):
            for k in range(2):
                got = bufs[2 * j + k].cpu().numpy()
                assert np.array_equal(got, expect[j][2 * pair + k]), (j, pair, k)
    for g in batched:
        assert g.step_index == 4
    b.close()
    for g in batched + alone:
        g.close()


def test_batch_outputs_particle_field_fp32(torch):
    """pdf_batch_create_out with a particle field of FP32 contexts: the graph
    converts u to FP64 through the context's conversion buffer after each
    step. Each step's copy holds the same values as the same case stepped
    on its own (exact integer reductions in the fp32 mode, so the particle
    order inside an element does not change the statistics; the copies are
    compared as sorted values because that order may differ)."""
    from paper_1003_4548_gb300 import capi
    cs = cases()[:2]
    streams = [torch.cuda.Stream() for _ in range(2 * len(cs) + 1)]
    batched = [make(torch, m, ppe, wm, k, streams[k], precision="fp32") for m, ppe, wm, k in cs]
    alone = [make(torch, m, ppe, wm, k, streams[len(cs) + k], precision="fp32") for m, ppe, wm, k in cs]
    dts = [cfl_dt(m, cfl=0.5, k0=1e-3) for m, _, _, _ in cs]
    bufs = [torch.zeros(g.num_particles, dtype=torch.float64, device="cuda") for g in batched for _ in range(2)]
    nbytes = [g.num_particles * 8 for g in batched]
    b = capi.Batch(batched, dts, streams[-1].cuda_stream, outputs=("u", [t.data_ptr() for t in bufs], nbytes))
    expect = []
    for g, dt in zip(alone, dts):
        per = []
        for _ in range(4):
            g.step(dt, 1)
            g.sync()
            per.append(np.sort(g.field("u")))
        expect.append(per)
    for pair in range(2):
        b.step(2)
        b.sync()
        for j in range(len(batched)):
            for k in range(2):
                got = np.sort(bufs[2 * j + k].cpu().numpy())
                assert np.array_equal(got, expect[j][2 * pair + k]), (j, pair, k)
    b.close()
    for g in batched + alone:
        g.close()


@pytest.mark.parametrize("wm", ["wf", "er"])
def test_batched_case_matches_oracle(torch, wm):
    """A case with its own Philox key (case_id = 3) advanced by the batch graph
    (one replay: two steps) against the oracle with the same key, from the
    same seeded ensemble: element ids exact except within 1e-9 of an edge,
    the state within 1e-12 of the oracle's (FP64)."""
    from oracle.oracle import Oracle
    from paper_1003_4548_gb300 import capi
    from tests.conftest import oracle_params_for
    mesh, ppe, _, _ = cases()[0 if wm == "wf" else 1]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    # both FE solves converge to 1e-14, far below the 1e-12 state bar
    g = make(torch, mesh, ppe, wm, 3, streams[0], cg_tol=1e-14)
    o = Oracle(oracle_params_for(mesh, wall_model=0 if wm == "wf" else 1, C0=2.1, seed=103, case_id=3,
                                 cg_tol=1e-14, cg_maxit=20000), mesh)
    g.sync()
    o.set_particles(g.particles(), step=g.step_index)
    o.estimate_stats()
    dt = cfl_dt(mesh, cfl=0.5, k0=1e-3)
    b = capi.Batch([g], [dt], streams[1].cuda_stream)
    b.step(2)
    b.sync()
    o.step(dt, 2)
    G, O = by_id(g), o.particles()
    oo = np.argsort(O["id"])
    O = {k: v[oo] for k, v in O.items()}
    assert np.array_equal(G["id"], O["id"])
    from tests.test_gpu_parity import assert_state_close, edge_distance
    near = np.abs(edge_distance(mesh, O)) < 1e-9
    assert np.all((G["elem"] == O["elem"]) | near)
    assert_state_close(G, O, 1e-12, skip=near)
    b.close()
    g.close()
