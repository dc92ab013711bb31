"""The allocation-free counting sort (pdf_sort_by_element_static, scratch in a
fixed device array of the library) against the context's own re-sort:
pdf_set_particles groups the particles by host element, and the sorted
element and id fields it leaves must be what the static sort's permutation
gives, on two calls in a row (the second call must find its counts cleared).
"""
import numpy as np
import pytest

from canyon_inputs.configs import yplus30
from canyon_inputs.mesh import canyon_mesh

pytestmark = pytest.mark.gpu


def _static_sort(torch, capi, elem, nt):
    n = len(elem)
    stream = torch.cuda.current_stream()
    elem_d = torch.from_numpy(np.ascontiguousarray(elem, np.int32)).cuda()
    perm_d = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    off_d = torch.full((nt + 1,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    capi.sort_by_element_static(elem_d.data_ptr(), n, nt, perm_d.data_ptr(), off_d.data_ptr(), stream.cuda_stream)
    return perm_d.cpu().numpy()[:n], off_d.cpu().numpy()


def test_static_sort_matches_context_sort_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1003_4548_gb300 import Canyon, canyon_params, capi
    mesh = canyon_mesh(offset=yplus30(), h=0.1, seed=5)
    g = Canyon(canyon_params(mesh, wall_model="wf", precision="fp64", C0=2.1, seed=7), mesh,
               stream=torch.cuda.current_stream().cuda_stream)
    g.seed_particles(40)
    base = g.particles()
    n, nt = len(base["x"]), g.nt
    assert n > 256 * 40  # several blocks of the count and scatter kernels
    rng = np.random.default_rng(11)
    for _ in range(2):
        order = rng.permutation(n)
        st = {k: v[order] for k, v in base.items() if k != "bin"}
        g.set_particles(st, step=0)  # the existing path: sorts by element inside the context
        ctx_elem, ctx_id = g.field("elem"), g.field("id")
        perm, off = _static_sort(torch, capi, st["elem"], nt)
        counts = np.bincount(st["elem"], minlength=nt)
        assert off[0] == 0 and np.array_equal(np.diff(off), counts)
        assert np.array_equal(np.sort(perm), np.arange(n))
        assert np.array_equal(st["elem"][perm], ctx_elem)
        # inside a segment the order is not fixed: compare (element, id) pairs
        mine = (st["elem"][perm].astype(np.int64) << 32) | st["id"][perm].astype(np.int64)
        theirs = (ctx_elem.astype(np.int64) << 32) | ctx_id.astype(np.int64)
        assert np.array_equal(np.sort(mine), np.sort(theirs))
    g.close()


def test_static_sort_limits_and_recovery():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1003_4548_gb300 import capi
    elem = np.array([0, 2, 1, 2, 2, 0], np.int32)
    with pytest.raises(capi.PdfError) as ei:
        _static_sort(torch, capi, elem, capi.SORT_STATIC_MAX_ELEMENTS + 1)
    assert ei.value.code == -10 and "maximum" in str(ei.value)
    # an index outside [0, nt) is clamped in bounds by the kernels and reported
    with pytest.raises(capi.PdfError) as ei:
        _static_sort(torch, capi, np.array([0, 5, 1], np.int32), 3)
    assert ei.value.code == -1
    # the next call starts from cleared counts and status
    perm, off = _static_sort(torch, capi, elem, 3)
    assert off.tolist() == [0, 2, 3, 6]
    assert sorted(perm[:2].tolist()) == [0, 5] and perm[2] == 2 and sorted(perm[3:].tolist()) == [1, 3, 4]
    # the largest element count and an empty ensemble
    perm, off = _static_sort(torch, capi, np.zeros(0, np.int32), capi.SORT_STATIC_MAX_ELEMENTS)
    assert not off.any()
