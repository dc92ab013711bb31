"""The C-ABI library loads and exports every entry point of include/*.h, its
defaults are the paper's constants, and mesh validation rejects malformed
meshes before touching the GPU (no compute call here)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def golden_constants():
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "table2_constants.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(pdf_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1003_4548_gb300 import capi
    L = capi.lib()
    names = declared_functions()
    assert len(names) >= 19
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(capi.EXPORTS) <= names


def test_defaults_are_the_paper_constants():
    from paper_1003_4548_gb300 import capi
    from oracle.oracle import default_params
    g = golden_constants()
    p = capi.default_params()
    o = default_params()
    for k, v in g.items():
        assert getattr(p, k) == v, k
        assert o[k] == v, k
    assert ctypes.sizeof(capi.pdf_params) == 344  # 34 doubles, 8 int32, the seed, 6 int32, 1 double


def _tiny_mesh():
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    tri = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    tag = np.array([[1, 0, 1], [1, 1, 0]], np.int32)
    return dict(xy=xy, tri=tri, edge_tag=tag, periodic_pair=-np.ones(4, np.int32))


@pytest.mark.parametrize("break_it", ["cw", "tag", "pair", "unmatched"])
def test_malformed_mesh_rejected(break_it):
    from paper_1003_4548_gb300 import capi
    m = _tiny_mesh()
    if break_it == "cw":
        m["tri"] = m["tri"][:, [0, 2, 1]].copy()
    elif break_it == "tag":
        m["edge_tag"][0, 0] = 7
    elif break_it == "pair":
        m["periodic_pair"][0] = 1
    else:
        m["edge_tag"][0, 1] = 1  # shared edge tagged as a wall on one side only
    with pytest.raises(capi.PdfError) as ei:
        capi.Canyon(capi.default_params(), m)
    assert ei.value.code in (-2, -1)
