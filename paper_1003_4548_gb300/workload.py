"""Parameters of a canyon run for the C ABI, from a mesh and a workload description.

The source sits at street level in the canyon centre (Section 3); the wall
offset, the periodic length and the roof height come from the mesh.
"""
from __future__ import annotations

from .capi import PRECISION, default_params


def canyon_params(mesh: dict, *, wall_model: str = "wf", precision: str = "fp64", C0: float | None = None,
                  bins=(2, 2, 2), seed: int = 0, k0: float = 1e-3, **over):
    p = default_params()
    p.wall_model = 0 if wall_model == "wf" else 1
    p.precision = PRECISION[precision]
    if C0 is not None:
        p.C0 = C0
    p.nb1, p.nb2, p.nb3 = bins
    p.seed = seed
    p.k0 = k0
    p.wall_offset = mesh["offset"]
    p.x0 = mesh["L"] / 2
    p.y0 = mesh["y_floor"]
    p.period = mesh["L"]
    p.y_roof = mesh["H"]
    for k, v in over.items():
        setattr(p, k, v)
    return p
