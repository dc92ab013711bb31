import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def wf_small_mesh():
    from canyon_inputs.configs import WORKLOADS, build_mesh
    return build_mesh(WORKLOADS["canyon_wf_small"])


@pytest.fixture(scope="session")
def tiny_wf_mesh():
    """A coarse wall-function canyon (a few hundred triangles)."""
    from canyon_inputs.mesh import canyon_mesh
    from canyon_inputs.configs import yplus30
    return canyon_mesh(offset=yplus30(), h=0.15, seed=3)


@pytest.fixture(scope="session")
def tiny_er_mesh():
    """A coarse wall-resolved canyon graded toward the walls."""
    from canyon_inputs.mesh import canyon_mesh
    return canyon_mesh(offset=0.0, h=0.12, y1=0.01, growth=1.3, seed=5)


def oracle_params_for(mesh, **over):
    """Oracle parameters for a canyon mesh (source at street level, canyon centre)."""
    from oracle.oracle import default_params
    p = default_params(wall_offset=mesh["offset"], x0=mesh["L"] / 2,
                       y0=mesh["y_floor"], period=mesh["L"], y_roof=mesh["H"])
    p.update(over)
    return p
