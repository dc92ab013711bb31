"""GB300 (sm_103a) particle-in-cell joint velocity-frequency-scalar PDF solver
for a periodic street canyon (Bakosi, Franzese & Boybeyi, Sections 2-3).

The compute path is the CUDA library built from csrc/ behind the C ABI of
include/pdf_canyon.h; ``capi`` is its ctypes binding.
"""
from .capi import Canyon, PdfError, default_params, lib  # noqa: F401
from .workload import canyon_params  # noqa: F401
