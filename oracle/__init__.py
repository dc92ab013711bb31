"""TEST INFRASTRUCTURE ONLY: the plain FP64 CPU oracle (see oracle.py)."""
