"""Shared helpers of the test suite (no arithmetic of the method here)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def ensure_lib():
    """Build libfe.so if needed and load it."""
    from paper_1710_08679_gb300 import build, fe
    build.build()
    return fe.load()


def rel_l2(a, b):
    import numpy as np
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
