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


def block_rel_err(got, ref):
    """Largest error of a 3x3 block relative to the largest entry of the same
    reference block (blocks of fixed nodes are the identity, those of free nodes
    scale like 1/stiffness, so one global scale would hide the free ones)."""
    import numpy as np
    got = np.asarray(got, dtype=np.float64).reshape(-1, 9)
    ref = np.asarray(ref, dtype=np.float64).reshape(-1, 9)
    scale = np.maximum(np.abs(ref).max(axis=1), 1e-300)
    return float((np.abs(got - ref).max(axis=1) / scale).max())
