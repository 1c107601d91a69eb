"""fe_block_jacobi_noalloc: the block-Jacobi preconditioner built without any
device allocation, for callers that cannot allocate where they need it
(latency-critical loops that must not take the allocator's lock, processes whose
device memory is held by another allocator's pool). Its scratch is a fixed file-scope device array shared by every call, so
the test checks two calls in a row (the second must not see the first's
leftovers), a second mesh, and the size limit.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from _util import block_rel_err, ensure_lib

from paper_1710_08679_gb300 import meshgen as mg

torch = pytest.importorskip("torch")

TOL = 1e-12   # the tolerance of the block-Jacobi parity test


def _blocks(lib, M, fn):
    out = torch.full((M.n_nodes, 3, 3), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = getattr(lib, fn)(M.handle, ctypes.c_void_p(out.data_ptr()), stream)
    torch.cuda.synchronize()
    return st, out.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_matches_block_jacobi_twice_in_a_row():
    lib = ensure_lib()
    from paper_1710_08679_gb300 import fe
    for m in (mg.plain_box(), mg.crust_block(shape=(9, 5, 4), h=1000.0, jitter=0.15, seed=2)[0]):
        M = fe.Mesh.from_mesh(m)
        st, ref = _blocks(lib, M, "fe_block_jacobi")
        assert st == fe.FE_OK
        for _ in range(2):
            st, got = _blocks(lib, M, "fe_block_jacobi_noalloc")
            assert st == fe.FE_OK, lib.fe_last_error()
            assert np.all(np.isfinite(got))
            assert block_rel_err(got, ref) <= TOL


@pytest.mark.gpu
def test_noalloc_rejects_meshes_above_its_limit():
    lib = ensure_lib()
    from paper_1710_08679_gb300 import fe
    m = mg.box_mesh((30, 30, 30), (3000.0, 3000.0, 3000.0))      # 226,981 nodes > 131,072
    M = fe.Mesh.from_mesh(m)
    out = torch.zeros((M.n_nodes, 3, 3), dtype=torch.float64, device="cuda")
    st = lib.fe_block_jacobi_noalloc(M.handle, ctypes.c_void_p(out.data_ptr()), None)
    assert st == fe.FE_EINVAL
    assert b"at most 131072 nodes" in lib.fe_last_error()
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
