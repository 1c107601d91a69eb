"""Failure detection without a GPU fault: each kind of bounded device-side wait
(the warp-specialised EBE kernel's mbarrier wait, the persistent inner loop's
grid-wide barrier) is made to run out on a wait that nothing ends; the kernel
returns, the mesh's status word reports FE_ETIMEOUT once, and the context stays
usable (a product afterwards still matches the oracle)."""
import numpy as np
import pytest

from _util import ensure_lib, rel_l2

import oracle
from paper_1710_08679_gb300 import meshgen as mg

torch = pytest.importorskip("torch")


@pytest.mark.gpu
@pytest.mark.parametrize("which", ["mbarrier", "grid"])
def test_bounded_wait_gives_up_and_reports_timeout(which):
    ensure_lib()
    from paper_1710_08679_gb300 import fe
    m = mg.plain_box(n=3, jitter=0.1, seed=0)
    M = fe.Mesh.from_mesh(m)
    M.device_status()                              # clear before the test
    M.wait_selftest(which, cycles=1 << 21)         # about a millisecond
    with pytest.raises(fe.FeError) as err:
        M.device_status()
    assert err.value.status == fe.FE_ETIMEOUT
    M.device_status()                              # read and cleared: clear again
    x = mg.random_vectors(m.n_nodes, 4, seed=3)
    y = M.ebe(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel_l2(y, oracle.spmv(oracle.assemble(m), x)) <= 1e-12
