"""The resumable many-case driver (paper_1710_08679_gb300.many) on the GPU: a run
over 7 double-couple cases stopped after its first chunk resumes with the pending
cases only, and every stored solution matches the oracle's direct solve."""
import numpy as np
import pytest

from _util import ensure_lib, rel_l2

import oracle
from paper_1710_08679_gb300 import meshgen as mg

torch = pytest.importorskip("torch")


class Stop(Exception):
    pass


@pytest.mark.gpu
def test_interrupted_many_case_run_resumes_and_matches_oracle(tmp_path):
    ensure_lib()
    from paper_1710_08679_gb300 import fe, many
    m = mg.plain_box()
    K = oracle.assemble(m)
    M = fe.Mesh.from_mesh(m)
    lx, ly, lz = m.lattice_shape()
    F = np.stack([mg.double_couple(m, (lx // 2 - 3 + k, ly // 2, lz // 2 + (k % 3) - 1), 1e12) for k in range(7)])
    f = torch.from_numpy(F).cuda()

    def stop(part):
        raise Stop

    with pytest.raises(Stop):
        many.solve_many_resumable(M, f, str(tmp_path), chunk=3, R_slots=2, on_chunk=stop, key="plain box 8^3")
    u, stats, solved = many.solve_many_resumable(M, f, str(tmp_path), chunk=3, R_slots=2, key="plain box 8^3")
    assert solved == [3, 4, 5, 6]
    ud = oracle.direct_solve(K, np.ascontiguousarray(F.transpose(1, 0, 2)))
    for c in range(7):
        assert stats[c]["status"] == 0 and stats[c]["relres"] <= 1e-8, (c, stats[c])
        assert rel_l2(u[c], ud[:, c]) <= 1e-6, c
    _, _, again = many.solve_many_resumable(M, f, str(tmp_path), chunk=3, R_slots=2, key="plain box 8^3")
    assert again == []
