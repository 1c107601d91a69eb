"""GPU parity of inner loop level 2 (the aggregation coarsening of the TET4 level,
Algorithm 1(a)) through the C ABI -- fe_level2_info, fe_level2_apply,
fe_level2_restrict, fe_level2_prolong, fe_level2_block_jacobi and the FCG_AMG
solver -- against the oracle's aggregate / galerkin_agg / fcg_ml.

The aggregation is integer work and must match exactly; A2 products and the
transfers are FP32 (bar 2e-6 on FP32-rounded inputs); solutions compare to the
direct solve, iteration counts to the oracle's three-level solve within a
margin."""
import numpy as np
import pytest

from _util import block_rel_err, ensure_lib, rel_l2

import oracle
from paper_1710_08679_gb300 import meshgen as mg

torch = pytest.importorskip("torch")

TOL32 = 2e-6


@pytest.fixture(scope="module")
def meshes():
    ensure_lib()
    from paper_1710_08679_gb300 import fe
    out = {}
    for name, m in {"box8": mg.plain_box(),
                    "crust10x8x5": mg.crust_block(shape=(10, 8, 5), h=1000.0, jitter=0.15, seed=2)[0]}.items():
        cm = oracle.coarse_mesh(m)
        K1 = oracle.assemble4(cm)
        agg = oracle.aggregate(K1)
        A2, free2 = oracle.galerkin_agg(K1, cm.free, agg)
        out[name] = (m, cm, K1, agg, A2, free2, fe.Mesh.from_mesh(m))
    return out


def cuda32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["box8", "crust10x8x5"])
def test_aggregation_matches_oracle_exactly(meshes, name):
    m, cm, K1, agg, A2, free2, M = meshes[name]
    na, got = M.level2_info()
    assert na == A2.n_nodes
    assert np.array_equal(got, agg)


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["box8", "crust10x8x5"])
@pytest.mark.parametrize("R", [1, 5, 16])
def test_level2_operator_and_transfers_match_oracle(meshes, name, R):
    m, cm, K1, agg, A2, free2, M = meshes[name]
    x2 = mg.random_vectors(A2.n_nodes, R, seed=60 + R).astype(np.float32).astype(np.float64)
    y2 = M.level2_apply(cuda32(x2)).double().cpu().numpy()
    assert rel_l2(y2, oracle.spmv(A2, x2)) <= TOL32
    # P2^T and P2 written out from the oracle's aggregation
    r4 = mg.random_vectors(cm.vertex.size, R, seed=70 + R).astype(np.float32).astype(np.float64)
    ref2 = np.zeros((A2.n_nodes, R, 3))
    np.add.at(ref2, agg, r4 * cm.free[:, None, :])
    assert rel_l2(M.level2_restrict(cuda32(r4)).double().cpu().numpy(), ref2) <= TOL32
    ref4 = x2[agg] * cm.free[:, None, :]
    assert np.array_equal(M.level2_prolong(cuda32(x2)).double().cpu().numpy(), ref4)


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["box8", "crust10x8x5"])
def test_level2_block_jacobi_matches_oracle(meshes, name):
    m, cm, K1, agg, A2, free2, M = meshes[name]
    ref = oracle.block_jacobi(A2)
    assert block_rel_err(M.level2_block_jacobi().cpu().numpy(), ref) <= 1e-10


@pytest.mark.gpu
@pytest.mark.parametrize("use_graph", [True, False])
def test_three_level_solve_matches_oracle(meshes, use_graph):
    m, cm, K1, agg, A2, free2, M = meshes["crust10x8x5"]
    K = oracle.assemble(m)
    F = mg.random_vectors(m.n_nodes, 4, seed=12) * 1e9 * m.free[:, None, :]
    F[:, 2] = 0.0                                             # a zero case
    u, stats, st = M.solve(torch.from_numpy(F).cuda(), solver="fcg_amg", tol=1e-8, use_graph=use_graph)
    assert st == 0, stats
    u = u.cpu().numpy()
    ud = oracle.direct_solve(K, F)
    _, outer, i0, i1, i2, _ = oracle.fcg_ml(K, F, cm, m.free, K1=K1, levels=3)
    for r in range(4):
        if r == 2:
            assert np.all(u[:, 2] == 0.0) and stats[2]["outer"] == 0 and stats[2]["inner2"] == 0
            continue
        assert stats[r]["relres"] <= 1e-8 and stats[r]["inner2"] > 0
        assert rel_l2(u[:, r], ud[:, r]) <= 1e-6
        assert abs(stats[r]["outer"] - int(outer[r])) <= max(2, 0.25 * outer[r])


@pytest.mark.gpu
def test_three_level_solve_many(meshes):
    m, cm, K1, agg, A2, free2, M = meshes["box8"]
    K = oracle.assemble(m)
    lx, ly, lz = m.lattice_shape()
    F = np.stack([mg.double_couple(m, (lx // 2 - 2 + k, ly // 2, lz // 2 + (k % 2)), 1e12) for k in range(5)])
    u, stats, st, R_used = M.solve_many(torch.from_numpy(F).cuda(), R_slots=2, solver="fcg_amg", tol=1e-8)
    assert st == 0 and R_used == 2
    ud = oracle.direct_solve(K, np.ascontiguousarray(F.transpose(1, 0, 2)))
    for c in range(5):
        assert stats[c]["relres"] <= 1e-8 and stats[c]["inner2"] > 0
        assert rel_l2(u.cpu().numpy()[c], ud[:, c]) <= 1e-6
