"""GPU parity of the TET4 coarse level (inner loop level 1 of Algorithm 1)
through the C ABI: fe_coarse_info, fe_ebe4_apply, fe_coarse_restrict,
fe_coarse_prolong, fe_coarse_block_jacobi and the FCG_MG solver, against the
oracle's coarse_mesh / assemble4 / restrict / prolong / block_jacobi / fcg_mg.

Bars: relative L2 <= 1e-12 in FP64 and <= 2e-6 in FP32 (inputs rounded to FP32
first) for the operators; transfers in FP64 are sums of at most a handful of
halves and compare to 1e-15. Solutions compare to the oracle's direct solve;
iteration counts to the oracle's two-level FCG within a margin (atomic summation
order makes iterates differ, never the solution)."""
import numpy as np
import pytest

from _util import block_rel_err, ensure_lib, rel_l2

import oracle
from paper_1710_08679_gb300 import meshgen as mg

torch = pytest.importorskip("torch")

TOL64, TOL32 = 1e-12, 2e-6


def _meshes():
    return {"box8": mg.plain_box(),
            "crust9x5x4": mg.crust_block(shape=(9, 5, 4), h=1000.0, jitter=0.15, seed=2)[0]}


@pytest.fixture(scope="module")
def meshes():
    ensure_lib()
    from paper_1710_08679_gb300 import fe
    out = {}
    for name, m in _meshes().items():
        cm = oracle.coarse_mesh(m)
        out[name] = (m, cm, fe.Mesh.from_mesh(m))
    return out


def cuda(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["box8", "crust9x5x4"])
def test_coarse_numbering_matches_oracle(meshes, name):
    m, cm, M = meshes[name]
    n4, vertex = M.coarse_info()
    assert n4 == cm.vertex.size
    assert np.array_equal(vertex, cm.vertex)


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["box8", "crust9x5x4"])
@pytest.mark.parametrize("R", [1, 3, 16])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_ebe4_matches_assembled_tet4_operator(meshes, name, R, dtype):
    m, cm, M = meshes[name]
    K1 = oracle.assemble4(cm)
    x = mg.random_vectors(cm.vertex.size, R, seed=300 + R)
    if dtype == "f32":
        x = x.astype(np.float32).astype(np.float64)
    tdt = torch.float32 if dtype == "f32" else torch.float64
    y = M.ebe4(cuda(x, tdt)).double().cpu().numpy()
    assert rel_l2(y, oracle.spmv(K1, x)) <= (TOL32 if dtype == "f32" else TOL64)


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["box8", "crust9x5x4"])
@pytest.mark.parametrize("R", [1, 3, 4, 8, 16, 32])
def test_assembled_coarse_operator_matches_oracle(meshes, name, R):
    """R a multiple of 4 takes the sliced copy of the matrix (8 rows per slice; a
    warp covers 4, 2, 1 or half a slice at R = 4, 8, 16, 32), other R the plain
    block-CSR arrays."""
    m, cm, M = meshes[name]
    K1 = oracle.assemble4(cm)
    x = mg.random_vectors(cm.vertex.size, R, seed=310 + R).astype(np.float32).astype(np.float64)
    y = M.coarse_apply(cuda(x, torch.float32)).double().cpu().numpy()
    assert rel_l2(y, oracle.spmv(K1, x)) <= TOL32


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["box8", "crust9x5x4"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("R", [5, 8])
def test_transfers_match_oracle(meshes, name, dtype, R):
    m, cm, M = meshes[name]
    tdt = torch.float32 if dtype == "f32" else torch.float64
    tol = 2e-6 if dtype == "f32" else 1e-15
    r10 = mg.random_vectors(m.n_nodes, R, seed=41)
    u4 = mg.random_vectors(cm.vertex.size, R, seed=42)
    if dtype == "f32":
        r10 = r10.astype(np.float32).astype(np.float64)
        u4 = u4.astype(np.float32).astype(np.float64)
    r4 = M.coarse_restrict(cuda(r10, tdt)).double().cpu().numpy()
    ref4 = oracle.restrict(cm, r10) * cm.free[:, None, :]
    assert rel_l2(r4, ref4) <= tol
    assert np.all(r4[cm.free[:, None, :].repeat(R, 1) == 0] == 0.0)
    u10 = M.coarse_prolong(cuda(u4, tdt)).double().cpu().numpy()
    ref10 = oracle.prolong(cm, u4) * m.free[:, None, :]
    assert rel_l2(u10, ref10) <= tol
    assert np.all(u10[m.free[:, None, :].repeat(R, 1) == 0] == 0.0)


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["box8", "crust9x5x4"])
def test_coarse_block_jacobi_matches_oracle(meshes, name):
    m, cm, M = meshes[name]
    ref = oracle.block_jacobi(oracle.assemble4(cm))
    got = M.coarse_block_jacobi().cpu().numpy()
    assert block_rel_err(got, ref) <= TOL64


@pytest.mark.gpu
def test_galerkin_identity_at_full_size():
    """On the 70 x 70 x 35 crust block (1.4M nodes) no oracle product fits in
    seconds; the coarse operator is checked through a property that holds at any
    size: on free coarse DOFs, P1^T K_bc P1 x4 = K1_bc x4 for masked x4 (a linear
    field is exact in TET10), all products on the GPU in FP64."""
    ensure_lib()
    from paper_1710_08679_gb300 import fe
    m, _ = mg.crust_block()
    M = fe.Mesh.from_mesh(m)
    n4, vertex = M.coarse_info()
    free4 = m.free[vertex]
    x4 = mg.random_vectors(n4, 2, seed=9) * free4[:, None, :]
    X4 = cuda(x4)
    lhs = M.coarse_restrict(M.ebe(M.coarse_prolong(X4))).cpu().numpy()
    rhs = M.ebe4(X4).cpu().numpy()
    mask = free4[:, None, :].repeat(2, 1) == 1
    assert rel_l2(lhs[mask], rhs[mask]) <= 1e-11
    # the assembled FP32 operator and the FP32 element-by-element product agree
    # with the FP64 product
    x32 = torch.from_numpy(x4.astype(np.float32)).cuda()
    y_asm = M.coarse_apply(x32).double().cpu().numpy()
    y_ebe = M.ebe4(x32).double().cpu().numpy()
    y64 = M.ebe4(x32.double()).cpu().numpy()
    assert rel_l2(y_asm, y64) <= TOL32 and rel_l2(y_ebe, y64) <= TOL32
    # R = 16: the sliced copy of the matrix against the FP64 element-by-element product
    x16 = (mg.random_vectors(n4, 16, seed=10) * free4[:, None, :]).astype(np.float32)
    x16t = torch.from_numpy(x16).cuda()
    assert rel_l2(M.coarse_apply(x16t).double().cpu().numpy(), M.ebe4(x16t.double()).cpu().numpy()) <= TOL32
    # sampled rows against element matrices of the oracle
    rng = np.random.default_rng(3)
    conn4 = np.searchsorted(vertex, m.conn[:, :4])
    rows = rng.choice(n4, 40, replace=False)
    for a in rows:
        elems = np.nonzero((conn4 == a).any(axis=1))[0]
        acc = np.zeros((2, 3))
        for e in elems:
            ke = oracle.tet4_stiffness(m.coords[m.conn[e, :4]], m.young[e], m.poisson[e])
            k = int(np.nonzero(conn4[e] == a)[0][0])
            xe = x4[conn4[e]]                      # [4, 2, 3]
            for r in range(2):
                acc[r] += ke[3 * k:3 * k + 3] @ xe[:, r, :].reshape(12)
        ref = np.where(free4[a][None, :] == 1, acc, x4[a])
        assert np.allclose(rhs[a], ref, rtol=1e-11, atol=1e-11 * np.abs(rhs).max())


@pytest.fixture(scope="module")
def box8_solve(meshes):
    m, cm, M = meshes["box8"]
    K = oracle.assemble(m)
    f = mg.plain_box_rhs(m)
    return m, cm, M, K, f


@pytest.mark.gpu
@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("coarse_op", ["assembled", "ebe"])
def test_fcg_mg_plain_box(box8_solve, use_graph, coarse_op):
    m, cm, M, K, f = box8_solve
    u, stats, st = M.solve(cuda(f), solver="fcg_mg", tol=1e-8, use_graph=use_graph, coarse_op=coarse_op)
    assert st == 0
    assert stats[0]["relres"] <= 1e-8
    ud = oracle.direct_solve(K, f)
    assert rel_l2(u.cpu().numpy(), ud) <= 1e-6
    _, outer, inner0, inner1, _ = oracle.fcg_mg(K, f, coarse=cm, free=m.free, tol=1e-8)
    assert abs(stats[0]["outer"] - int(outer[0])) <= max(2, 0.25 * outer[0])
    assert stats[0]["inner1"] > 0
    assert stats[0]["inner"] <= 30 * stats[0]["outer"]
    # the coarse level moves level-0 work down (Sec. 2), as in the oracle
    _, s1, _ = M.solve(cuda(f), solver="fcg_mixed", tol=1e-8, use_graph=use_graph)
    assert stats[0]["inner"] < s1[0]["inner"] / 2
    assert abs(stats[0]["inner"] - int(inner0[0])) <= max(10, 0.3 * inner0[0])


@pytest.mark.gpu
def test_fcg_mg_zero_level1_steps_still_converges(box8_solve):
    """n_inner1 = 0: level 1 only restricts and prolongs the block-Jacobi guess,
    which is then P1 P1^T Mbar^-1 rbar; the solve still converges."""
    m, cm, M, K, f = box8_solve
    u, stats, st = M.solve(cuda(f), solver="fcg_mg", tol=1e-8, n_inner1=0)
    assert st == 0 and stats[0]["inner1"] == 0 and stats[0]["relres"] <= 1e-8
    ud = oracle.direct_solve(K, f)
    assert rel_l2(u.cpu().numpy(), ud) <= 1e-6


@pytest.mark.gpu
@pytest.mark.parametrize("solver", ["fcg_mg"])
def test_fcg_mg_batched_uneven_cases_with_zero_rhs(box8_solve, solver):
    m, cm, M, K, f = box8_solve
    lx, ly, lz = m.lattice_shape()
    cases = [f[:, 0],
             mg.double_couple(m, (lx // 2 - 5, ly // 2 + 3, lz - 3), 1e12),
             np.zeros((m.n_nodes, 3)),
             mg.random_vectors(m.n_nodes, 1, seed=3)[:, 0] * 1e9 * m.free]
    F = np.stack(cases, axis=1)
    u, stats, st = M.solve(cuda(F), solver=solver, tol=1e-8)
    assert st == 0, stats
    u = u.cpu().numpy()
    ud = oracle.direct_solve(K, F)
    for r in (0, 1, 3):
        assert stats[r]["relres"] <= 1e-8
        assert rel_l2(u[:, r], ud[:, r]) <= 1e-6
    assert np.all(u[:, 2] == 0.0) and stats[2]["outer"] == 0 and stats[2]["inner1"] == 0


@pytest.mark.gpu
def test_fcg_mg_on_ragged_crust(meshes):
    m, cm, M = meshes["crust9x5x4"]
    K = oracle.assemble(m)
    F = mg.random_vectors(m.n_nodes, 3, seed=17) * 1e9 * m.free[:, None, :]
    u, stats, st = M.solve(cuda(F), solver="fcg_mg", tol=1e-8)
    assert st == 0
    ud = oracle.direct_solve(K, F)
    for r in range(3):
        assert stats[r]["relres"] <= 1e-8 and stats[r]["inner1"] > 0
        assert rel_l2(u.cpu().numpy()[:, r], ud[:, r]) <= 1e-6
    _, outer, _, _, _ = oracle.fcg_mg(K, F, coarse=cm, free=m.free, tol=1e-8)
    for r in range(3):
        assert abs(stats[r]["outer"] - int(outer[r])) <= max(2, 0.25 * outer[r])


@pytest.mark.gpu
def test_solve_many_with_coarse_level(box8_solve):
    m, cm, M, K, f = box8_solve
    lx, ly, lz = m.lattice_shape()
    cases = [mg.double_couple(m, (lx // 2 - 3 + k, ly // 2, lz // 2 + (k % 3)), 1e12) for k in range(6)]
    F = np.stack(cases, axis=0)
    u, stats, st, R_used = M.solve_many(cuda(F), R_slots=4, solver="fcg_mg", tol=1e-8)
    assert st == 0 and R_used == 4
    ud = oracle.direct_solve(K, np.ascontiguousarray(F.transpose(1, 0, 2)))
    for c in range(F.shape[0]):
        assert stats[c]["relres"] <= 1e-8 and stats[c]["inner1"] > 0
        assert rel_l2(u.cpu().numpy()[c], ud[:, c]) <= 1e-6


@pytest.mark.gpu
def test_set_log_young_rebuilds_coarse_preconditioner(meshes):
    ensure_lib()
    from paper_1710_08679_gb300 import fe
    m = mg.plain_box()
    cm = oracle.coarse_mesh(m)
    M = fe.Mesh.from_mesh(m)
    before = M.coarse_block_jacobi().cpu().numpy()
    M.coarse_apply(cuda(np.zeros((cm.vertex.size, 1, 3)), torch.float32))   # assembled before the change
    le = np.log(m.young) + 0.2 * np.random.default_rng(6).standard_normal(m.n_elem)
    M.set_log_young(cuda(le))
    after = M.coarse_block_jacobi().cpu().numpy()
    ref = oracle.block_jacobi(oracle.assemble4(cm, young=np.exp(le)))
    assert block_rel_err(after, ref) <= TOL64
    assert block_rel_err(after, before) > 1e-3
    x = mg.random_vectors(cm.vertex.size, 2, seed=8)
    K1 = oracle.assemble4(cm, young=np.exp(le))
    y = M.ebe4(cuda(x)).cpu().numpy()
    assert rel_l2(y, oracle.spmv(K1, x)) <= TOL64
    x32 = x.astype(np.float32).astype(np.float64)
    y32 = M.coarse_apply(cuda(x32, torch.float32)).double().cpu().numpy()
    assert rel_l2(y32, oracle.spmv(K1, x32)) <= TOL32
    # the sliced copy (R a multiple of 4) is refreshed with the new values too
    x4 = mg.random_vectors(cm.vertex.size, 4, seed=18).astype(np.float32).astype(np.float64)
    y4 = M.coarse_apply(cuda(x4, torch.float32)).double().cpu().numpy()
    assert rel_l2(y4, oracle.spmv(K1, x4)) <= TOL32


def _uneven_cases(m, R, seed):
    """R right-hand sides of different scales and shapes (random loads on the free
    DOFs), so that the cases converge at different outer iterations."""
    F = mg.random_vectors(m.n_nodes, R, seed=seed) * m.free[:, None, :]
    return F * (1e9 * 10.0 ** (np.arange(R) % 5))[None, :, None]


@pytest.mark.gpu
@pytest.mark.parametrize("solver", ["fcg_mg", "fcg_amg"])
@pytest.mark.parametrize("R", [4, 8, 16, 32])
def test_persistent_inner_loop_matches_per_step_launches(meshes, solver, R):
    """The level-1 (and level-2) inner loop as one cooperative kernel against the
    same loop issued as one launch per vector pass: the same Algorithm 1(b)
    arithmetic, so the same counts (up to the order of the FP64 atomic sums) and
    solutions that agree with each other and with the oracle's direct solve."""
    m, cm, M = meshes["crust9x5x4"]
    F = _uneven_cases(m, R, seed=40 + R)
    res = {}
    for kind in ("persistent", "steps"):
        u, stats, st = M.solve(cuda(F), solver=solver, tol=1e-8, inner_kernel=kind)
        assert st == 0, (kind, stats)
        M.device_status()                                # raises if a barrier wait ran out
        res[kind] = (u.cpu().numpy(), stats)
    (up, sp), (us, ss) = res["persistent"], res["steps"]
    K = oracle.assemble(m)
    ud = oracle.direct_solve(K, F)
    for r in range(R):
        assert sp[r]["relres"] <= 1e-8 and sp[r]["inner1"] > 0
        assert abs(sp[r]["outer"] - ss[r]["outer"]) <= 1
        assert abs(sp[r]["inner1"] - ss[r]["inner1"]) <= max(3, 0.05 * ss[r]["inner1"])
        if solver == "fcg_amg":
            assert sp[r]["inner2"] > 0 and abs(sp[r]["inner2"] - ss[r]["inner2"]) <= max(5, 0.05 * ss[r]["inner2"])
        assert rel_l2(up[:, r], ud[:, r]) <= 1e-6
        assert rel_l2(up[:, r], us[:, r]) <= 1e-6


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["persistent", "steps"])
@pytest.mark.parametrize("n1", [1, 7])
def test_level1_loop_runs_n1_steps_when_eps1_is_zero(meshes, kind, n1):
    """eps_inner1 = 0: the stop rule never holds, so every outer iteration runs
    exactly n_inner1 level-1 steps for every active case (Algorithm 1(b) with
    eps = 0), in the persistent kernel as in the per-step launches."""
    m, cm, M = meshes["crust9x5x4"]
    F = _uneven_cases(m, 8, seed=5)
    F[:, 3] = 0.0                                     # a zero case stays inactive: no steps counted
    u, stats, st = M.solve(cuda(F), solver="fcg_mg", tol=1e-8, eps_inner1=0.0, n_inner1=n1, inner_kernel=kind)
    assert st == 0
    for r in range(8):
        if r == 3:
            assert stats[r]["outer"] == 0 and stats[r]["inner1"] == 0
        else:
            assert stats[r]["relres"] <= 1e-8
            assert stats[r]["inner1"] == n1 * stats[r]["outer"], (r, stats[r])
