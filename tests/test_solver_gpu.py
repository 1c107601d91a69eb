"""GPU solver parity (fe_pcg_solve, fe_block_jacobi, fe_adjoint_grad through the
C ABI) against the CPU oracle.

Solutions are unique (K_bc is SPD) but iterates and atomic summation order are
not, so the checks compare solutions, true residuals and iteration counts within
a margin, never iterates.
"""
import numpy as np
import pytest

from _util import block_rel_err, ensure_lib, rel_l2

import oracle
from paper_1710_08679_gb300 import meshgen as mg

torch = pytest.importorskip("torch")


def gpu_mesh(m):
    ensure_lib()
    from paper_1710_08679_gb300 import fe
    return fe.Mesh.from_mesh(m)


@pytest.fixture(scope="module")
def box8():
    m = mg.plain_box()
    K = oracle.assemble(m)
    return m, K, gpu_mesh(m)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.gpu
def test_block_jacobi_matches_oracle(box8):
    m, K, M = box8
    ref = oracle.block_jacobi(K)
    got = M.block_jacobi().cpu().numpy()
    assert block_rel_err(got, ref) <= 1e-12


@pytest.mark.gpu
def test_pcg64_plain_box(box8):
    m, K, M = box8
    f = mg.plain_box_rhs(m)
    u, stats, st = M.solve(cuda(f), solver="pcg64", tol=1e-8)
    assert st == 0 and stats[0]["status"] == 0
    assert stats[0]["relres"] <= 1e-8
    ud = oracle.direct_solve(K, f)
    assert rel_l2(u.cpu().numpy(), ud) <= 1e-6
    _, it, _ = oracle.pcg(K, f, tol=1e-8)
    assert abs(stats[0]["outer"] - int(it[0])) <= max(3, 0.05 * it[0])


@pytest.mark.gpu
@pytest.mark.parametrize("use_graph", [True, False])
def test_fcg_mixed_plain_box(box8, use_graph):
    m, K, M = box8
    f = mg.plain_box_rhs(m)
    u, stats, st = M.solve(cuda(f), solver="fcg_mixed", tol=1e-8, use_graph=use_graph)
    assert st == 0
    assert stats[0]["relres"] <= 1e-8
    ud = oracle.direct_solve(K, f)
    assert rel_l2(u.cpu().numpy(), ud) <= 1e-6
    _, outer, inner, _ = oracle.fcg_mixed(K, f, tol=1e-8)
    assert abs(stats[0]["outer"] - int(outer[0])) <= max(2, 0.25 * outer[0])
    assert stats[0]["inner"] <= 30 * stats[0]["outer"]


def _three_cases(m):
    lx, ly, lz = m.lattice_shape()
    f = mg.plain_box_rhs(m)
    fa = mg.double_couple(m, (lx // 2 - 4, ly // 2 + 2, lz // 2 + 3), 1e12)[:, None, :]
    fg = (np.tile(np.array([0.0, 0.0, -1e9]), (m.n_nodes, 1)) * m.free)[:, None, :]
    return np.concatenate([f, fa, fg], axis=1)


@pytest.mark.gpu
def test_fcg_inner_counts_match_oracle(box8):
    """Per-case outer and inner iteration counts of the GPU's Algorithm 1 (three
    cases in one batch, the paper's loop settings) against the oracle's. The two
    round differently (GPU atomics, per-block partial sums), so the counts may
    differ by a step: margin 1 outer iteration and 10 % + 3 inner steps per case."""
    m, K, M = box8
    F = _three_cases(m)
    _, stats, st = M.solve(cuda(F), solver="fcg_mixed", tol=1e-8)
    assert st == 0
    _, outer, inner, _ = oracle.fcg_mixed(K, F, tol=1e-8)
    for c in range(3):
        assert abs(stats[c]["outer"] - int(outer[c])) <= 1, (c, stats[c], outer, inner)
        assert abs(stats[c]["inner"] - int(inner[c])) <= 0.1 * inner[c] + 3, (c, stats[c], outer, inner)


@pytest.mark.gpu
@pytest.mark.parametrize("n0", [30, 7])
def test_fcg_inner_loop_runs_n0_steps_when_eps_is_zero(box8, n0):
    m, K, M = box8
    F = _three_cases(m)
    _, stats, st = M.solve(cuda(F), solver="fcg_mixed", tol=1e-8, eps_inner=0.0, n_inner=n0)
    assert st == 0
    for c in range(3):
        assert stats[c]["inner"] == n0 * stats[c]["outer"], (c, stats[c])


@pytest.mark.gpu
def test_fcg_inner_stop_rule_is_on_the_squared_ratio(box8):
    """As the oracle's pin: in the first outer iteration the inner loop takes no step
    when rho0^2 <= eps < rho0 (rho0 = ||f - K M^-1 f|| / ||f|| from scipy and numpy),
    and at least one when eps < rho0^2."""
    m, K, M = box8
    f = mg.plain_box_rhs(m)
    A = K.to_scipy().tocsr()
    Minv = np.stack([np.linalg.inv(A[3 * i:3 * i + 3, 3 * i:3 * i + 3].toarray()) for i in range(m.n_nodes)])
    fv = f[:, 0, :]
    rho0 = np.linalg.norm(fv.reshape(-1) - A @ np.einsum("nij,nj->ni", Minv, fv).reshape(-1)) / np.linalg.norm(fv)
    _, s1, _ = M.solve(cuda(f), solver="fcg_mixed", tol=1e-8, max_outer=1, eps_inner=rho0 ** 1.5,
                       raise_on_fail=False)
    _, s2, _ = M.solve(cuda(f), solver="fcg_mixed", tol=1e-8, max_outer=1, eps_inner=rho0 ** 2.5,
                       raise_on_fail=False)
    assert s1[0]["outer"] == 1 and s1[0]["inner"] == 0
    assert s2[0]["outer"] == 1 and s2[0]["inner"] >= 1


@pytest.mark.gpu
def test_fcg_inner_stop_ignores_converged_cases(box8):
    """A case that starts converged (initial guess = its direct solution) leaves
    another case's counts unchanged (the inner stop is judged over active cases);
    one step of rounding slack for the GPU's atomic summation order."""
    m, K, M = box8
    F = _three_cases(m)[:, :2]
    ua = oracle.direct_solve(K, F[:, 1:2])
    _, s1, st1 = M.solve(cuda(F[:, :1]), solver="fcg_mixed", tol=1e-8)
    U0 = np.concatenate([np.zeros_like(ua), ua], axis=1)
    _, s2, st2 = M.solve(cuda(F), u0=cuda(U0), solver="fcg_mixed", tol=1e-8)
    assert st1 == 0 and st2 == 0
    assert s2[1]["outer"] == 0 and s2[1]["relres"] <= 1e-8
    assert abs(s2[0]["outer"] - s1[0]["outer"]) <= 1
    assert abs(s2[0]["inner"] - s1[0]["inner"]) <= 3


@pytest.mark.gpu
def test_fcg_zero_inner_steps_tracks_pcg(box8):
    m, K, M = box8
    f = mg.plain_box_rhs(m)
    _, sp, _ = M.solve(cuda(f), solver="pcg64", tol=1e-8)
    _, sf, st = M.solve(cuda(f), solver="fcg_mixed", tol=1e-8, n_inner=0)
    assert st == 0 and sf[0]["inner"] == 0
    assert abs(sf[0]["outer"] - sp[0]["outer"]) <= max(3, 0.05 * sp[0]["outer"])


@pytest.mark.gpu
@pytest.mark.parametrize("solver", ["pcg64", "fcg_mixed"])
def test_batched_uneven_cases_with_zero_rhs(box8, solver):
    """Four cases of different difficulty plus an all-zero case: per-case masking."""
    m, K, M = box8
    lx, ly, lz = m.lattice_shape()
    cases = [mg.plain_box_rhs(m)[:, 0],
             mg.double_couple(m, (lx // 2 - 5, ly // 2 + 3, lz - 3), 1e12),
             np.zeros((m.n_nodes, 3)),
             mg.random_vectors(m.n_nodes, 1, seed=3)[:, 0] * 1e9 * m.free]
    f = np.stack(cases, axis=1)
    u, stats, st = M.solve(cuda(f), solver=solver, tol=1e-8)
    assert st == 0, stats
    u = u.cpu().numpy()
    ud = oracle.direct_solve(K, f)
    for r in (0, 1, 3):
        assert stats[r]["relres"] <= 1e-8
        assert rel_l2(u[:, r], ud[:, r]) <= 1e-6
    assert np.all(u[:, 2] == 0.0) and stats[2]["outer"] == 0
    its = [stats[r]["outer"] for r in (0, 1, 3)]
    assert len(set(its)) > 1          # the cases really stopped at different iterations


@pytest.mark.gpu
def test_iteration_cap_reports_noconv(box8):
    m, K, M = box8
    f = mg.plain_box_rhs(m)
    u, stats, st = M.solve(cuda(f), solver="fcg_mixed", max_outer=2, raise_on_fail=False)
    from paper_1710_08679_gb300 import fe
    assert st == fe.FE_ENOCONV
    assert stats[0]["status"] == fe.FE_ENOCONV and stats[0]["outer"] == 2
    assert stats[0]["relres"] > 1e-8 and np.isfinite(stats[0]["relres"])


@pytest.mark.gpu
def test_warm_start_from_solution(box8):
    m, K, M = box8
    f = mg.plain_box_rhs(m)
    u, s1, _ = M.solve(cuda(f), solver="fcg_mixed", tol=1e-9)
    u2, s2, st = M.solve(cuda(f), u0=u, solver="fcg_mixed", tol=1e-8)
    assert st == 0 and s2[0]["outer"] == 0 and s2[0]["relres"] <= 1e-8


@pytest.mark.gpu
def test_slip_sources_on_ragged_crust():
    """Split-node unit-slip sources: f = -sum_{e in E+} K_e s_e computed by the GPU
    (fe_ebe_apply on the hanging-wall sub-mesh) and by the oracle (assembled sub-mesh
    matrix), then a batched mixed solve against the oracle's direct solve."""
    m, iface = mg.crust_block(shape=(12, 6, 6), h=1000.0, jitter=0.15, seed=1)
    cases = mg.patch_grid_cases(m, iface, n_along=2, spacing=2000.0, size=2000.0)
    cases = [c for c in cases if len(c.elems)][:3]
    assert len(cases) >= 2
    K = oracle.assemble(m)
    M = gpu_mesh(m)
    from paper_1710_08679_gb300 import fe
    f_gpu, f_ref = [], []
    for c in cases:
        sub = mg.Mesh(coords=m.coords, conn=m.conn[c.elems], young=m.young[c.elems], poisson=m.poisson[c.elems],
                      free=np.ones_like(m.free), shape=m.shape, h=m.h, lengths=m.lengths)
        Ms = fe.Mesh.from_mesh(sub)
        f_gpu.append(-(Ms.ebe(cuda(c.slip[:, None, :])).cpu().numpy()[:, 0]) * m.free)
        Ks = oracle.assemble(sub, apply_bc=False)
        f_ref.append(-oracle.spmv(Ks, c.slip[:, None, :])[:, 0] * m.free)
    f_gpu = np.stack(f_gpu, axis=1)
    f_ref = np.stack(f_ref, axis=1)
    assert rel_l2(f_gpu, f_ref) <= 1e-12
    u, stats, st = M.solve(cuda(f_gpu), solver="fcg_mixed", tol=1e-8)
    assert st == 0
    ud = oracle.direct_solve(K, f_ref)
    for r in range(len(cases)):
        assert stats[r]["relres"] <= 1e-8
        assert rel_l2(u.cpu().numpy()[:, r], ud[:, r]) <= 1e-5


@pytest.mark.gpu
def test_adjoint_grad_matches_oracle(box8):
    m, K, M = box8
    u = mg.random_vectors(m.n_nodes, 3, seed=21)
    lam = mg.random_vectors(m.n_nodes, 3, seed=22)
    g = M.adjoint_grad(cuda(u), cuda(lam)).cpu().numpy()
    ref = oracle.adjoint_grad(m, u, lam)
    assert rel_l2(g, ref) <= 1e-12


@pytest.mark.gpu
def test_set_log_young_changes_operator(box8):
    m, K, _ = box8
    M = gpu_mesh(m)
    rng = np.random.default_rng(5)
    le = np.log(m.young) + 0.1 * rng.standard_normal(m.n_elem)
    M.set_log_young(cuda(le))
    x = mg.random_vectors(m.n_nodes, 2, seed=8)
    y = M.ebe(cuda(x)).cpu().numpy()
    K2 = oracle.assemble(m, young=np.exp(le))
    assert rel_l2(y, oracle.spmv(K2, x)) <= 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("solver,R_slots", [("fcg_mixed", 4), ("pcg64", 3), ("fcg_mixed", 0)])
def test_solve_many_streams_cases_through_slots(box8, solver, R_slots):
    """11 cases (double couples at different places, a zero case, random loads)
    through at most R_slots slots: every case is solved to 1e-8 and matches the
    oracle's direct solve; a converged slot is refilled with the next case."""
    m, K, M = box8
    lx, ly, lz = m.lattice_shape()
    cases = []
    for k in range(8):
        cases.append(mg.double_couple(m, (lx // 2 - 4 + k, ly // 2 + (k % 3) - 1, lz // 2 + (k % 4)), 1e12))
    cases.append(np.zeros((m.n_nodes, 3)))
    rng = np.random.default_rng(4)
    for k in range(2):
        cases.append(rng.standard_normal((m.n_nodes, 3)) * 1e9 * m.free)
    F = np.stack(cases, axis=0)                        # [n_cases, N, 3]
    u, stats, st, R_used = M.solve_many(cuda(F), R_slots=R_slots, solver=solver, tol=1e-8)
    assert st == 0, stats
    assert 1 <= R_used <= (R_slots if R_slots else 32)
    u = u.cpu().numpy()
    ud = oracle.direct_solve(K, np.ascontiguousarray(F.transpose(1, 0, 2)))
    for c in range(F.shape[0]):
        if c == 8:
            assert np.all(u[c] == 0.0) and stats[c]["relres"] == 0.0
            continue
        assert stats[c]["status"] == 0 and stats[c]["relres"] <= 1e-8, (c, stats[c])
        assert rel_l2(u[c], ud[:, c]) <= 1e-6, c


@pytest.mark.gpu
@pytest.mark.parametrize("solver", ["pcg64", "fcg_mixed", "fcg_mg"])
def test_all_zero_batch_returns_at_once(box8, solver):
    """Every right-hand side zero: u = 0 for every case, no iteration."""
    m, K, M = box8
    f = np.zeros((m.n_nodes, 5, 3))
    u, stats, st = M.solve(cuda(f), u0=cuda(np.ones((m.n_nodes, 5, 3))), solver=solver, tol=1e-8)
    assert st == 0
    assert np.all(u.cpu().numpy() == 0.0)
    assert all(s["outer"] == 0 and s["relres"] == 0.0 for s in stats)


@pytest.mark.gpu
def test_64_cases_in_one_batch(box8):
    """R = 64 cases at once through the two-level solver (the ABI's largest R)."""
    m, K, M = box8
    rng = np.random.default_rng(64)
    F = rng.standard_normal((m.n_nodes, 64, 3)) * 1e9 * m.free[:, None, :]
    u, stats, st = M.solve(cuda(F), solver="fcg_mg", tol=1e-8)
    assert st == 0
    ud = oracle.direct_solve(K, F)
    for r in range(64):
        assert stats[r]["relres"] <= 1e-8
        assert rel_l2(u.cpu().numpy()[:, r], ud[:, r]) <= 1e-6


@pytest.mark.gpu
@pytest.mark.slow
@pytest.mark.parametrize("solver", ["fcg_mg", "fcg_amg"])
def test_full_size_two_level_solve_sampled_residual(solver):
    """The batched solves the benchmark times: 16 unit-slip patches on the 70x70x35
    crust block (4,234,653 DOF), levels 1 and 0 (and levels 2, 1 and 0), to true
    relative residual 1e-8.
    The right-hand sides come from the oracle (assembled hanging-wall sub-meshes);
    the residual f - K_bc u is recomputed by the oracle's element-by-element row
    sums at every node of the patches' elements and at 2,000 random nodes: each
    entry is bounded by ||f - K_bc u|| <= 1e-8 ||f|| (x2 for the oracle's own
    rounding). One case is compared with the plain FP64 PCG solve."""
    ensure_lib()
    from paper_1710_08679_gb300 import fe
    m, iface = mg.crust_block()
    cases = mg.patch_grid_cases(m, iface)[:16]
    R = len(cases)
    assert R == 16
    f = np.zeros((m.n_nodes, R, 3))
    for r, c in enumerate(cases):
        sub = mg.Mesh(coords=m.coords, conn=m.conn[c.elems], young=m.young[c.elems], poisson=m.poisson[c.elems],
                      free=np.ones_like(m.free), shape=m.shape, h=m.h, lengths=m.lengths)
        Ks = oracle.assemble(sub, apply_bc=False)
        f[:, r] = -oracle.spmv(Ks, c.slip[:, None, :])[:, 0] * m.free
    M = fe.Mesh.from_mesh(m)
    u, stats, st = M.solve(cuda(f), solver=solver, tol=1e-8)
    assert st == 0 and all(s["relres"] <= 1e-8 for s in stats)
    un = u.cpu().numpy()
    rng = np.random.default_rng(11)
    near = np.unique(np.concatenate([m.conn[c.elems].ravel() for c in cases]))
    nodes = np.unique(np.concatenate([near, rng.integers(0, m.n_nodes, 2000)]))
    res = f[nodes] - oracle.sampled_product(m, un, nodes)
    for r in range(R):
        assert np.abs(res[:, r]).max() <= 2e-8 * np.linalg.norm(f[:, r]), r
    u1, s1, st1 = M.solve(cuda(f[:, :1]), solver="pcg64", tol=1e-8)
    assert st1 == 0 and s1[0]["relres"] <= 1e-8
    assert rel_l2(u1.cpu().numpy()[:, 0], un[:, 0]) <= 1e-4


@pytest.mark.gpu
@pytest.mark.parametrize("solver", ["fcg_mixed", "fcg_mg"])
def test_solver_with_paired_and_colour_kernels(solver):
    """The solvers do not depend on the kernel choice: with the paired-arithmetic
    kernel for the FP32 products and the colour-by-colour kernel for the FP64 ones
    (R = 8), the batch reaches 1e-8 and matches the oracle's direct solve."""
    m = mg.plain_box()
    K = oracle.assemble(m)
    M = gpu_mesh(m)
    R = 8
    M.set_variant(R, "f32", 4, 24)
    M.set_variant(R, "f64", 5, 0)
    assert M.get_variant(R, "f32")[0] == 4 and M.get_variant(R, "f64")[0] == 5
    f = mg.random_vectors(m.n_nodes, R, seed=41) * m.free[:, None, :]
    u, stats, st = M.solve(cuda(f), solver=solver, tol=1e-8)
    assert st == 0 and all(s["relres"] <= 1e-8 for s in stats)
    ud = oracle.direct_solve(K, f)
    for r in range(R):
        assert rel_l2(u.cpu().numpy()[:, r], ud[:, r]) <= 1e-5


@pytest.mark.gpu
@pytest.mark.slow
def test_full_size_many_case_driver_sampled_residual():
    """The many-case workload at full size (120x120x60 hexahedra, 6 layers,
    21,083,403 DOF): the first 12 of its 96 unit-slip cases through fe_solve_many
    with the memory-sized slot count and the two-level solver, right-hand sides
    from the oracle (assembled hanging-wall sub-meshes). Every case reaches 1e-8;
    for three cases the oracle recomputes f - K_bc u at every node of the patch's
    elements and at 1,000 random nodes (each entry bounded by 1e-8 ||f||, x2 for
    the oracle's rounding)."""
    ensure_lib()
    from paper_1710_08679_gb300 import fe
    m, iface = mg.crust_block(shape=(120, 120, 60), h=1000.0, jitter=0.10, seed=3, n_layers=6)
    cases = mg.many_cases(m, iface, n_patches=48, seed=3)[:12]
    F = np.zeros((len(cases), m.n_nodes, 3))
    for c, sc in enumerate(cases):
        if len(sc.elems) == 0:
            continue
        sub = mg.Mesh(coords=m.coords, conn=m.conn[sc.elems], young=m.young[sc.elems], poisson=m.poisson[sc.elems],
                      free=np.ones_like(m.free), shape=m.shape, h=m.h, lengths=m.lengths)
        F[c] = -oracle.spmv(oracle.assemble(sub, apply_bc=False), sc.slip[:, None, :])[:, 0] * m.free
    M = fe.Mesh.from_mesh(m)
    u, stats, st, R_used = M.solve_many(cuda(F), R_slots=0, solver="fcg_mg", tol=1e-8)
    assert st == 0 and R_used >= 1
    assert all(s["relres"] <= 1e-8 for s in stats)
    rng = np.random.default_rng(12)
    for c in (0, 5, 11):
        if not F[c].any():
            continue
        near = np.unique(m.conn[cases[c].elems].ravel())
        nodes = np.unique(np.concatenate([near, rng.integers(0, m.n_nodes, 1000)]))
        uc = u[c].cpu().numpy()[:, None, :]
        res = F[c][nodes] - oracle.sampled_product(m, uc, nodes)[:, 0]
        assert np.abs(res).max() <= 2e-8 * np.linalg.norm(F[c]), c
