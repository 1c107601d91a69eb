"""Adjoint gradient of a surface misfit (torch.autograd.Function over libfe)
against central finite differences and against the oracle's assembled adjoint.

J(m, a) = 1/2 |P u - d|^2, K_bc(m) u_k = f_k (16 double couples), u = sum a_k u_k,
m_e = log E_e. Finite differences at h = 1e-6 need solves far tighter than 1e-8
(a 1e-8 solve leaves ~1e-2 FD error), so these solves use tol = 1e-13.
"""
import numpy as np
import pytest

from _util import ensure_lib, rel_l2

import oracle
from paper_1710_08679_gb300 import meshgen as mg

torch = pytest.importorskip("torch")

OPTS = dict(solver="fcg_mixed", tol=1e-13)


def setup_problem(n, n_obs, seed=2):
    ensure_lib()
    from paper_1710_08679_gb300 import adjoint, fe
    m = mg.adjoint_box(n=n)
    F = mg.adjoint_sources(m)
    obs_np = mg.surface_observations(m, n_obs, (500.0, 7500.0), seed)
    M = fe.Mesh.from_mesh(m)
    obs = adjoint.Observation(M, obs_np.node, obs_np.weight)
    sources = torch.from_numpy(F).cuda()
    # synthetic data from the perturbed log-modulus field, 5% noise
    m_true = torch.from_numpy(mg.adjoint_true_logE(m)).cuda()
    a1 = torch.ones(16, dtype=torch.float64, device="cuda")
    M.set_log_young(m_true)
    G, _, _ = M.solve(sources, **OPTS)
    clean = obs.apply(M.combine_cases(G, a1))
    rms = torch.sqrt(torch.mean(clean ** 2))
    d = clean + 0.05 * rms * torch.from_numpy(mg.noise(tuple(clean.shape), seed)).cuda()
    logE0 = torch.from_numpy(np.log(m.young)).cuda()
    return m, M, obs, obs_np, sources, d, logE0, a1


@pytest.mark.gpu
def test_adjoint_vs_finite_differences_and_oracle():
    from paper_1710_08679_gb300 import adjoint
    m, M, obs, obs_np, sources, d, logE0, a = setup_problem(8, 200)
    J0, g_logE, g_a = adjoint.misfit_and_grad(M, logE0, a, sources, obs, d, OPTS)
    assert J0 > 0
    # oracle: assembled K_bc, direct solves, assembled adjoint gradient
    K = oracle.assemble(m)
    F = sources.cpu().numpy()
    G = oracle.direct_solve(K, F)
    u = np.einsum("nkc,k->nc", G, a.cpu().numpy())
    Pm = obs_np.matrix(m.n_nodes)
    r = Pm @ u.reshape(-1) - d.cpu().numpy().reshape(-1)
    rhs = (Pm.T @ r).reshape(m.n_nodes, 1, 3) * m.free[:, None, :]
    lam = oracle.direct_solve(K, rhs)
    g_ref = oracle.adjoint_grad(m, u[:, None, :], lam)
    ga_ref = np.einsum("nkc,nc->k", F * m.free[:, None, :], lam[:, 0])
    assert rel_l2(g_logE.cpu().numpy(), g_ref) <= 1e-8
    assert rel_l2(g_a.cpu().numpy(), ga_ref) <= 1e-8
    # central differences along random unit directions over (logE, a)
    h = 1e-6
    V = mg.unit_directions(6, m.n_elem + 16, seed=2)
    for v in V:
        ve = torch.from_numpy(v[:m.n_elem]).cuda()
        va = torch.from_numpy(v[m.n_elem:]).cuda()
        Jp = adjoint.misfit(M, logE0 + h * ve, a + h * va, sources, obs, d, OPTS)
        Jm = adjoint.misfit(M, logE0 - h * ve, a - h * va, sources, obs, d, OPTS)
        fd = (Jp - Jm) / (2 * h)
        an = float(g_logE @ ve + g_a @ va)
        assert an == pytest.approx(fd, rel=1e-4, abs=1e-8 * abs(J0))


@pytest.mark.gpu
@pytest.mark.slow
def test_adjoint_24cube_fd_50_directions_and_oracle():
    """The 24^3-hexahedra box (82,944 elements, 352,947 DOF), 1,000 observations:
    gradient w.r.t. 82,944 log-moduli and 16 amplitudes against the oracle's
    assembled adjoint gradient (oracle PCG solves to 1e-13) and against central
    differences at h = 1e-6 on 50 random unit directions."""
    from paper_1710_08679_gb300 import adjoint
    m, M, obs, obs_np, sources, d, logE0, a = setup_problem(24, 1000)
    J0, g_logE, g_a = adjoint.misfit_and_grad(M, logE0, a, sources, obs, d, OPTS)
    # oracle: assembled K_bc, block-Jacobi PCG for the 16 Green's functions and the
    # adjoint state, assembled adjoint gradient
    K = oracle.assemble(m)
    F = sources.cpu().numpy()
    # (the oracle stops on its recursive residual; its true residual lands within
    # FP64 rounding of 1e-13)
    G, _, relG = oracle.pcg(K, F, tol=1e-13)
    assert relG.max() <= 1e-12
    u = np.einsum("nkc,k->nc", G, a.cpu().numpy())
    Pm = obs_np.matrix(m.n_nodes)
    r = Pm @ u.reshape(-1) - d.cpu().numpy().reshape(-1)
    rhs = (Pm.T @ r).reshape(m.n_nodes, 1, 3) * m.free[:, None, :]
    lam, _, relL = oracle.pcg(K, rhs, tol=1e-13)
    assert relL.max() <= 1e-12
    g_ref = oracle.adjoint_grad(m, u[:, None, :], lam)
    ga_ref = np.einsum("nkc,nc->k", F * m.free[:, None, :], lam[:, 0])
    assert rel_l2(g_logE.cpu().numpy(), g_ref) <= 1e-8
    assert rel_l2(g_a.cpu().numpy(), ga_ref) <= 1e-8
    h = 1e-6
    V = mg.unit_directions(50, m.n_elem + 16, seed=2)
    errs = []
    for v in V:
        ve = torch.from_numpy(v[:m.n_elem]).cuda()
        va = torch.from_numpy(v[m.n_elem:]).cuda()
        Jp = adjoint.misfit(M, logE0 + h * ve, a + h * va, sources, obs, d, OPTS)
        Jm = adjoint.misfit(M, logE0 - h * ve, a - h * va, sources, obs, d, OPTS)
        fd = (Jp - Jm) / (2 * h)
        an = float(g_logE @ ve + g_a @ va)
        errs.append((abs(an - fd), abs(fd)))
    # solves at relative residual 1e-13 leave J with an absolute noise of a few
    # 1e-15 |J0|, which central differences at h = 1e-6 turn into a floor of a few
    # 1e-9 |J0|: the absolute bar is 1e-8 |J0| (about three times that floor),
    # all other directions are judged to 1e-4 relative
    floor = max(e for e, _ in errs) / abs(J0)
    bad = [(e, f) for e, f in errs if e > 1e-4 * f + 1e-8 * abs(J0)]
    assert not bad, (bad, abs(J0), floor)


@pytest.mark.gpu
def test_observation_and_vector_steps_match_numpy():
    """fe_obs_apply / fe_obs_adjoint against the sparse observation matrix,
    fe_combine_cases and fe_case_dots against einsum, on a 3-case batch."""
    ensure_lib()
    from paper_1710_08679_gb300 import fe
    m = mg.adjoint_box(n=6)
    M = fe.Mesh.from_mesh(m)
    obs_np = mg.surface_observations(m, 150, (500.0, 7500.0), 3)
    obs = fe.Observation(M, obs_np.node, obs_np.weight)
    Pm = obs_np.matrix(m.n_nodes)
    rng = np.random.default_rng(4)
    U = rng.standard_normal((m.n_nodes, 3, 3))
    Uo = obs.apply(torch.from_numpy(U).cuda()).cpu().numpy()
    for r in range(3):
        assert rel_l2(Uo[:, r], (Pm @ U[:, r].reshape(-1)).reshape(-1, 3)) <= 1e-14
    g = rng.standard_normal((obs.n_obs, 3, 3))
    A = obs.adjoint(torch.from_numpy(g).cuda()).cpu().numpy()
    for r in range(3):
        ref = (Pm.T @ g[:, r].reshape(-1)).reshape(-1, 3) * m.free
        assert rel_l2(A[:, r], ref) <= 1e-14
    a = rng.standard_normal(3)
    u = M.combine_cases(torch.from_numpy(U).cuda(), torch.from_numpy(a).cuda()).cpu().numpy()
    assert rel_l2(u, np.einsum("nkc,k->nc", U, a)) <= 1e-14
    lam = rng.standard_normal((m.n_nodes, 3))
    dots = M.case_dots(torch.from_numpy(U).cuda(), torch.from_numpy(lam).cuda()).cpu().numpy()
    assert rel_l2(dots, np.einsum("nkc,nc->k", U * m.free[:, None, :], lam)) <= 1e-13


@pytest.mark.gpu
def test_observation_rejects_bad_node_ids():
    ensure_lib()
    from paper_1710_08679_gb300 import fe
    m = mg.adjoint_box(n=2)
    M = fe.Mesh.from_mesh(m)
    node = np.zeros((4, 6), dtype=np.int32)
    node[2, 3] = m.n_nodes          # one past the last node
    with pytest.raises(fe.FeError, match="out of range"):
        fe.Observation(M, node, np.ones((4, 6)))


@pytest.mark.gpu
def test_backward_uses_the_forward_moduli():
    """A set_log_young between forward and backward (here a second model) does not
    change the gradient: backward restores the moduli of its forward pass."""
    from paper_1710_08679_gb300 import adjoint
    m, M, obs, obs_np, sources, d, logE0, a = setup_problem(6, 100)
    J_ref, g_ref, ga_ref = adjoint.misfit_and_grad(M, logE0, a, sources, obs, d, OPTS)
    AdjointSolve = adjoint.make_adjoint_solve()
    logE = logE0.detach().clone().requires_grad_(True)
    aa = a.detach().clone().requires_grad_(True)
    u_obs = AdjointSolve.apply(logE, aa, M, sources, obs, OPTS)
    M.set_log_young(logE0 + 0.3)   # the mesh now holds other moduli
    J = 0.5 * torch.sum((u_obs - d) ** 2)
    J.backward()
    assert rel_l2(logE.grad.cpu().numpy(), g_ref.cpu().numpy()) <= 1e-9
    assert rel_l2(aa.grad.cpu().numpy(), ga_ref.cpu().numpy()) <= 1e-9
