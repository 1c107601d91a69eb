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
    obs = adjoint.Observation(obs_np.node, obs_np.weight)
    sources = torch.from_numpy(F).cuda()
    # synthetic data from the perturbed log-modulus field, 5% noise
    m_true = torch.from_numpy(mg.adjoint_true_logE(m)).cuda()
    a1 = torch.ones(16, dtype=torch.float64, device="cuda")
    M.set_log_young(m_true)
    G, _, _ = M.solve(sources, **OPTS)
    clean = obs.apply(torch.einsum("nkc,k->nc", G, a1))
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
        assert an == pytest.approx(fd, rel=1e-4, abs=1e-6 * abs(J0))


@pytest.mark.gpu
@pytest.mark.slow
def test_adjoint_24cube_fd_50_directions():
    """The 24^3-hexahedra box (82,944 elements, 352,947 DOF), 1,000 observations:
    gradient w.r.t. 82,944 log-moduli and 16 amplitudes vs central differences at
    h = 1e-6 on 50 random unit directions."""
    from paper_1710_08679_gb300 import adjoint
    m, M, obs, obs_np, sources, d, logE0, a = setup_problem(24, 1000)
    J0, g_logE, g_a = adjoint.misfit_and_grad(M, logE0, a, sources, obs, d, OPTS)
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
    # 1e-9 |J0| on every direction; directions whose derivative is that small are
    # judged against the floor, all others to 1e-4 relative
    bad = [(e, f) for e, f in errs if e > 1e-4 * f + 1e-7 * abs(J0)]
    assert not bad, (bad, abs(J0))
