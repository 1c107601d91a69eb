"""Pins of the CPU oracle against facts fixed by the mathematics (not by itself).

Each test below would fail for a plausible mistake in the oracle: a dropped
term, a wrong sign or index, a transposed operand, a wrong elasticity matrix, a
wrong quadrature weight, a wrong boundary treatment or a wrong CG update.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1710_08679_gb300 import meshgen as mg


def lame(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def jittered_element(seed=0):
    """A random straight-sided TET10 (corners jittered from a unit-ish tet)."""
    rng = np.random.default_rng(seed)
    c = np.array([[0, 0, 0], [1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]]) * 700.0 + rng.uniform(-100, 100, (4, 3))
    pts = list(c) + [0.5 * (c[a] + c[b]) for a, b in mg.EDGES]
    return np.array(pts)


def tet_volume(xe):
    return np.linalg.det(np.stack([xe[1] - xe[0], xe[2] - xe[0], xe[3] - xe[0]])) / 6.0


def rigid_modes(xe):
    """6 rigid-body displacement fields on the element nodes, [6, 30]."""
    out = []
    for t in range(3):
        u = np.zeros((10, 3)); u[:, t] = 1.0; out.append(u.reshape(-1))
    for w in np.eye(3):
        out.append(np.cross(w, xe).reshape(-1))
    return np.array(out)


# ---------------------------------------------------------------------------
# element level
# ---------------------------------------------------------------------------

def test_element_rigid_body_modes_and_rank():
    xe = jittered_element(1)
    Ke = oracle.element_stiffness(xe, 5.0e10, 0.27)
    scale = np.abs(Ke).max()
    for u in rigid_modes(xe):
        assert np.abs(Ke @ u).max() <= 1e-12 * scale * np.abs(u).max() * 30
    w = np.linalg.eigvalsh(Ke)
    assert np.all(np.abs(w[:6]) <= 1e-12 * w[-1])
    assert np.all(w[6:] > 1e-6 * w[-1])        # rank 24: no spurious zero-energy mode


def test_element_symmetric():
    Ke = oracle.element_stiffness(jittered_element(2), 3.0e10, 0.3)
    assert np.abs(Ke - Ke.T).max() <= 1e-14 * np.abs(Ke).max()


def test_element_linear_energy_closed_form():
    """u = A x (constant strain): u^T K_e u = V (lam tr(eps)^2 + 2 mu eps:eps)."""
    rng = np.random.default_rng(3)
    xe = jittered_element(3)
    E, nu = 4.0e10, 0.25
    Ke = oracle.element_stiffness(xe, E, nu)
    A = rng.standard_normal((3, 3)) * 1e-3
    u = (xe @ A.T).reshape(-1)
    eps = 0.5 * (A + A.T)
    lam, mu = lame(E, nu)
    energy = tet_volume(xe) * (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps))
    assert u @ Ke @ u == pytest.approx(energy, rel=1e-12)


def _monomial_integral(xe, f_of_L):
    """Exact integral over the tetrahedron of a polynomial in volume coordinates
    given as {(a0,a1,a2,a3): coeff}: int L0^a0 L1^a1 L2^a2 L3^a3 = 6V a0!a1!a2!a3!/(sum+3)!"""
    V = tet_volume(xe)
    tot = 0.0
    for exps, cf in f_of_L.items():
        num = math.prod(math.factorial(a) for a in exps)
        tot += cf * 6 * V * num / math.factorial(sum(exps) + 3)
    return tot


def test_element_quadratic_energy_closed_form():
    """u quadratic: u^T K_e u = int (lam tr(eps)^2 + 2 mu eps:eps) dV computed by exact
    monomial integration in volume coordinates (independent of any quadrature)."""
    rng = np.random.default_rng(4)
    xe = jittered_element(4)
    E, nu = 6.0e10, 0.22
    lam, mu = lame(E, nu)
    Ke = oracle.element_stiffness(xe, E, nu)
    # u_c(x) = sum_jk Q[c,j,k] y_j y_k with y = x - x0 (element-local)
    Q = rng.standard_normal((3, 3, 3)) * 1e-6
    Q = 0.5 * (Q + Q.transpose(0, 2, 1))
    x0 = xe[0]
    u = np.einsum("cjk,nj,nk->nc", Q, xe - x0, xe - x0).reshape(-1)
    # grad u_c / dx_j = 2 sum_k Q[c,j,k] y_k  is linear in y; y = sum_a L_a (x_a - x0)
    Y = xe[:4] - x0                                   # y at the corners
    G = [2 * np.einsum("cjk,k->cj", Q, Y[a]) for a in range(4)]  # grad u at corner a
    # energy density is quadratic: W(L) = sum_ab L_a L_b w(G_a, G_b)
    def w(Ga, Gb):
        ea, eb = 0.5 * (Ga + Ga.T), 0.5 * (Gb + Gb.T)
        return lam * np.trace(ea) * np.trace(eb) + 2 * mu * np.sum(ea * eb)
    poly = {}
    for a in range(4):
        for b in range(4):
            ex = [0, 0, 0, 0]; ex[a] += 1; ex[b] += 1
            poly[tuple(ex)] = poly.get(tuple(ex), 0.0) + w(G[a], G[b])
    energy = _monomial_integral(xe, poly)
    assert u @ Ke @ u == pytest.approx(energy, rel=1e-11)


def test_element_scaling_and_material_linearity():
    xe = jittered_element(5)
    K1 = oracle.element_stiffness(xe, 2.0e10, 0.3)
    K2 = oracle.element_stiffness(xe, 6.0e10, 0.3)
    assert np.allclose(K2, 3.0 * K1, rtol=1e-13, atol=1e-13 * np.abs(K2).max())
    Ks = oracle.element_stiffness(2.5 * xe, 2.0e10, 0.3)       # K scales with length
    assert np.allclose(Ks, 2.5 * K1, rtol=1e-12, atol=1e-12 * np.abs(Ks).max())
    Kt = oracle.element_stiffness(xe + np.array([1e3, -2e3, 5e2]), 2.0e10, 0.3)
    assert np.allclose(Kt, K1, rtol=1e-9, atol=1e-11 * np.abs(K1).max())


def test_element_rotation_covariance():
    """K_e(R x) = Rb K_e(x) Rb^T with Rb = blockdiag(R) (isotropy + frame invariance)."""
    xe = jittered_element(6)
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1.0]])
    ax = np.array([1.0, 2.0, 2.0]) / 3.0
    Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    R = R @ (np.eye(3) + math.sin(0.4) * Kx + (1 - math.cos(0.4)) * Kx @ Kx)
    K1 = oracle.element_stiffness(xe, 3.0e10, 0.28)
    K2 = oracle.element_stiffness(xe @ R.T, 3.0e10, 0.28)
    Rb = np.kron(np.eye(10), R)
    assert np.allclose(K2, Rb @ K1 @ Rb.T, rtol=1e-10, atol=1e-11 * np.abs(K1).max())


def test_element_rejects_inverted():
    xe = jittered_element(7)
    bad = xe.copy()
    bad[[1, 2]] = bad[[2, 1]]
    bad[4:] = np.array([0.5 * (bad[a] + bad[b]) for a, b in mg.EDGES])
    with pytest.raises(ValueError):
        oracle.element_stiffness(bad, 1e10, 0.25)


# ---------------------------------------------------------------------------
# assembled operator
# ---------------------------------------------------------------------------

def _dense_from_elements(mesh, apply_bc=True):
    """Dense K assembled in numpy from oracle element matrices (checks the C
    sparsity pattern, block indexing and BC treatment)."""
    n = mesh.n_dof
    K = np.zeros((n, n))
    for e in range(mesh.n_elem):
        ce = mesh.conn[e]
        Ke = oracle.element_stiffness(mesh.coords[ce], mesh.young[e], mesh.poisson[e])
        dofs = (3 * ce[:, None] + np.arange(3)[None, :]).reshape(-1)
        K[np.ix_(dofs, dofs)] += Ke
    if apply_bc:
        p = mesh.free.reshape(-1).astype(float)
        K = (p[:, None] * K * p[None, :]) + np.diag(1.0 - p)
    return K


@pytest.mark.parametrize("n", [1, 2])
def test_dense_vs_block_csr(n):
    m = mg.plain_box(n=n, jitter=0.1, seed=3)
    Kd = _dense_from_elements(m)
    Kc = oracle.assemble(m).dense()
    assert np.abs(Kd - Kc).max() <= 1e-12 * np.abs(Kd).max()
    x = mg.random_vectors(m.n_nodes, 3, seed=1)
    y = oracle.spmv(oracle.assemble(m), x)
    yd = np.einsum("ij,rj->ri", Kd, x.transpose(1, 0, 2).reshape(3, -1)).reshape(3, m.n_nodes, 3).transpose(1, 0, 2)
    assert np.linalg.norm(y - yd) <= 1e-13 * np.linalg.norm(yd)


def test_unconstrained_nullspace_is_rigid():
    m = mg.plain_box(n=2, jitter=0.1, seed=5)
    K = oracle.assemble(m, apply_bc=False).dense()
    w = np.linalg.eigvalsh(K)
    assert np.all(np.abs(w[:6]) <= 1e-12 * w[-1])
    assert w[6] > 1e-8 * w[-1]


def test_constrained_spd_and_symmetric():
    m = mg.plain_box(n=2, jitter=0.1, seed=6)
    K = oracle.assemble(m).dense()
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    assert np.linalg.eigvalsh(K)[0] > 0.0


def test_block_jacobi_inverts_diagonal_blocks():
    """M^-1 times the 3x3 diagonal blocks of K_bc (taken from a dense matrix
    assembled here from element matrices) is the identity at every node."""
    m = mg.plain_box(n=2, jitter=0.1, seed=9)
    Kd = _dense_from_elements(m)
    Minv = oracle.block_jacobi(oracle.assemble(m))
    for n in range(m.n_nodes):
        B = Kd[3 * n:3 * n + 3, 3 * n:3 * n + 3]
        assert np.abs(Minv[n] @ B - np.eye(3)).max() <= 1e-12


def _interior_nodes(m):
    lx, ly, lz = m.lattice_shape()
    i = np.arange(m.n_nodes) % lx
    j = (np.arange(m.n_nodes) // lx) % ly
    k = np.arange(m.n_nodes) // (lx * ly)
    return (i > 0) & (i < lx - 1) & (j > 0) & (j < ly - 1) & (k > 0) & (k < lz - 1)


def test_linear_patch_test():
    """u = A x + b gives zero force at every interior node (no BC applied)."""
    m = mg.plain_box(n=3, jitter=0.15, seed=7)
    m.young[:] = 4.0e10                                   # homogeneous: stress is constant
    m.poisson[:] = 0.25
    K = oracle.assemble(m, apply_bc=False)
    A = np.array([[1.0, 2.0, -0.5], [0.3, -1.0, 0.7], [0.2, 0.4, 1.5]]) * 1e-4
    u = (m.coords @ A.T + np.array([0.1, -0.2, 0.3]))[:, None, :]
    y = oracle.spmv(K, u)[:, 0, :]
    inner = _interior_nodes(m)
    scale = np.abs(K.vals).max() * np.abs(u).max()
    assert np.abs(y[inner]).max() <= 1e-10 * scale
    assert np.abs(y[~inner]).max() > 1e-3 * scale          # boundary tractions are not zero


def test_quadratic_patch_test():
    """Quadratic u on a homogeneous jittered mesh: at interior nodes,
    (K u)_i = -div(sigma) * sum_{e containing i} int N_i, with int N_corner = -V/20,
    int N_edge = V/5 and div(sigma) constant (computed here from the formula)."""
    m = mg.box_mesh((3, 3, 3), (3000.0, 3000.0, 3000.0), jitter=0.15, seed=8)
    E, nu = 5.0e10, 0.26
    m.young[:] = E
    m.poisson[:] = nu
    lam, mu = lame(E, nu)
    rng = np.random.default_rng(9)
    A = rng.standard_normal((3, 3, 3)) * 1e-7
    A = 0.5 * (A + A.transpose(0, 2, 1))                  # u_c = sum_jk A[c,j,k] x_j x_k
    x = m.coords
    u = np.einsum("cjk,nj,nk->nc", A, x, x)
    # d_c = 2 lam sum_j A[j,j,c] + 2 mu sum_j (A[c,j,j] + A[j,c,j])
    d = np.array([2 * lam * sum(A[j, j, c] for j in range(3)) +
                  2 * mu * sum(A[c, j, j] + A[j, c, j] for j in range(3)) for c in range(3)])
    K = oracle.assemble(m, apply_bc=False)
    y = oracle.spmv(K, u[:, None, :])[:, 0, :]
    intN = np.zeros(m.n_nodes)
    X = m.coords[m.conn[:, :4]]
    V = np.linalg.det(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=1)) / 6
    for a in range(4):
        np.add.at(intN, m.conn[:, a], -V / 20)
    for a in range(4, 10):
        np.add.at(intN, m.conn[:, a], V / 5)
    expect = -intN[:, None] * d[None, :]
    inner = _interior_nodes(m)
    err = np.abs(y[inner] - expect[inner]).max()
    assert err <= 1e-9 * np.abs(expect[inner]).max()


def test_sampled_product_matches_assembled():
    m, _ = mg.crust_block(shape=(4, 3, 3), h=1000.0, jitter=0.15, seed=2)
    K = oracle.assemble(m)
    x = mg.random_vectors(m.n_nodes, 2, seed=11)
    y = oracle.spmv(K, x)
    nodes = np.arange(0, m.n_nodes, 7)
    ys = oracle.sampled_product(m, x, nodes)
    assert np.abs(ys - y[nodes]).max() <= 1e-12 * np.abs(y).max()


def test_bad_connectivity_rejected():
    m = mg.plain_box(n=1)
    m.conn = m.conn.copy()
    m.conn[0, 3] = m.n_nodes + 5
    with pytest.raises(ValueError):
        oracle.assemble(m)


# ---------------------------------------------------------------------------
# exact FE solutions
# ---------------------------------------------------------------------------

def _column(n_xy=2, nz=6, layers=((0.0, 8e10, 0.27), (3000.0, 4e10, 0.25))):
    """Unjittered column, 1 km hexahedra, layers with boundaries on lattice planes."""
    m = mg.box_mesh((n_xy, n_xy, nz), (1000.0 * n_xy, 1000.0 * n_xy, 1000.0 * nz), jitter=0.0)
    zc = m.centroids()[:, 2]
    for z0, E, nu in layers:
        sel = zc > z0
        m.young[sel] = E
        m.poisson[sel] = nu
    return m


def _constrained_modulus(E, nu):
    lam, mu = lame(E, nu)
    return lam + 2 * mu


def _top_pressure_load(m, p):
    """Consistent nodal loads of uniform pressure p (downward) on the top face: the
    6-node triangle gives 0 to corners and A/3 to each edge node."""
    f = np.zeros((m.n_nodes, 3))
    lx, ly, lz = m.lattice_shape()
    hx, hy, _ = m.h
    ktop = lz - 1
    A = 0.5 * hx * hy
    for ci in range(m.shape[0]):
        for cj in range(m.shape[1]):
            bi, bj = 2 * ci, 2 * cj
            for v1 in ((2, 0), (0, 2)):
                tri = [(0, 0), v1, (2, 2)]
                for a, b in ((0, 1), (1, 2), (0, 2)):
                    li = bi + (tri[a][0] + tri[b][0]) // 2
                    lj = bj + (tri[a][1] + tri[b][1]) // 2
                    f[m.node_id(li, lj, ktop), 2] -= p * A / 3
    return f


def test_oedometer_exact():
    """Roller sides, clamped base, uniform top pressure: u_x = u_y = 0 and
    u_z(z) = -p int_0^z dz / M(z) (piecewise linear), reproduced exactly."""
    m = _column()
    p = 1.0e6
    f = _top_pressure_load(m, p)[:, None, :] * m.free[:, None, :]
    K = oracle.assemble(m)
    ud = oracle.direct_solve(K, f)[:, 0, :]
    z = m.coords[:, 2]
    M_lo = _constrained_modulus(8e10, 0.27)
    M_hi = _constrained_modulus(4e10, 0.25)
    uz = np.where(z <= 3000.0, -p * z / M_lo, -p * 3000.0 / M_lo - p * (z - 3000.0) / M_hi)
    exact = np.zeros_like(ud)
    exact[:, 2] = uz
    assert np.abs(ud - exact).max() <= 1e-10 * np.abs(uz).max()
    u, it, rel = oracle.pcg(K, f, tol=1e-12)
    assert rel[0] <= 1e-12
    assert np.abs(u[:, 0, :] - exact).max() <= 1e-8 * np.abs(uz).max()


def test_gravity_column_exact():
    """Uniform body force -rho g z_hat: sigma_zz = -rho g (H - z), u_z piecewise
    quadratic; nodal loads b * int N_i (corner -V/20, edge V/5)."""
    m = _column(nz=4, layers=((0.0, 8e10, 0.27), (2000.0, 4e10, 0.25)))
    rg = 2700.0 * 9.81
    H = m.lengths[2]
    X = m.coords[m.conn[:, :4]]
    V = np.linalg.det(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=1)) / 6
    f = np.zeros((m.n_nodes, 3))
    for a in range(4):
        np.add.at(f[:, 2], m.conn[:, a], -rg * (-V / 20))
    for a in range(4, 10):
        np.add.at(f[:, 2], m.conn[:, a], -rg * (V / 5))
    f = (f * m.free)[:, None, :]
    K = oracle.assemble(m)
    ud = oracle.direct_solve(K, f)[:, 0, :]
    z = m.coords[:, 2]
    M_lo = _constrained_modulus(8e10, 0.27)
    M_hi = _constrained_modulus(4e10, 0.25)
    # M u_z' = -rg (H - z)  ->  u_z = -(rg/M) (H z - z^2/2) + const per layer
    def prim(zz):
        return H * zz - 0.5 * zz * zz
    uz = np.where(z <= 2000.0, -rg / M_lo * prim(z),
                  -rg / M_lo * prim(2000.0) - rg / M_hi * (prim(z) - prim(2000.0)))
    assert np.abs(ud[:, 2] - uz).max() <= 1e-10 * np.abs(uz).max()
    assert np.abs(ud[:, :2]).max() <= 1e-10 * np.abs(uz).max()


# ---------------------------------------------------------------------------
# solvers
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def box8():
    m = mg.plain_box()
    K = oracle.assemble(m)
    f = mg.plain_box_rhs(m)
    return m, K, f


def test_pcg_matches_direct(box8):
    m, K, f = box8
    ud = oracle.direct_solve(K, f)
    u, it, rel = oracle.pcg(K, f, tol=1e-10)
    assert rel[0] <= 1e-10
    assert np.linalg.norm(u - ud) <= 1e-7 * np.linalg.norm(ud)
    assert 50 < it[0] < 1000


def test_fcg_mixed_matches_direct(box8):
    m, K, f = box8
    ud = oracle.direct_solve(K, f)
    u, outer, inner, rel = oracle.fcg_mixed(K, f, tol=1e-8)
    assert rel[0] <= 1.5e-8
    assert np.linalg.norm(u - ud) <= 1e-5 * np.linalg.norm(ud)
    _, it, _ = oracle.pcg(K, f, tol=1e-8)
    assert outer[0] < it[0] / 3                       # the inner solve does the work


def test_fcg_zero_inner_is_pcg(box8):
    """With no inner steps the preconditioner is the fixed block Jacobi, flexible CG
    reduces to PCG (same iteration count up to FP32 preconditioner rounding)."""
    m, K, f = box8
    _, it, rel_p = oracle.pcg(K, f, tol=1e-8)
    u, outer, inner, rel = oracle.fcg_mixed(K, f, tol=1e-8, n_inner=0)
    assert inner[0] == 0
    assert abs(int(outer[0]) - int(it[0])) <= max(3, 0.03 * it[0])
    assert rel[0] <= 1.5e-8


def _block_jacobi_numpy(K):
    """Inverse 3x3 diagonal blocks of the assembled K_bc, from scipy's matrix and
    numpy's inverse (independent of the oracle's own block-Jacobi routine)."""
    A = K.to_scipy().tocsr()
    n = A.shape[0] // 3
    return np.stack([np.linalg.inv(A[3 * i:3 * i + 3, 3 * i:3 * i + 3].toarray()) for i in range(n)]), A


def test_fcg_inner_loop_runs_n0_steps_when_eps_is_zero(box8):
    """Algorithm 1(b) with a zero tolerance never stops early: every outer iteration
    runs exactly N_0 inner steps (the cap of 30, not the 29 of a literal 'i < N')."""
    m, K, f = box8
    for n0 in (30, 7):
        u, outer, inner, rel = oracle.fcg_mixed(K, f, tol=1e-8, eps_inner=0.0, n_inner=n0)
        assert rel[0] <= 1.5e-8
        assert inner[0] == n0 * outer[0]


def test_fcg_inner_stop_rule_is_on_the_squared_ratio(box8):
    """The inner loop stops before a step once ||e||^2 / ||rbar||^2 <= eps (the squared
    ratio of Algorithm 1(b)). In the first outer iteration (u = 0, rbar = f) the first
    test sees e = f - K M^-1 f; rho0 = ||e|| / ||f|| is computed here from scipy's
    matrix and numpy's block inverses. With eps between rho0^2 and rho0 the squared
    and the unsquared rule disagree on whether any step runs."""
    m, K, f = box8
    Minv, A = _block_jacobi_numpy(K)
    fv = f[:, 0, :]
    e = fv.reshape(-1) - A @ np.einsum("nij,nj->ni", Minv, fv).reshape(-1)
    rho0 = np.linalg.norm(e) / np.linalg.norm(fv)
    assert 0.2 < rho0 < 0.9                      # margins for the two tolerances below
    _, outer, inner, _ = oracle.fcg_mixed(K, f, tol=1e-8, max_outer=1, eps_inner=rho0 ** 1.5)
    assert outer[0] == 1 and inner[0] == 0       # rho0^2 <= eps < rho0: no step
    _, outer, inner, _ = oracle.fcg_mixed(K, f, tol=1e-8, max_outer=1, eps_inner=rho0 ** 2.5)
    assert outer[0] == 1 and inner[0] >= 1       # eps < rho0^2: at least one step


def test_fcg_inner_stop_ignores_converged_cases(box8):
    """The inner stop rule takes the maximum over the cases still active: a case that
    starts converged (initial guess = its direct solution, so its FP32 residual is
    rounding noise with an inner ratio far above eps) does not change another case's
    iteration counts or solution."""
    m, K, f = box8
    lx, ly, lz = m.lattice_shape()
    fa = mg.double_couple(m, (lx // 2 - 4, ly // 2 + 2, lz // 2 + 3), 1e12)[:, None, :]
    ua = oracle.direct_solve(K, fa)
    u1, outer1, inner1, rel1 = oracle.fcg_mixed(K, f, tol=1e-8)
    F = np.concatenate([f, fa], axis=1)
    U0 = np.concatenate([np.zeros_like(f), ua], axis=1)
    u2, outer2, inner2, rel2 = oracle.fcg_mixed(K, F, u0=U0, tol=1e-8)
    assert outer2[1] == 0 and inner2[1] == 0 and rel2[1] <= 1e-8
    assert outer2[0] == outer1[0] and inner2[0] == inner1[0]
    assert np.array_equal(u2[:, 0], u1[:, 0])


def test_batched_cases_betti_and_linearity(box8):
    m, K, f1 = box8
    lx, ly, lz = m.lattice_shape()
    f2 = mg.double_couple(m, (lx // 2 - 4, ly // 2 + 2, lz // 2 + 3), 1e12)[:, None, :]
    F = np.concatenate([f1, f2, 2.0 * f1 - 3.0 * f2], axis=1)
    u, outer, inner, rel = oracle.fcg_mixed(K, F, tol=1e-10)
    assert np.all(rel <= 1.5e-10)
    b12 = np.sum(F[:, 0] * u[:, 1])
    b21 = np.sum(F[:, 1] * u[:, 0])
    assert b12 == pytest.approx(b21, rel=1e-7)
    lin = 2.0 * u[:, 0] - 3.0 * u[:, 1]
    assert np.linalg.norm(u[:, 2] - lin) <= 1e-8 * np.linalg.norm(lin)


def test_literal_beta_flag_runs(box8):
    m, K, f = box8
    u, outer, inner, rel = oracle.fcg_mixed(K, f, tol=1e-8, literal_beta=True, max_outer=400)
    assert np.isfinite(rel[0])


# ---------------------------------------------------------------------------
# adjoint
# ---------------------------------------------------------------------------

def test_adjoint_gradient_matches_finite_differences():
    """dJ/dm_e for J = 1/2 |P u - d|^2, K_bc(m) u = f, m_e = log E_e, against central
    differences of J with sparse direct solves (brute force on a tiny mesh)."""
    m = mg.plain_box(n=2, jitter=0.1, seed=1)
    rng = np.random.default_rng(12)
    f = mg.plain_box_rhs(m, force=1e12)
    f = f + 0.0
    Pm = np.zeros((12, m.n_dof))
    free_top = np.nonzero(m.free.reshape(-1))[0]
    rows = rng.choice(free_top, size=12, replace=False)
    Pm[np.arange(12), rows] = 1.0
    d = rng.standard_normal(12) * 1e-3
    logE = np.log(m.young)

    def J(le):
        K = oracle.assemble(m, young=np.exp(le))
        u = oracle.direct_solve(K, f)[:, 0, :].reshape(-1)
        r = Pm @ u - d
        return 0.5 * r @ r, u

    J0, u = J(logE)
    K = oracle.assemble(m)
    g_rhs = (Pm.T @ (Pm @ u - d)).reshape(m.n_nodes, 1, 3) * m.free[:, None, :]
    lam = oracle.direct_solve(K, g_rhs)
    g = oracle.adjoint_grad(m, u.reshape(m.n_nodes, 1, 3), lam)
    h = 1e-5
    for e in (0, 3, 7, 11):
        lp = logE.copy(); lp[e] += h
        lm = logE.copy(); lm[e] -= h
        fd = (J(lp)[0] - J(lm)[0]) / (2 * h)
        assert g[e] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(g).max())
    v = rng.standard_normal(m.n_elem)
    v /= np.linalg.norm(v)
    fd = (J(logE + h * v)[0] - J(logE - h * v)[0]) / (2 * h)
    assert g @ v == pytest.approx(fd, rel=1e-5)


def test_golden_loop_config():
    """Inner-loop tolerance/iteration table of the paper (Table 'loopconfig')."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "loop_config.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    table = {int(r[0]): (float(r[1]), int(r[2])) for r in rows}
    assert table[0] == (0.1, 30)
    assert table[1] == (0.05, 300)
    assert table[2] == (0.025, 3000)


# ---------------------------------------------------------------------------
# first-order (TET4) coarse level
# ---------------------------------------------------------------------------

def test_tet4_element_rigid_modes_and_energy():
    xe = jittered_element(11)[:4]
    E, nu = 3.0e10, 0.26
    Ke = oracle.tet4_stiffness(xe, E, nu)
    w = np.linalg.eigvalsh(Ke)
    assert np.all(np.abs(w[:6]) <= 1e-12 * w[-1]) and np.all(w[6:] > 1e-6 * w[-1])
    A = np.random.default_rng(5).standard_normal((3, 3)) * 1e-3
    u = (xe @ A.T).reshape(-1)
    eps = 0.5 * (A + A.T)
    lam, mu = lame(E, nu)
    assert u @ Ke @ u == pytest.approx(tet_volume(xe) * (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps)),
                                       rel=1e-12)


def test_coarse_operator_is_galerkin_projection():
    """Linear functions on the tetrahedra lie in the quadratic space, so the TET4
    stiffness is exactly P1^T K P1 (P1: vertex values kept, edge nodes averaged)."""
    m = mg.plain_box(n=2, jitter=0.12, seed=10)
    cm = oracle.coarse_mesh(m)
    K = oracle.assemble(m, apply_bc=False).to_scipy()
    K1 = oracle.assemble4(cm, apply_bc=False).dense()
    n4 = cm.coords.shape[0]
    P = np.zeros((m.n_dof, 3 * n4))
    for n, (a, b) in enumerate(cm.ends):
        for i in range(3):
            P[3 * n + i, 3 * a + i] += 0.5
            P[3 * n + i, 3 * b + i] += 0.5
    G = P.T @ (K @ P)
    assert np.abs(G - K1).max() <= 1e-12 * np.abs(K1).max()


def test_prolongation_reproduces_linear_fields_and_restriction_is_its_transpose():
    m = mg.plain_box(n=3, jitter=0.15, seed=12)
    cm = oracle.coarse_mesh(m)
    A = np.array([[1.0, 2.0, -1.0], [0.5, -0.3, 0.2], [0.1, 0.0, 0.7]])
    lin4 = (cm.coords @ A.T)[:, None, :]
    lin10 = (m.coords @ A.T)[:, None, :]
    assert np.abs(oracle.prolong(cm, lin4) - lin10).max() <= 1e-9 * np.abs(lin10).max()
    rng = np.random.default_rng(3)
    a = rng.standard_normal((cm.coords.shape[0], 2, 3))
    b = rng.standard_normal((m.n_nodes, 2, 3))
    assert np.sum(oracle.restrict(cm, b) * a) == pytest.approx(np.sum(b * oracle.prolong(cm, a)), rel=1e-12)


def test_linear_patch_test_tet4():
    m = mg.plain_box(n=3, jitter=0.15, seed=7)
    m.young[:] = 4.0e10
    m.poisson[:] = 0.25
    cm = oracle.coarse_mesh(m)
    K1 = oracle.assemble4(cm, apply_bc=False)
    A = np.array([[1.0, 2.0, -0.5], [0.3, -1.0, 0.7], [0.2, 0.4, 1.5]]) * 1e-4
    u = (cm.coords @ A.T)[:, None, :]
    y = oracle.spmv(K1, u)[:, 0]
    lx, ly, lz = m.lattice_shape()
    v = cm.vertex
    i, j, k = v % lx, (v // lx) % ly, v // (lx * ly)
    inner = (i > 0) & (i < lx - 1) & (j > 0) & (j < ly - 1) & (k > 0) & (k < lz - 1)
    assert np.abs(y[inner]).max() <= 1e-10 * np.abs(K1.vals).max() * np.abs(u).max()


def test_two_level_fcg_matches_direct_and_moves_work_to_the_coarse_level(box8):
    """The TET4 level shifts the inner work from the quadratic mesh to the linear
    one (Sec. 2): same solution, far fewer level-0 inner steps."""
    m, K, f = box8
    cm = oracle.coarse_mesh(m)
    ud = oracle.direct_solve(K, f)
    u1, o1, i1, j1, rel1 = oracle.fcg_mg(K, f, tol=1e-8)
    u2, o2, i2, j2, rel2 = oracle.fcg_mg(K, f, coarse=cm, free=m.free, tol=1e-8)
    assert rel2[0] <= 1.5e-8 and j2[0] > 0 and j1[0] == 0
    assert np.linalg.norm(u2 - ud) <= 1e-5 * np.linalg.norm(ud)
    assert i2[0] < i1[0] / 2


# ---------------------------------------------------------------------------
# level 2: aggregation coarsening of the TET4 level (Sec. 2)
# ---------------------------------------------------------------------------

def make_tet4_levels():
    m = mg.crust_block(shape=(10, 8, 5), h=1000.0, jitter=0.15, seed=2)[0]
    cm = oracle.coarse_mesh(m)
    K1 = oracle.assemble4(cm)
    return m, cm, K1


@pytest.fixture(scope="module")
def tet4_levels():
    return make_tet4_levels()


def test_aggregation_is_a_partition_into_connected_aggregates(tet4_levels):
    """Every coarse node lies in exactly one aggregate, every aggregate is
    connected in the matrix graph, and each has a seed whose whole neighbourhood
    it contains and within two graph steps of which all its members lie (a
    pass-2 node joins the aggregate of a neighbour), checked by searches written
    here, independent of the oracle."""
    m, cm, K1 = tet4_levels
    agg = oracle.aggregate(K1)
    N4 = K1.n_nodes
    assert agg.shape == (N4,) and agg.min() == 0
    NA = int(agg.max()) + 1
    assert np.array_equal(np.unique(agg), np.arange(NA))
    nbr = [K1.col[K1.rowptr[n]:K1.rowptr[n + 1]] for n in range(N4)]
    for A in range(NA):
        mem = set(np.nonzero(agg == A)[0].tolist())
        start = min(mem)
        seen, todo = {start}, [start]
        while todo:
            n = todo.pop()
            for j in nbr[n].tolist():
                if j in mem and j not in seen:
                    seen.add(j)
                    todo.append(j)
        assert seen == mem, A
        seeds = [s for s in mem if set(nbr[s].tolist()) <= mem]
        assert seeds, A                                              # a seed's whole neighbourhood
        two_steps = lambda s: set(nbr[s].tolist()).union(*[set(nbr[j].tolist()) for j in nbr[s].tolist()])
        assert any(mem <= two_steps(s) for s in seeds), A
    assert N4 / 40 < NA < N4 / 4


def test_galerkin_aggregation_matrix_is_the_triple_product(tet4_levels):
    """A2 equals P2^T K1_bc P2 formed with scipy from an explicit P2 (aggregate
    value copied to the members' free DOFs), with identity on aggregate DOFs that
    have no free member; it is symmetric positive definite."""
    import scipy.sparse as sp
    m, cm, K1 = tet4_levels
    agg = oracle.aggregate(K1)
    A2, free2 = oracle.galerkin_agg(K1, cm.free, agg)
    N4, NA = K1.n_nodes, A2.n_nodes
    rows, cols = [], []
    for n in range(N4):
        for c in range(3):
            if cm.free[n, c]:
                rows.append(3 * n + c)
                cols.append(3 * agg[n] + c)
    P = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(3 * N4, 3 * NA))
    ref = (P.T @ K1.to_scipy() @ P).toarray()
    fixed2 = np.nonzero(free2.reshape(-1) == 0)[0]
    ref[fixed2, fixed2] = 1.0
    got = A2.dense()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # rows and columns of aggregate DOFs without a free member are exactly unit
    assert np.array_equal(got[fixed2], np.eye(3 * NA)[fixed2])
    assert np.array_equal(got[:, fixed2], np.eye(3 * NA)[:, fixed2])
    assert np.allclose(got, got.T, rtol=0, atol=1e-12 * np.abs(got).max())
    assert np.linalg.eigvalsh(got).min() > 0
    for c in range(3):                       # an aggregate DOF is free iff a member DOF is
        assert np.array_equal(free2[:, c] > 0, np.bincount(agg, weights=cm.free[:, c], minlength=NA) > 0)


def test_three_level_fcg_matches_direct_and_reduces_level1_work(tet4_levels):
    """Levels 2, 1, 0 (Algorithm 1(a)): the direct solution, with fewer level-1
    steps than levels 1 and 0 alone (level 2 resolves the low-frequency part)."""
    m, cm, K1 = tet4_levels
    K = oracle.assemble(m)
    F = mg.random_vectors(m.n_nodes, 2, seed=12) * 1e9 * m.free[:, None, :]
    ud = oracle.direct_solve(K, F)
    u2, o2, i02, i12, i22, rel2 = oracle.fcg_ml(K, F, cm, m.free, K1=K1, levels=2)
    u3, o3, i03, i13, i23, rel3 = oracle.fcg_ml(K, F, cm, m.free, K1=K1, levels=3)
    assert np.all(rel3 <= 1.5e-8) and np.all(i23 > 0) and np.all(i22 == 0)
    assert np.linalg.norm(u3 - ud) <= 1e-5 * np.linalg.norm(ud)
    assert np.all(i13 < i12)
