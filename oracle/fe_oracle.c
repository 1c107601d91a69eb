/*
 * fe_oracle.c -- plain FP64 CPU oracle for the element-by-element (EBE) product and
 * the conjugate-gradient solvers of the multiple-case implicit FE crust solver
 * (Yamaguchi et al., "Implicit Low-Order Unstructured Finite-Element Multiple
 * Simulation Enhanced by Dense Computation using OpenACC").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do. It shares no code with the CUDA path.
 *
 * What it computes, by plain definitions:
 *   - the element stiffness of a 10-node tetrahedron for isotropic linear
 *     elasticity (Sec. 2, Eq. 1a-1c discretised into Eq. 2), by the textbook
 *     isoparametric B^T D B integrand and the 4-point degree-2 Gauss rule (exact
 *     for straight-sided elements because the integrand is quadratic);
 *   - the assembled global matrix K = sum_i Q_i K_i Q_i^T (Eq. 3) in node-block
 *     compressed-row storage (3x3 blocks), with Dirichlet rows and columns
 *     replaced by identity: K_bc = P K P + (I - P);
 *   - y = K_bc x for R vectors stored [node][R][3] (the multiple-vector layout
 *     of Sec. 3.1);
 *   - 3x3 block Jacobi M = diag[K_bc] (Algorithm 1(a), its set-up);
 *   - preconditioned CG with 3x3 block Jacobi (the PCGE baseline of Sec. 4);
 *   - the flexible (adaptive) CG of Algorithm 1(a) with the FP32 inner PCG of
 *     Algorithm 1(b) at level 0, and optionally at level 1 (the TET4 mesh of the
 *     same corners) and level 2 (an aggregation coarsening of level 1), for R
 *     cases at once;
 *   - the adjoint element sensitivity g_e = -sum_r lambda_r^T (dK_bc/dm_e) u_r
 *     for m_e = log E_e (no counterpart in the paper).
 *
 * Readings where the paper is silent are listed in the design notes; the ones that
 * matter here: straight-sided elements, VTK node order, Voigt order
 * (xx,yy,zz,yz,xz,xy) with engineering shear strain, stopping on ||r||/||f||.
 *
 * All entry points return 0 on success and a negative code on bad input.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* VTK TET10 edges: local node 4+q lies at the midpoint of corners EDGE[q][0..1] */
static const int EDGE[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};

/* thread count of the OpenMP loops (timing of the CPU baseline on one core or all) */
void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* element stiffness                                                          */
/* ------------------------------------------------------------------------- */

/* derivatives of the 10 quadratic shape functions with respect to the natural
 * coordinates (xi, eta, zeta) = (L1, L2, L3), L0 = 1 - xi - eta - zeta, at the
 * point with volume coordinates L[4].  dN[a][k] = dN_a / dxi_k. */
static void tet10_dshape(const double L[4], double dN[10][3]) {
  /* dL_a / dxi_k */
  static const double dL[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) dN[a][k] = (4.0 * L[a] - 1.0) * dL[a][k];   /* N_a = L_a (2 L_a - 1) */
  for (int q = 0; q < 6; ++q) {
    int a = EDGE[q][0], b = EDGE[q][1];
    for (int k = 0; k < 3; ++k) dN[4 + q][k] = 4.0 * (L[b] * dL[a][k] + L[a] * dL[b][k]); /* N_ab = 4 L_a L_b */
  }
}

static double inv3(const double A[3][3], double Ai[3][3]) {
  double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
             - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
             + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  if (det == 0.0) return 0.0;
  double id = 1.0 / det;
  Ai[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) * id;
  Ai[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * id;
  Ai[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * id;
  Ai[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) * id;
  Ai[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * id;
  Ai[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * id;
  Ai[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) * id;
  Ai[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * id;
  Ai[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * id;
  return det;
}

/* Isotropic elasticity matrix in Voigt order (xx,yy,zz,yz,xz,xy), engineering shear. */
static void elasticity_D(double E, double nu, double D[6][6]) {
  double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  double mu = E / (2.0 * (1.0 + nu));
  memset(D, 0, sizeof(double) * 36);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) D[i][j] = lam;
  for (int i = 0; i < 3; ++i) D[i][i] = lam + 2.0 * mu;
  for (int i = 3; i < 6; ++i) D[i][i] = mu;
}

/* Ke[30*30] (row-major, DOF 3a+i = component i of local node a) of a TET10 with
 * node coordinates xe[10*3], Young's modulus E, Poisson ratio nu.
 * K_e = sum_q w_q det(J_q) B_q^T D B_q with the 4-point rule (volume coordinates
 * (a,b,b,b) and permutations, a = (5+3 sqrt5)/20, b = (5-sqrt5)/20, w = 1/24).
 * Returns 0, or -1 for a non-positive Jacobian. */
int oracle_tet10_stiffness(const double* xe, double E, double nu, double* Ke) {
  const double qa = (5.0 + 3.0 * sqrt(5.0)) / 20.0, qb = (5.0 - sqrt(5.0)) / 20.0;
  double D[6][6];
  elasticity_D(E, nu, D);
  memset(Ke, 0, sizeof(double) * 900);
  for (int qp = 0; qp < 4; ++qp) {
    double L[4] = {qb, qb, qb, qb};
    L[qp] = qa;
    double dN[10][3];
    tet10_dshape(L, dN);
    double J[3][3] = {{0}}; /* J[i][k] = dx_i / dxi_k */
    for (int n = 0; n < 10; ++n)
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) J[i][k] += xe[3 * n + i] * dN[n][k];
    double Ji[3][3];
    double det = inv3(J, Ji);
    if (!(det > 0.0)) return -1;
    /* dN_n/dx_i = sum_k dN_n/dxi_k * dxi_k/dx_i = sum_k dN[n][k] * Ji[k][i] */
    double B[6][30];
    memset(B, 0, sizeof(B));
    for (int n = 0; n < 10; ++n) {
      double g[3];
      for (int i = 0; i < 3; ++i) g[i] = dN[n][0] * Ji[0][i] + dN[n][1] * Ji[1][i] + dN[n][2] * Ji[2][i];
      int c = 3 * n;
      B[0][c + 0] = g[0];
      B[1][c + 1] = g[1];
      B[2][c + 2] = g[2];
      B[3][c + 1] = g[2]; B[3][c + 2] = g[1];   /* gamma_yz */
      B[4][c + 0] = g[2]; B[4][c + 2] = g[0];   /* gamma_xz */
      B[5][c + 0] = g[1]; B[5][c + 1] = g[0];   /* gamma_xy */
    }
    double w = det / 24.0;
    double DB[6][30];
    for (int i = 0; i < 6; ++i)
      for (int s = 0; s < 30; ++s) {
        double acc = 0.0;
        for (int j = 0; j < 6; ++j) acc += D[i][j] * B[j][s];
        DB[i][s] = acc;
      }
    for (int r = 0; r < 30; ++r)
      for (int s = 0; s < 30; ++s) {
        double acc = 0.0;
        for (int i = 0; i < 6; ++i) acc += B[i][r] * DB[i][s];
        Ke[30 * r + s] += w * acc;
      }
  }
  return 0;
}

static void gather_element(const double* coords, const int32_t* conn_e, double xe[30]) {
  for (int a = 0; a < 10; ++a)
    for (int i = 0; i < 3; ++i) xe[3 * a + i] = coords[3 * (int64_t)conn_e[a] + i];
}

/* ------------------------------------------------------------------------- */
/* sparsity pattern and assembly (node-block CSR, 3x3 blocks)                 */
/* ------------------------------------------------------------------------- */

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* node -> element incidence lists (CSR) for elements of `nen` nodes; caller frees *nptr and *nel */
static int node_elements_n(int64_t N, int64_t E, int nen, const int32_t* conn, int64_t** nptr, int64_t** nel) {
  int64_t* ptr = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
  if (!ptr) return -2;
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < nen; ++a) ptr[conn[nen * e + a] + 1]++;
  for (int64_t n = 0; n < N; ++n) ptr[n + 1] += ptr[n];
  int64_t* lst = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ptr[N] > 0 ? ptr[N] : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  if (!lst || !fill) { free(ptr); free(lst); free(fill); return -2; }
  for (int64_t n = 0; n < N; ++n) fill[n] = ptr[n];
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < nen; ++a) {
      int32_t n = conn[nen * e + a];
      /* an element lists a node once; a repeated node would be a malformed element */
      lst[fill[n]++] = e;
    }
  free(fill);
  *nptr = ptr;
  *nel = lst;
  return 0;
}

static int node_elements(int64_t N, int64_t E, const int32_t* conn, int64_t** nptr, int64_t** nel) {
  return node_elements_n(N, E, 10, conn, nptr, nel);
}

static int check_conn_n(int64_t N, int64_t E, int nen, const int32_t* conn) {
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < nen; ++a) {
      if (conn[nen * e + a] < 0 || conn[nen * e + a] >= N) return -1;
      for (int b = 0; b < a; ++b)
        if (conn[nen * e + a] == conn[nen * e + b]) return -1;
    }
  return 0;
}

static int check_conn(int64_t N, int64_t E, const int32_t* conn) { return check_conn_n(N, E, 10, conn); }

/* Block pattern of K for elements of `nen` nodes (10: TET10, 4: TET4): block (n, m)
 * present iff nodes n and m share an element. rowptr[N+1] is always written; col[]
 * (sorted per row) only when col != NULL. Returns the number of blocks, or a
 * negative code. */
int64_t oracle_pattern_n(int64_t N, int64_t E, int nen, const int32_t* conn, int64_t* rowptr, int32_t* col) {
  if (N <= 0 || E < 0 || (nen != 4 && nen != 10) || check_conn_n(N, E, nen, conn)) return -1;
  int64_t *nptr, *nel;
  if (node_elements_n(N, E, nen, conn, &nptr, &nel)) return -2;
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * 4096);
  size_t cap = 4096;
  rowptr[0] = 0;
  for (int64_t n = 0; n < N; ++n) {
    size_t cnt = 0;
    for (int64_t p = nptr[n]; p < nptr[n + 1]; ++p) {
      if (cnt + (size_t)nen > cap) { cap *= 2; buf = (int32_t*)realloc(buf, sizeof(int32_t) * cap); }
      for (int a = 0; a < nen; ++a) buf[cnt++] = conn[nen * nel[p] + a];
    }
    if (cnt == 0) buf[cnt++] = (int32_t)n;   /* isolated node keeps its diagonal block */
    qsort(buf, cnt, sizeof(int32_t), cmp_i32);
    size_t u = 0;
    for (size_t i = 0; i < cnt; ++i)
      if (u == 0 || buf[i] != buf[u - 1]) buf[u++] = buf[i];
    if (col) memcpy(col + rowptr[n], buf, sizeof(int32_t) * u);
    rowptr[n + 1] = rowptr[n] + (int64_t)u;
  }
  free(buf);
  free(nptr);
  free(nel);
  return rowptr[N];
}

int64_t oracle_pattern(int64_t N, int64_t E, const int32_t* conn, int64_t* rowptr, int32_t* col) {
  return oracle_pattern_n(N, E, 10, conn, rowptr, col);
}

static int64_t find_block(const int64_t* rowptr, const int32_t* col, int32_t n, int32_t m) {
  int64_t lo = rowptr[n], hi = rowptr[n + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (col[mid] == m) return mid;
    if (col[mid] < m) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* vals[nnzb*9] (block (n,m) entry (i,j) at 9*b + 3*i + j) = sum_e Q_e K_e Q_e^T. */
int oracle_assemble(int64_t N, const double* coords, int64_t E, const int32_t* conn,
                    const double* young, const double* poisson,
                    const int64_t* rowptr, const int32_t* col, double* vals) {
  memset(vals, 0, sizeof(double) * 9 * (size_t)rowptr[N]);
  double Ke[900], xe[30];
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* ce = conn + 10 * e;
    gather_element(coords, ce, xe);
    if (oracle_tet10_stiffness(xe, young[e], poisson[e], Ke)) return -1;
    for (int a = 0; a < 10; ++a)
      for (int b = 0; b < 10; ++b) {
        int64_t blk = find_block(rowptr, col, ce[a], ce[b]);
        if (blk < 0) return -3;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) vals[9 * blk + 3 * i + j] += Ke[30 * (3 * a + i) + 3 * b + j];
      }
  }
  return 0;
}

/* K_bc = P K P + (I - P): constrained rows and columns become the identity. */
int oracle_apply_bc(int64_t N, const int64_t* rowptr, const int32_t* col, double* vals, const uint8_t* free_mask) {
  for (int64_t n = 0; n < N; ++n)
    for (int64_t b = rowptr[n]; b < rowptr[n + 1]; ++b) {
      int64_t m = col[b];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          int fi = free_mask[3 * n + i], fj = free_mask[3 * m + j];
          if (!fi || !fj) vals[9 * b + 3 * i + j] = (n == m && i == j) ? 1.0 : 0.0;
        }
    }
  return 0;
}

/* y[N][R][3] = K x[N][R][3] */
void oracle_spmv(int64_t N, const int64_t* rowptr, const int32_t* col, const double* vals, int R,
                 const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    for (int r = 0; r < R; ++r) {
      double acc[3] = {0.0, 0.0, 0.0};
      for (int64_t b = rowptr[n]; b < rowptr[n + 1]; ++b) {
        const double* xm = x + 3 * ((int64_t)col[b] * R + r);
        const double* K = vals + 9 * b;
        for (int i = 0; i < 3; ++i) acc[i] += K[3 * i] * xm[0] + K[3 * i + 1] * xm[1] + K[3 * i + 2] * xm[2];
      }
      for (int i = 0; i < 3; ++i) y[3 * (n * R + r) + i] = acc[i];
    }
  }
}

/* FP32 product: matrix entries and vector rounded to float, float arithmetic. */
static void spmv_f32(int64_t N, const int64_t* rowptr, const int32_t* col, const float* vals, int R,
                     const float* x, float* y) {
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    for (int r = 0; r < R; ++r) {
      float acc[3] = {0.f, 0.f, 0.f};
      for (int64_t b = rowptr[n]; b < rowptr[n + 1]; ++b) {
        const float* xm = x + 3 * ((int64_t)col[b] * R + r);
        const float* K = vals + 9 * b;
        for (int i = 0; i < 3; ++i) acc[i] += K[3 * i] * xm[0] + K[3 * i + 1] * xm[1] + K[3 * i + 2] * xm[2];
      }
      for (int i = 0; i < 3; ++i) y[3 * (n * R + r) + i] = acc[i];
    }
  }
}

/* ------------------------------------------------------------------------- */
/* first-order (TET4) coarse level of the multigrid inner solve (Sec. 2: the   */
/* same mesh without edge nodes)                                              */
/* ------------------------------------------------------------------------- */

/* Ke[12*12] of a 4-node (linear) tetrahedron: K_e = V B^T D B with the constant
 * B of the linear shape functions N_a = L_a (one-point rule, exact). */
int oracle_tet4_stiffness(const double* xe, double E, double nu, double* Ke) {
  static const double dL[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  double D[6][6];
  elasticity_D(E, nu, D);
  double J[3][3] = {{0}}; /* J[i][k] = dx_i / dxi_k */
  for (int n = 0; n < 4; ++n)
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) J[i][k] += xe[3 * n + i] * dL[n][k];
  double Ji[3][3];
  double det = inv3(J, Ji);
  if (!(det > 0.0)) return -1;
  double B[6][12];
  memset(B, 0, sizeof(B));
  for (int n = 0; n < 4; ++n) {
    double g[3];
    for (int i = 0; i < 3; ++i) g[i] = dL[n][0] * Ji[0][i] + dL[n][1] * Ji[1][i] + dL[n][2] * Ji[2][i];
    int c = 3 * n;
    B[0][c + 0] = g[0];
    B[1][c + 1] = g[1];
    B[2][c + 2] = g[2];
    B[3][c + 1] = g[2]; B[3][c + 2] = g[1];
    B[4][c + 0] = g[2]; B[4][c + 2] = g[0];
    B[5][c + 0] = g[1]; B[5][c + 1] = g[0];
  }
  double V = det / 6.0;
  for (int r = 0; r < 12; ++r)
    for (int s = 0; s < 12; ++s) {
      double acc = 0.0;
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) acc += B[i][r] * D[i][j] * B[j][s];
      Ke[12 * r + s] = V * acc;
    }
  return 0;
}

/* Assembled K_1 = sum_e Q_e K_e^(4) Q_e^T of a TET4 mesh (coords4 [N4][3], conn4 [E][4]). */
int oracle_assemble4(int64_t N, const double* coords, int64_t E, const int32_t* conn,
                     const double* young, const double* poisson,
                     const int64_t* rowptr, const int32_t* col, double* vals) {
  memset(vals, 0, sizeof(double) * 9 * (size_t)rowptr[N]);
  double Ke[144], xe[12];
  for (int64_t e = 0; e < E; ++e) {
    const int32_t* ce = conn + 4 * e;
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) xe[3 * a + i] = coords[3 * (int64_t)ce[a] + i];
    if (oracle_tet4_stiffness(xe, young[e], poisson[e], Ke)) return -1;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        int64_t blk = find_block(rowptr, col, ce[a], ce[b]);
        if (blk < 0) return -3;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) vals[9 * blk + 3 * i + j] += Ke[12 * (3 * a + i) + 3 * b + j];
      }
  }
  return 0;
}

/* Mapping between the TET4 and TET10 node sets: ends[2n], ends[2n+1] are the TET4
 * nodes whose linear interpolation gives TET10 node n (equal for a vertex). */
/* u10 = P u4 (prolongation: vertices copied, edge nodes the mean of their ends) */
void oracle_prolong(int64_t N10, int R, const int32_t* ends, const double* u4, double* u10) {
  for (int64_t n = 0; n < N10; ++n)
    for (int r = 0; r < R; ++r)
      for (int i = 0; i < 3; ++i) {
        int32_t a = ends[2 * n], b = ends[2 * n + 1];
        u10[3 * (n * R + r) + i] = (a == b) ? u4[3 * ((int64_t)a * R + r) + i]
                                            : 0.5 * (u4[3 * ((int64_t)a * R + r) + i] + u4[3 * ((int64_t)b * R + r) + i]);
      }
}

/* r4 = P^T r10 (restriction, the transpose of oracle_prolong) */
void oracle_restrict(int64_t N10, int64_t N4, int R, const int32_t* ends, const double* r10, double* r4) {
  memset(r4, 0, sizeof(double) * 3 * (size_t)N4 * R);
  for (int64_t n = 0; n < N10; ++n)
    for (int r = 0; r < R; ++r)
      for (int i = 0; i < 3; ++i) {
        int32_t a = ends[2 * n], b = ends[2 * n + 1];
        double v = r10[3 * (n * R + r) + i];
        if (a == b) {
          r4[3 * ((int64_t)a * R + r) + i] += v;
        } else {
          r4[3 * ((int64_t)a * R + r) + i] += 0.5 * v;
          r4[3 * ((int64_t)b * R + r) + i] += 0.5 * v;
        }
      }
}

static void prolong_f32(int64_t N10, int R, const int32_t* ends, const float* u4, float* u10) {
  for (int64_t n = 0; n < N10; ++n)
    for (int r = 0; r < R; ++r)
      for (int i = 0; i < 3; ++i) {
        int32_t a = ends[2 * n], b = ends[2 * n + 1];
        u10[3 * (n * R + r) + i] = (a == b) ? u4[3 * ((int64_t)a * R + r) + i]
                                            : 0.5f * (u4[3 * ((int64_t)a * R + r) + i] + u4[3 * ((int64_t)b * R + r) + i]);
      }
}

static void mask_f32(int64_t N, int R, const uint8_t* free_mask, float* v) {
  for (int64_t n = 0; n < N; ++n)
    for (int r = 0; r < R; ++r)
      for (int i = 0; i < 3; ++i)
        if (!free_mask[3 * n + i]) v[3 * (n * R + r) + i] = 0.0f;
}

static void restrict_f32(int64_t N10, int64_t N4, int R, const int32_t* ends, const float* r10, float* r4) {
  memset(r4, 0, sizeof(float) * 3 * (size_t)N4 * R);
  for (int64_t n = 0; n < N10; ++n)
    for (int r = 0; r < R; ++r)
      for (int i = 0; i < 3; ++i) {
        int32_t a = ends[2 * n], b = ends[2 * n + 1];
        float v = r10[3 * (n * R + r) + i];
        if (a == b) {
          r4[3 * ((int64_t)a * R + r) + i] += v;
        } else {
          r4[3 * ((int64_t)a * R + r) + i] += 0.5f * v;
          r4[3 * ((int64_t)b * R + r) + i] += 0.5f * v;
        }
      }
}

/* ------------------------------------------------------------------------- */
/* products on sampled rows (full-size checks without assembling everything)  */
/* ------------------------------------------------------------------------- */

/* y_s[S][R][3] = rows `nodes[s]` of K_bc x, computed element by element from the
 * definition: (K_bc x)_(n,i) = x_(n,i) if (n,i) is constrained, otherwise the sum
 * over elements e containing n of row (n,i) of K_e applied to the masked x_e. */
int oracle_sampled_product(int64_t N, const double* coords, int64_t E, const int32_t* conn,
                           const double* young, const double* poisson, const uint8_t* free_mask,
                           int R, const double* x, int64_t S, const int64_t* nodes, double* ys) {
  if (check_conn(N, E, conn)) return -1;
  int64_t *nptr, *nel;
  if (node_elements(N, E, conn, &nptr, &nel)) return -2;
  int rc = 0;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t s = 0; s < S; ++s) {
    double Ke[900], xe[30];
    int64_t n = nodes[s];
    double* out = ys + 3 * s * R;
    for (int k = 0; k < 3 * R; ++k) out[k] = 0.0;
    for (int64_t p = nptr[n]; p < nptr[n + 1]; ++p) {
      int64_t e = nel[p];
      const int32_t* ce = conn + 10 * e;
      gather_element(coords, ce, xe);
      if (oracle_tet10_stiffness(xe, young[e], poisson[e], Ke)) { rc = -1; continue; }
      int la = 0;
      while (ce[la] != n) ++la;
      for (int r = 0; r < R; ++r)
        for (int i = 0; i < 3; ++i) {
          double acc = 0.0;
          for (int b = 0; b < 10; ++b)
            for (int j = 0; j < 3; ++j) {
              int64_t m = ce[b];
              if (free_mask[3 * m + j]) acc += Ke[30 * (3 * la + i) + 3 * b + j] * x[3 * (m * R + r) + j];
            }
          out[3 * r + i] += acc;
        }
    }
    for (int r = 0; r < R; ++r)
      for (int i = 0; i < 3; ++i)
        if (!free_mask[3 * n + i]) out[3 * r + i] = x[3 * (n * R + r) + i];
  }
  free(nptr);
  free(nel);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* 3x3 block Jacobi                                                           */
/* ------------------------------------------------------------------------- */

/* Minv[N][9] = inverse of the diagonal 3x3 block of K_bc per node (Algorithm 1(a), set-up). */
int oracle_block_jacobi(int64_t N, const int64_t* rowptr, const int32_t* col, const double* vals, double* Minv) {
  for (int64_t n = 0; n < N; ++n) {
    int64_t b = find_block(rowptr, col, (int32_t)n, (int32_t)n);
    if (b < 0) return -1;
    double A[3][3], Ai[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A[i][j] = vals[9 * b + 3 * i + j];
    if (inv3(A, Ai) == 0.0) return -4;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Minv[9 * n + 3 * i + j] = Ai[i][j];
  }
  return 0;
}

static void apply_blocks(int64_t N, int R, const double* Minv, const double* e, double* z) {
  for (int64_t n = 0; n < N; ++n)
    for (int r = 0; r < R; ++r) {
      const double* v = e + 3 * (n * R + r);
      double* o = z + 3 * (n * R + r);
      const double* M = Minv + 9 * n;
      for (int i = 0; i < 3; ++i) o[i] = M[3 * i] * v[0] + M[3 * i + 1] * v[1] + M[3 * i + 2] * v[2];
    }
}

static void apply_blocks_f32(int64_t N, int R, const float* Minv, const float* e, float* z) {
  for (int64_t n = 0; n < N; ++n)
    for (int r = 0; r < R; ++r) {
      const float* v = e + 3 * (n * R + r);
      float* o = z + 3 * (n * R + r);
      const float* M = Minv + 9 * n;
      for (int i = 0; i < 3; ++i) o[i] = M[3 * i] * v[0] + M[3 * i + 1] * v[1] + M[3 * i + 2] * v[2];
    }
}

/* per-case dot products d[r] = sum_n sum_i a[n][r][i] b[n][r][i] */
static void dots(int64_t N, int R, const double* a, const double* b, double* d) {
  for (int r = 0; r < R; ++r) d[r] = 0.0;
  for (int64_t n = 0; n < N; ++n)
    for (int r = 0; r < R; ++r)
      for (int i = 0; i < 3; ++i) d[r] += a[3 * (n * R + r) + i] * b[3 * (n * R + r) + i];
}

static void dots_f32(int64_t N, int R, const float* a, const float* b, double* d) {
  for (int r = 0; r < R; ++r) d[r] = 0.0;
  for (int64_t n = 0; n < N; ++n)
    for (int r = 0; r < R; ++r)
      for (int i = 0; i < 3; ++i) d[r] += (double)(a[3 * (n * R + r) + i] * b[3 * (n * R + r) + i]);
}

/* ------------------------------------------------------------------------- */
/* PCG with 3x3 block Jacobi (PCGE), R independent cases                      */
/* ------------------------------------------------------------------------- */

/* Solves K_bc u_r = f_r for every case r, starting from the given u, until
 * ||r||/||f|| <= tol (recursively updated residual) or maxit iterations.
 * iters[r], relres[r] (true residual ||f - K u|| / ||f|| at exit) are written. */
int oracle_pcg(int64_t N, const int64_t* rowptr, const int32_t* col, const double* vals, const double* Minv,
               int R, const double* f, double* u, double tol, int maxit, int32_t* iters, double* relres) {
  size_t nv = (size_t)N * R * 3;
  double *r = malloc(nv * 8), *z = malloc(nv * 8), *p = malloc(nv * 8), *q = malloc(nv * 8);
  double *fn = malloc(R * 8), *rho = malloc(R * 8), *rho_new = malloc(R * 8), *gam = malloc(R * 8), *rn = malloc(R * 8);
  int* active = malloc(R * sizeof(int));
  if (!r || !z || !p || !q || !fn || !rho || !rho_new || !gam || !rn || !active) return -2;
  oracle_spmv(N, rowptr, col, vals, R, u, q);
  for (size_t k = 0; k < nv; ++k) r[k] = f[k] - q[k];
  apply_blocks(N, R, Minv, r, z);
  memcpy(p, z, nv * 8);
  dots(N, R, z, r, rho);
  dots(N, R, f, f, fn);
  for (int c = 0; c < R; ++c) { iters[c] = 0; active[c] = fn[c] > 0.0; }
  for (int it = 0; it < maxit; ++it) {
    dots(N, R, r, r, rn);
    int any = 0;
    for (int c = 0; c < R; ++c) {
      if (active[c] && sqrt(rn[c] / fn[c]) <= tol) active[c] = 0;
      any |= active[c];
    }
    if (!any) break;
    oracle_spmv(N, rowptr, col, vals, R, p, q);
    dots(N, R, p, q, gam);
    for (int64_t n = 0; n < N; ++n)
      for (int c = 0; c < R; ++c) {
        if (!active[c]) continue;
        double alpha = rho[c] / gam[c];
        for (int i = 0; i < 3; ++i) {
          size_t k = 3 * (n * R + c) + i;
          u[k] += alpha * p[k];
          r[k] -= alpha * q[k];
        }
      }
    apply_blocks(N, R, Minv, r, z);
    dots(N, R, z, r, rho_new);
    for (int64_t n = 0; n < N; ++n)
      for (int c = 0; c < R; ++c) {
        if (!active[c]) continue;
        double beta = rho_new[c] / rho[c];
        for (int i = 0; i < 3; ++i) {
          size_t k = 3 * (n * R + c) + i;
          p[k] = z[k] + beta * p[k];
        }
      }
    for (int c = 0; c < R; ++c)
      if (active[c]) { rho[c] = rho_new[c]; iters[c]++; }
  }
  oracle_spmv(N, rowptr, col, vals, R, u, q);
  for (size_t k = 0; k < nv; ++k) r[k] = f[k] - q[k];
  dots(N, R, r, r, rn);
  for (int c = 0; c < R; ++c) relres[c] = fn[c] > 0.0 ? sqrt(rn[c] / fn[c]) : 0.0;
  free(r); free(z); free(p); free(q); free(fn); free(rho); free(rho_new); free(gam); free(rn); free(active);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Flexible (adaptive) CG of Algorithm 1(a) with the level-0 inner loop only  */
/* (levels 1 and 2: oracle_fcg_ml below), and the FP32 inner PCG of          */
/* Algorithm 1(b), R cases at once                                           */
/* ------------------------------------------------------------------------- */

/* Algorithm 1(b) on one level, FP32 vectors and products, dots accumulated in FP64:
 *   e = rb - Kbar ub; while max_r ||e_r||^2/||rb_r||^2 > eps and steps < n_steps:
 *   z = Mbar^-1 e; rho_a = (z, e); beta = rho_a/rho_b (after the first step);
 *   p = z + beta p; q = Kbar p; gamma = (p, q); alpha = rho_a/gamma; rho_b = rho_a;
 *   e -= alpha q; ub += alpha p.
 * Only cases with active[c] take part (their count of steps goes to steps[c]). */
static int inner_pcg_f32(int64_t N, const int64_t* rowptr, const int32_t* col, const float* vals32,
                         const float* Minv32, int R, const float* rb, float* ub, int n_steps, double eps,
                         const int* active, int32_t* steps) {
  size_t nv = (size_t)N * R * 3;
  float *eb = malloc(nv * 4), *zb = malloc(nv * 4), *pb = malloc(nv * 4), *qb = malloc(nv * 4);
  double *rbn = malloc(R * 8), *en = malloc(R * 8), *rho_a = malloc(R * 8), *rho_b = malloc(R * 8), *gb = malloc(R * 8);
  if (!eb || !zb || !pb || !qb || !rbn || !en || !rho_a || !rho_b || !gb) return -2;
  spmv_f32(N, rowptr, col, vals32, R, ub, qb);
  for (size_t k = 0; k < nv; ++k) eb[k] = rb[k] - qb[k];
  dots_f32(N, R, rb, rb, rbn);
  for (int step = 0; step < n_steps; ++step) {
    dots_f32(N, R, eb, eb, en);
    double worst = 0.0;
    for (int c = 0; c < R; ++c)
      if (active[c] && rbn[c] > 0.0 && en[c] / rbn[c] > worst) worst = en[c] / rbn[c];
    if (!(worst > eps)) break;
    apply_blocks_f32(N, R, Minv32, eb, zb);
    dots_f32(N, R, zb, eb, rho_a);
    for (int64_t n = 0; n < N; ++n)
      for (int c = 0; c < R; ++c) {
        if (!active[c]) continue;
        float beta = step > 0 ? (float)(rho_a[c] / rho_b[c]) : 0.0f;
        for (int i = 0; i < 3; ++i) {
          size_t k = 3 * (n * R + c) + i;
          pb[k] = zb[k] + beta * (step > 0 ? pb[k] : 0.0f);
        }
      }
    spmv_f32(N, rowptr, col, vals32, R, pb, qb);
    dots_f32(N, R, pb, qb, gb);
    for (int64_t n = 0; n < N; ++n)
      for (int c = 0; c < R; ++c) {
        if (!active[c]) continue;
        float alpha = (float)(rho_a[c] / gb[c]);
        for (int i = 0; i < 3; ++i) {
          size_t k = 3 * (n * R + c) + i;
          eb[k] -= alpha * qb[k];
          ub[k] += alpha * pb[k];
        }
      }
    for (int c = 0; c < R; ++c)
      if (active[c]) { rho_b[c] = rho_a[c]; steps[c]++; }
  }
  free(eb); free(zb); free(pb); free(qb); free(rbn); free(en); free(rho_a); free(rho_b); free(gb);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* level 2: algebraic coarsening of the TET4 level (Sec. 2)                   */
/* ------------------------------------------------------------------------- */

/* Plain aggregation of the nodes of a block matrix's graph (neighbours: the
 * other columns of a node's block row), two passes in node order:
 *   pass 1: a node that is not aggregated and none of whose neighbours is
 *           aggregated starts a new aggregate made of itself and all its
 *           neighbours;
 *   pass 2: each node still without aggregate joins the pass-1 aggregate of its
 *           lowest-numbered neighbour that has one (every such node has one: it
 *           was skipped in pass 1 because a neighbour was taken).
 * Writes agg[N] and returns the number of aggregates. */
int64_t oracle_aggregate(int64_t N, const int64_t* rowptr, const int32_t* col, int32_t* agg) {
  for (int64_t n = 0; n < N; ++n) agg[n] = -1;
  int64_t count = 0;
  for (int64_t n = 0; n < N; ++n) {
    if (agg[n] >= 0) continue;
    int all_free = 1;
    for (int64_t q = rowptr[n]; q < rowptr[n + 1]; ++q)
      if (col[q] != n && agg[col[q]] >= 0) { all_free = 0; break; }
    if (!all_free) continue;
    agg[n] = (int32_t)count;
    for (int64_t q = rowptr[n]; q < rowptr[n + 1]; ++q) agg[col[q]] = (int32_t)count;
    ++count;
  }
  int32_t* first = malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
  if (!first) return -2;
  memcpy(first, agg, sizeof(int32_t) * (size_t)N);
  for (int64_t n = 0; n < N; ++n) {
    if (first[n] >= 0) continue;
    int32_t best = -1;
    for (int64_t q = rowptr[n]; q < rowptr[n + 1]; ++q) {
      const int32_t j = col[q];
      if (j != n && first[j] >= 0 && (best < 0 || j < best)) best = j;
    }
    if (best < 0) { free(first); return -1; }
    agg[n] = first[best];
  }
  free(first);
  return count;
}

/* Galerkin coarse matrix of the aggregation: with P2 the piecewise-constant
 * prolongation (aggregate value copied to each member node, component by
 * component, on the member's free DOFs only),
 *   A2 = P2^T K1_bc P2 on the free aggregate DOFs (those with a free member),
 *   identity on the others.
 * Block-row a of K1 adds its blocks, restricted to free (row, column) DOFs, into
 * block-row agg[a] at block-column agg[b]. Outputs A2 in block CSR (columns
 * increasing within a row; capacity rowptr[N] blocks, always enough) and
 * free2[NA][3]. Returns the number of blocks of A2. */
int64_t oracle_galerkin_agg(int64_t N, const int64_t* rowptr, const int32_t* col, const double* vals,
                            const uint8_t* free_mask, const int32_t* agg, int64_t NA, int64_t* rowptr2,
                            int32_t* col2, double* vals2, uint8_t* free2) {
  int64_t* mstart = calloc((size_t)NA + 1, sizeof(int64_t));
  int64_t* members = malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  int64_t* pos = malloc(sizeof(int64_t) * (size_t)(NA > 0 ? NA : 1));
  if (!mstart || !members || !pos) return -2;
  for (int64_t n = 0; n < N; ++n) mstart[agg[n] + 1]++;
  for (int64_t A = 0; A < NA; ++A) mstart[A + 1] += mstart[A];
  {
    int64_t* fill = malloc(sizeof(int64_t) * (size_t)(NA > 0 ? NA : 1));
    if (!fill) return -2;
    memcpy(fill, mstart, sizeof(int64_t) * (size_t)NA);
    for (int64_t n = 0; n < N; ++n) members[fill[agg[n]]++] = n;
    free(fill);
  }
  for (int64_t A = 0; A < NA; ++A) pos[A] = -1;
  int64_t nnz = 0;
  rowptr2[0] = 0;
  for (int64_t A = 0; A < NA; ++A) {
    const int64_t row0 = nnz;
    for (int i = 0; i < 3; ++i) free2[3 * A + i] = 0;
    for (int64_t k = mstart[A]; k < mstart[A + 1]; ++k) {
      const int64_t a = members[k];
      for (int i = 0; i < 3; ++i) free2[3 * A + i] |= free_mask[3 * a + i];
      for (int64_t q = rowptr[a]; q < rowptr[a + 1]; ++q) {
        const int64_t b = col[q];
        const int32_t B = agg[b];
        if (pos[B] < 0) {
          pos[B] = nnz;
          col2[nnz] = B;
          for (int t = 0; t < 9; ++t) vals2[9 * nnz + t] = 0.0;
          ++nnz;
        }
        double* dst = vals2 + 9 * pos[B];
        const double* src = vals + 9 * q;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            if (free_mask[3 * a + i] && free_mask[3 * b + j]) dst[3 * i + j] += src[3 * i + j];
      }
    }
    for (int64_t t = row0; t < nnz; ++t) {
      if (col2[t] == A)
        for (int i = 0; i < 3; ++i)
          if (!free2[3 * A + i]) vals2[9 * t + 4 * i] = 1.0;
      pos[col2[t]] = -1;
    }
    /* columns in increasing order within the row (insertion sort, rows are short) */
    for (int64_t t = row0 + 1; t < nnz; ++t) {
      const int32_t c = col2[t];
      double v[9];
      for (int k = 0; k < 9; ++k) v[k] = vals2[9 * t + k];
      int64_t w = t;
      while (w > row0 && col2[w - 1] > c) {
        col2[w] = col2[w - 1];
        for (int k = 0; k < 9; ++k) vals2[9 * w + k] = vals2[9 * (w - 1) + k];
        --w;
      }
      col2[w] = c;
      for (int k = 0; k < 9; ++k) vals2[9 * w + k] = v[k];
    }
    rowptr2[A + 1] = nnz;
  }
  free(mstart); free(members); free(pos);
  return nnz;
}

/* r2 = P2^T r1 (free fine DOFs summed into their aggregate) */
static void restrict_agg_f32(int64_t N, int64_t NA, int R, const int32_t* agg, const uint8_t* free_mask,
                             const float* r1, float* r2) {
  memset(r2, 0, sizeof(float) * 3 * (size_t)NA * R);
  for (int64_t n = 0; n < N; ++n)
    for (int r = 0; r < R; ++r)
      for (int i = 0; i < 3; ++i)
        if (free_mask[3 * n + i]) r2[3 * ((int64_t)agg[n] * R + r) + i] += r1[3 * (n * R + r) + i];
}

/* u1 = P2 u2 (aggregate value on each member's free DOFs) */
static void prolong_agg_f32(int64_t N, int R, const int32_t* agg, const uint8_t* free_mask, const float* u2,
                            float* u1) {
  for (int64_t n = 0; n < N; ++n)
    for (int r = 0; r < R; ++r)
      for (int i = 0; i < 3; ++i)
        u1[3 * (n * R + r) + i] = free_mask[3 * n + i] ? u2[3 * ((int64_t)agg[n] * R + r) + i] : 0.0f;
}

/* Outer loop (FP64), per case r while ||r||/||f|| > tol (per-case masking):
 *   rbar = (float) r; ubar = Mbar^-1 rbar
 *   with the TET4 level (N4 > 0), inner loop level 1:
 *     rbar1 = P1^T rbar; ubar1 = P1^T ubar
 *     with the aggregation level (N2 > 0), inner loop level 2:
 *       rbar2 = P2^T rbar1; ubar2 = P2^T ubar1
 *       inner loop (b) on Abar2 ubar2 = rbar2 with eps_inner2, n_inner2
 *       ubar1 = P2 ubar2
 *     inner loop (b) on Kbar1 ubar1 = rbar1 with eps_inner1, n_inner1
 *     ubar = P1 ubar1
 *   inner loop level 0: (b) on Kbar ubar = rbar with eps_inner, n_inner
 *   z = (double) ubar                                 (printed "u <= ubar", read as z)
 *   if i > 1: beta = -(z, q_prev) / (p_prev, q_prev)   (flexible CG; the paper
 *             prints gamma=(z,q), beta=gamma/rho, read as this form -- with
 *             literal_beta != 0 the printed form is used instead)
 *   p = z + beta p;  q = K p;  rho = (z, r);  gamma = (p, q);  alpha = rho/gamma;
 *   r -= alpha q;  u += alpha p.
 * Kbar, Kbar1 are K_bc, K1_bc with entries rounded to FP32. Cases whose outer loop
 * has converged are frozen (they skip the inner loops and do not count in their
 * max rule). outer[r], inner_total[r] (level 0 steps), inner1_total[r] (level 1
 * steps), relres[r] (true residual) are written. */
int oracle_fcg_ml(int64_t N, const int64_t* rowptr, const int32_t* col, const double* vals, const double* Minv,
                  int R, const double* f, double* u, double tol, int max_outer, int n_inner, double eps_inner,
                  int literal_beta, const uint8_t* free_mask, int64_t N4, const int64_t* rowptr4,
                  const int32_t* col4, const double* vals4, const double* Minv4, const uint8_t* free4,
                  const int32_t* ends, int n_inner1, double eps_inner1, int64_t N2, const int64_t* rowptr2,
                  const int32_t* col2, const double* vals2, const double* Minv2, const int32_t* agg,
                  int n_inner2, double eps_inner2, int32_t* outer, int32_t* inner_total, int32_t* inner1_total,
                  int32_t* inner2_total, double* relres) {
  size_t nv = (size_t)N * R * 3, nv4 = (size_t)(N4 > 0 ? N4 : 1) * R * 3;
  int64_t nnzb = rowptr[N];
  float* vals32 = malloc(sizeof(float) * 9 * (size_t)nnzb);
  float* Minv32 = malloc(sizeof(float) * 9 * (size_t)N);
  float *vals4_32 = NULL, *Minv4_32 = NULL, *rb1 = NULL, *ub1 = NULL;
  float *vals2_32 = NULL, *Minv2_32 = NULL, *rb2 = NULL, *ub2 = NULL;
  double *r = malloc(nv * 8), *z = malloc(nv * 8), *p = malloc(nv * 8), *q = malloc(nv * 8);
  float *rb = malloc(nv * 4), *ub = malloc(nv * 4);
  double *fn = malloc(R * 8), *rn = malloc(R * 8), *rho = malloc(R * 8), *gam = malloc(R * 8),
         *zq = malloc(R * 8), *pq_prev = malloc(R * 8), *rho_prev = malloc(R * 8), *bet = malloc(R * 8);
  int* active = malloc(R * sizeof(int));
  if (!vals32 || !Minv32 || !r || !z || !p || !q || !rb || !ub || !fn || !rn || !rho || !gam || !zq || !pq_prev ||
      !rho_prev || !bet || !active)
    return -2;
  for (int64_t k = 0; k < 9 * nnzb; ++k) vals32[k] = (float)vals[k];
  for (int64_t k = 0; k < 9 * N; ++k) Minv32[k] = (float)Minv[k];
  if (N4 > 0) {
    vals4_32 = malloc(sizeof(float) * 9 * (size_t)rowptr4[N4]);
    Minv4_32 = malloc(sizeof(float) * 9 * (size_t)N4);
    rb1 = malloc(nv4 * 4);
    ub1 = malloc(nv4 * 4);
    if (!vals4_32 || !Minv4_32 || !rb1 || !ub1) return -2;
    for (int64_t k = 0; k < 9 * rowptr4[N4]; ++k) vals4_32[k] = (float)vals4[k];
    for (int64_t k = 0; k < 9 * N4; ++k) Minv4_32[k] = (float)Minv4[k];
  }
  if (N4 > 0 && N2 > 0) {
    const size_t nv2 = (size_t)N2 * R * 3;
    vals2_32 = malloc(sizeof(float) * 9 * (size_t)rowptr2[N2]);
    Minv2_32 = malloc(sizeof(float) * 9 * (size_t)N2);
    rb2 = malloc(nv2 * 4);
    ub2 = malloc(nv2 * 4);
    if (!vals2_32 || !Minv2_32 || !rb2 || !ub2) return -2;
    for (int64_t k = 0; k < 9 * rowptr2[N2]; ++k) vals2_32[k] = (float)vals2[k];
    for (int64_t k = 0; k < 9 * N2; ++k) Minv2_32[k] = (float)Minv2[k];
  }

  oracle_spmv(N, rowptr, col, vals, R, u, q);            /* r = f - K u */
  for (size_t k = 0; k < nv; ++k) r[k] = f[k] - q[k];
  memset(p, 0, nv * 8);
  dots(N, R, f, f, fn);
  for (int c = 0; c < R; ++c) {
    outer[c] = 0; inner_total[c] = 0; if (inner1_total) inner1_total[c] = 0; if (inner2_total) inner2_total[c] = 0;
    active[c] = fn[c] > 0.0;
  }
  int rc = 0;
  for (int it = 1; it <= max_outer; ++it) {
    dots(N, R, r, r, rn);
    int any = 0;
    for (int c = 0; c < R; ++c) {
      if (active[c] && sqrt(rn[c] / fn[c]) <= tol) active[c] = 0;
      any |= active[c];
    }
    if (!any) break;
    for (size_t k = 0; k < nv; ++k) rb[k] = (float)r[k];
    apply_blocks_f32(N, R, Minv32, rb, ub);
    if (N4 > 0) {
      /* transfers between the levels keep Dirichlet DOFs at zero (reading: the
       * paper's mapping matrices act on the free DOFs of each level) */
      restrict_f32(N, N4, R, ends, rb, rb1);
      restrict_f32(N, N4, R, ends, ub, ub1);
      mask_f32(N4, R, free4, rb1);
      mask_f32(N4, R, free4, ub1);
      if (N2 > 0) {
        restrict_agg_f32(N4, N2, R, agg, free4, rb1, rb2);
        restrict_agg_f32(N4, N2, R, agg, free4, ub1, ub2);
        rc = inner_pcg_f32(N2, rowptr2, col2, vals2_32, Minv2_32, R, rb2, ub2, n_inner2, eps_inner2, active,
                           inner2_total);
        if (rc) break;
        prolong_agg_f32(N4, R, agg, free4, ub2, ub1);
      }
      rc = inner_pcg_f32(N4, rowptr4, col4, vals4_32, Minv4_32, R, rb1, ub1, n_inner1, eps_inner1, active,
                         inner1_total);
      if (rc) break;
      prolong_f32(N, R, ends, ub1, ub);
      mask_f32(N, R, free_mask, ub);
    }
    rc = inner_pcg_f32(N, rowptr, col, vals32, Minv32, R, rb, ub, n_inner, eps_inner, active, inner_total);
    if (rc) break;
    for (size_t k = 0; k < nv; ++k) z[k] = (double)ub[k];
    if (it > 1) {
      dots(N, R, z, q, zq);
      for (int c = 0; c < R; ++c) bet[c] = literal_beta ? zq[c] / rho_prev[c] : -zq[c] / pq_prev[c];
    } else {
      for (int c = 0; c < R; ++c) bet[c] = 0.0;
    }
    for (int64_t n = 0; n < N; ++n)
      for (int c = 0; c < R; ++c) {
        if (!active[c]) continue;
        for (int i = 0; i < 3; ++i) {
          size_t k = 3 * (n * R + c) + i;
          p[k] = z[k] + bet[c] * p[k];
        }
      }
    oracle_spmv(N, rowptr, col, vals, R, p, q);
    dots(N, R, z, r, rho);
    dots(N, R, p, q, gam);
    for (int64_t n = 0; n < N; ++n)
      for (int c = 0; c < R; ++c) {
        if (!active[c]) continue;
        double alpha = rho[c] / gam[c];
        for (int i = 0; i < 3; ++i) {
          size_t k = 3 * (n * R + c) + i;
          r[k] -= alpha * q[k];
          u[k] += alpha * p[k];
        }
      }
    for (int c = 0; c < R; ++c)
      if (active[c]) { pq_prev[c] = gam[c]; rho_prev[c] = rho[c]; outer[c]++; }
  }
  oracle_spmv(N, rowptr, col, vals, R, u, q);
  for (size_t k = 0; k < nv; ++k) r[k] = f[k] - q[k];
  dots(N, R, r, r, rn);
  for (int c = 0; c < R; ++c) relres[c] = fn[c] > 0.0 ? sqrt(rn[c] / fn[c]) : 0.0;
  free(vals2_32); free(Minv2_32); free(rb2); free(ub2);
  free(vals32); free(Minv32); free(vals4_32); free(Minv4_32); free(rb1); free(ub1); free(r); free(z); free(p);
  free(q); free(rb); free(ub); free(fn); free(rn); free(rho); free(gam); free(zq); free(pq_prev); free(rho_prev);
  free(bet); free(active);
  return rc;
}

/* Levels 1 and 0 only. */
int oracle_fcg_mg(int64_t N, const int64_t* rowptr, const int32_t* col, const double* vals, const double* Minv,
                  int R, const double* f, double* u, double tol, int max_outer, int n_inner, double eps_inner,
                  int literal_beta, const uint8_t* free_mask, int64_t N4, const int64_t* rowptr4,
                  const int32_t* col4, const double* vals4, const double* Minv4, const uint8_t* free4,
                  const int32_t* ends, int n_inner1, double eps_inner1,
                  int32_t* outer, int32_t* inner_total, int32_t* inner1_total, double* relres) {
  return oracle_fcg_ml(N, rowptr, col, vals, Minv, R, f, u, tol, max_outer, n_inner, eps_inner, literal_beta,
                       free_mask, N4, rowptr4, col4, vals4, Minv4, free4, ends, n_inner1, eps_inner1, 0, NULL, NULL,
                       NULL, NULL, NULL, 0, 0.0, outer, inner_total, inner1_total, NULL, relres);
}

/* The flexible mixed CG with the inner loop at level 0 only. */
int oracle_fcg_mixed(int64_t N, const int64_t* rowptr, const int32_t* col, const double* vals, const double* Minv,
                     int R, const double* f, double* u, double tol, int max_outer, int n_inner, double eps_inner,
                     int literal_beta, int32_t* outer, int32_t* inner_total, double* relres) {
  return oracle_fcg_mg(N, rowptr, col, vals, Minv, R, f, u, tol, max_outer, n_inner, eps_inner, literal_beta, NULL,
                       0, NULL, NULL, NULL, NULL, NULL, NULL, 0, 0.0, outer, inner_total, NULL, relres);
}

/* ------------------------------------------------------------------------- */
/* adjoint element sensitivity                                                */
/* ------------------------------------------------------------------------- */

/* g[e] = -sum_r (P lambda_r)_e^T K_e (P u_r)_e, the derivative of J with respect
 * to m_e = log E_e given the adjoint state lambda (K_e is linear in E_e, so
 * dK_e/dm_e = K_e, and dK_bc/dm_e = P Q_e K_e Q_e^T P). */
int oracle_adjoint_grad(int64_t N, const double* coords, int64_t E, const int32_t* conn,
                        const double* young, const double* poisson, const uint8_t* free_mask,
                        int R, const double* u, const double* lam, double* g) {
  if (check_conn(N, E, conn)) return -1;
  int rc = 0;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < E; ++e) {
    double Ke[900], xe[30], ue[30], le[30];
    const int32_t* ce = conn + 10 * e;
    gather_element(coords, ce, xe);
    if (oracle_tet10_stiffness(xe, young[e], poisson[e], Ke)) { rc = -1; g[e] = 0.0; continue; }
    double acc = 0.0;
    for (int r = 0; r < R; ++r) {
      for (int a = 0; a < 10; ++a)
        for (int i = 0; i < 3; ++i) {
          int64_t k = 3 * ((int64_t)ce[a] * R + r) + i;
          int fr = free_mask[3 * (int64_t)ce[a] + i];
          ue[3 * a + i] = fr ? u[k] : 0.0;
          le[3 * a + i] = fr ? lam[k] : 0.0;
        }
      for (int s = 0; s < 30; ++s) {
        double ks = 0.0;
        for (int t = 0; t < 30; ++t) ks += Ke[30 * s + t] * ue[t];
        acc += le[s] * ks;
      }
    }
    g[e] = -acc;
  }
  return rc;
}
