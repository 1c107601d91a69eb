// Solvers of K_bc u_r = f_r for R cases at once.
//
//  * FE_SOLVER_PCG64: CG with 3x3 block Jacobi in FP64 (the paper's PCGE
//    reference solver of Sec. 4: Algorithm 1(a) with the preconditioner a
//    single block-Jacobi application instead of the inner loops).
//  * FE_SOLVER_FCG_MIXED: Algorithm 1 with the inner loop at level 0 only: an
//    FP64 flexible (adaptive) CG whose preconditioner z = K^-1 r is an FP32
//    block-Jacobi CG (Algorithm 1(b)) stopped at N steps or when
//    max_r ||e_r||^2/||rbar_r||^2 <= eps (the max-over-cases rule of Sec. 3.1).
//  * FE_SOLVER_FCG_MG: as FCG_MIXED with the inner loop at level 1 first: the
//    residual and the block-Jacobi guess are restricted to the TET4 mesh,
//    solved there by the same FP32 CG with the TET4 operator and its own block
//    Jacobi, and the coarse solution is prolonged as the initial guess of the
//    level-0 loop (Algorithm 1(a), inner loop level 1).
//  * FE_SOLVER_FCG_AMG: as FCG_MG with the aggregation level first: the level-1
//    residual and guess are restricted to the aggregates, solved there by the
//    same FP32 CG with A2 and its block Jacobi, and prolonged as the initial
//    guess of the level-1 loop (Algorithm 1(a), inner loop level 2).
//
// GPU design: every per-case scalar (rho, gamma, alpha, beta, norms, masks)
// lives in device arrays of length R; kernels read them directly, so one outer
// iteration (including all N inner steps) runs without host round trips and is
// captured once as a CUDA graph and replayed. Each inner loop is a while node
// of that graph whose condition the stop-test kernel sets, so it runs only the
// steps it needs; without a graph, the steps after the stop return at once
// (each kernel checks a device flag). Each case is
// masked on its own once it converges. Vectors are [N][R][3]; a vector kernel's
// thread handles one (node, case) pair and neighbouring threads touch
// neighbouring addresses. Dot products accumulate per thread (FP32 products in
// FP32 for the inner loop, FP64 otherwise), then per block in FP64 shared
// memory, then with one FP64 atomic add per block and case.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "fe_element.cuh"
#include "fe_internal.cuh"

namespace fe {

// ---------------------------------------------------------------------------
// per-case device state
// ---------------------------------------------------------------------------
enum DField {
  D_FN2 = 0, D_RN2, D_RHO, D_GAM, D_ZQ, D_PQP, D_RHOP, D_ALPHA, D_BETA,
  D_RBN2, D_EN2, D_RHOA, D_RHOB, D_GAMI, D_ALPHAI, D_BETAI, D_RT2, D_RELRES, D_RBN21, D_RBN22, D_COUNT
};
enum IField { I_ACTIVE = 0, I_CAND, I_RESTART, I_FIRST, I_STATUS, I_OUTER, I_INNER, I_INNER1, I_INNER2, I_COUNT };

struct Cases {
  double* d;      // [D_COUNT][R]
  int* i;         // [I_COUNT][R]
  int* done;      // inner-loop stop flag (1 int), the inner step counter (1 int), and a flag
                  // set while every free component of u is zero (1 int; the start skips K u)
  int R;
  double* hist = nullptr;   // PCG64: (alpha, beta) per iteration and case, [hist_len][R][2] (optional)
  int hist_len = 0;
  __device__ __forceinline__ int& step() const { return done[1]; }
  __device__ __forceinline__ double& D(int f, int r) const { return d[f * R + r]; }
  __device__ __forceinline__ int& I(int f, int r) const { return i[f * R + r]; }
};

struct SolverWork {
  int R = 0;
  int64_t N = 0;
  DevBuf r, p, q;                 // double [N][R][3]
  DevBuf rb, ub, eb, pb, qb;      // float  [N][R][3]
  DevBuf rb1, ub1, eb1, pb1, qb1; // float  [N4][R][3] (level 1, allocated when used)
  DevBuf rb2, ub2, eb2, pb2, qb2; // float  [NA][R][3] (level 2, allocated when used)
  DevBuf tu, tq;                  // double [N][3] (single-case true residual)
  DevBuf tall;                    // double [N][R][3] (true residuals of several cases at once, lazily)
  DevBuf d, i;                    // case state
  DevBuf pers;                    // persistent inner loop: sums [2][3][R], barrier and abort words
  cudaStream_t stream = nullptr;
  cudaStream_t body = nullptr;    // records the bodies of the graph's inner-loop nodes
  cudaEvent_t ev = nullptr;
  ~SolverWork() {
    if (ev) cudaEventDestroy(ev);
    if (stream) cudaStreamDestroy(stream);
    if (body) cudaStreamDestroy(body);
  }
};

void free_solver_work(fe_mesh* m) {
  delete m->work;
  m->work = nullptr;
}

// ---------------------------------------------------------------------------
// launch geometry for [N][R][3] vector kernels: blocks of K*R threads, thread
// (j, r) = (threadIdx.x / R, threadIdx.x % R) handles node n = block*K + j
// (grid-stride) and case r. K is the largest power of two with K*R <= 256.
// ---------------------------------------------------------------------------
struct VGeom {
  int R, K, tpb;
  unsigned grid;
};

static VGeom vgeom(int64_t N, int R, int sms) {
  VGeom g;
  g.R = R;
  g.K = 1;
  while (g.K * 2 * R <= 256) g.K *= 2;
  g.tpb = g.K * R;
  const int64_t need = (N + g.K - 1) / g.K;
  const int64_t cap = (int64_t)sms * 8;
  g.grid = (unsigned)(need < cap ? need : cap);
  return g;
}

// sums v over the K threads of each case in the block and adds the block total
// to out[r] (FP64 atomics). Every thread of the block must call it.
__device__ __forceinline__ void reduce_cases(double v, int R, int K, double* sm, double* out) {
  sm[threadIdx.x] = v;
  __syncthreads();
  const int j = threadIdx.x / R;
  for (int s = K >> 1; s > 0; s >>= 1) {
    if (j < s) sm[threadIdx.x] += sm[threadIdx.x + s * R];
    __syncthreads();
  }
  if (j == 0) atomicAdd(out + threadIdx.x, sm[threadIdx.x]);
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void mv3(const T* __restrict__ Mi, const T v[3], T z[3]) {
  z[0] = Mi[0] * v[0] + Mi[1] * v[1] + Mi[2] * v[2];
  z[1] = Mi[3] * v[0] + Mi[4] * v[1] + Mi[5] * v[2];
  z[2] = Mi[6] * v[0] + Mi[7] * v[1] + Mi[8] * v[2];
}

#define VEC_LOOP_BEGIN                                    \
  const int R = C.R;                                      \
  const int r = threadIdx.x % R;                          \
  const int K = blockDim.x / R;                           \
  const int64_t stride = (int64_t)gridDim.x * K;          \
  for (int64_t n = (int64_t)blockIdx.x * K + threadIdx.x / R; n < N; n += stride) { \
    const int64_t o = (n * R + r) * 3;

#define VEC_LOOP_END }

// ---------------------------------------------------------------------------
// block Jacobi: diagonal 3x3 blocks of K from the element closed form
//   B_aa = (lam + mu) G_a + mu tr(G_a) I,  G_a = int grad N_a (x) grad N_a dV,
//   corner: G_a = (3V/5) g_a g_a^T,
//   edge kl: G = (8V/5)(g_k g_k^T + g_l g_l^T) + (4V/5)(g_k g_l^T + g_l g_k^T),
// summed over elements, masked (constrained rows/columns -> identity), inverted.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void add_block(double* D, const double G[3][3], double lam, double mu) {
  const double tr = G[0][0] + G[1][1] + G[2][2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) atomicAdd(D + 3 * i + j, (lam + mu) * G[i][j] + (i == j ? mu * tr : 0.0));
}

__global__ void jacobi_diag_kernel(MeshView<double> M, double* __restrict__ Dg) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M.n_elem) return;
  int nd[10];
  for (int a = 0; a < 10; ++a) nd[a] = M.conn[10 * e + a];
  double xc[4][3];
  for (int k = 0; k < 4; ++k)
    for (int i = 0; i < 3; ++i) xc[k][i] = M.xyz[3 * (int64_t)nd[k] + i];
  ElemGeo<double> G;
  elem_geometry(xc[0], xc[1], xc[2], xc[3], M.mat[2 * e], M.mat[2 * e + 1], G);
  const double V = 20.0 * G.c;
  for (int a = 0; a < 4; ++a) {
    double Ga[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Ga[i][j] = 0.6 * V * G.g[a][i] * G.g[a][j];
    add_block(Dg + 9 * (int64_t)nd[a], Ga, G.lam, G.mu);
  }
  const int EK[6] = {0, 1, 0, 0, 1, 2}, EL[6] = {1, 2, 2, 3, 3, 3};
  for (int q = 0; q < 6; ++q) {
    const int k = EK[q], l = EL[q];
    double Ga[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        Ga[i][j] = 1.6 * V * (G.g[k][i] * G.g[k][j] + G.g[l][i] * G.g[l][j]) +
                   0.8 * V * (G.g[k][i] * G.g[l][j] + G.g[l][i] * G.g[k][j]);
    add_block(Dg + 9 * (int64_t)nd[edge_node(k, l)], Ga, G.lam, G.mu);
  }
}

__global__ void jacobi_invert_kernel(int64_t N, const uint8_t* __restrict__ nmask, const double* __restrict__ Dg,
                                     double* __restrict__ B64, float* __restrict__ B32, int* __restrict__ bad) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int mk = nmask[n];
  double A[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const bool fi = (mk >> i) & 1, fj = (mk >> j) & 1;
      A[i][j] = (fi && fj) ? Dg[9 * n + 3 * i + j] : (i == j ? 1.0 : 0.0);
    }
  const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
  const double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
  const double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
  const double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
  if (!(det > 0.0) || !isfinite(det)) {
    atomicExch(bad, 1);
    for (int k = 0; k < 9; ++k) {
      B64[9 * n + k] = (k % 4 == 0) ? 1.0 : 0.0;
      B32[9 * n + k] = (k % 4 == 0) ? 1.f : 0.f;
    }
    return;
  }
  const double id = 1.0 / det;
  double I[9];
  I[0] = c00 * id;
  I[1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * id;
  I[2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * id;
  I[3] = c01 * id;
  I[4] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * id;
  I[5] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * id;
  I[6] = c02 * id;
  I[7] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * id;
  I[8] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * id;
  for (int k = 0; k < 9; ++k) {
    B64[9 * n + k] = I[k];
    B32[9 * n + k] = (float)I[k];
  }
}

void build_block_jacobi(fe_mesh* m, cudaStream_t s) {
  if (m->jacobi_ready) return;
  const int64_t N = m->n_nodes, E = m->n_elem;
  DevBuf D, bad;
  D.alloc((size_t)N * 9 * sizeof(double));
  bad.alloc(sizeof(int));
  if (!m->binv64.ptr) m->binv64.alloc((size_t)N * 9 * sizeof(double));
  if (!m->binv32.ptr) m->binv32.alloc((size_t)N * 9 * sizeof(float));
  FE_CUDA(cudaMemsetAsync(D.ptr, 0, D.bytes, s));
  FE_CUDA(cudaMemsetAsync(bad.ptr, 0, sizeof(int), s));
  jacobi_diag_kernel<<<(unsigned)((E + 127) / 128), 128, 0, s>>>(m->view<double>(), D.as<double>());
  FE_CHECK_LAUNCH();
  jacobi_invert_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, m->nmask.as<uint8_t>(), D.as<double>(),
                                                                   m->binv64.as<double>(), m->binv32.as<float>(),
                                                                   bad.as<int>());
  FE_CHECK_LAUNCH();
  int hbad = 0;
  FE_CUDA(cudaMemcpyAsync(&hbad, bad.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  FE_CUDA(cudaStreamSynchronize(s));
  FE_REQUIRE(hbad == 0, "block Jacobi: a free node has a singular or indefinite diagonal block "
                        "(node touched by no element, or a degenerate material)");
  m->jacobi_ready = true;
}

// ---------------------------------------------------------------------------
// vector kernels (N nodes, R cases; blockDim = K*R)
// ---------------------------------------------------------------------------

// u <- P u ; fn2 += ||P f||^2 ; clears the u-is-zero flag (set to 1 before) if a
// free component of u is nonzero
__global__ void k_prepare(int64_t N, Cases C, const uint8_t* __restrict__ nmask, const double* __restrict__ f,
                          double* __restrict__ u) {
  extern __shared__ double sm[];
  double acc = 0.0;
  bool nz = false;
  VEC_LOOP_BEGIN
  const int mk = nmask[n];
  for (int c = 0; c < 3; ++c) {
    const bool fr = (mk >> c) & 1;
    const double fv = fr ? f[o + c] : 0.0;
    acc += fv * fv;
    if (!fr) u[o + c] = 0.0;
    else if (u[o + c] != 0.0) nz = true;
  }
  VEC_LOOP_END
  if (__any_sync(__activemask(), nz) && (threadIdx.x & 31) == 0) atomicAnd(C.done + 2, 0);
  reduce_cases(acc, C.R, blockDim.x / C.R, sm, C.d + D_FN2 * C.R);
}

// r = P f - q (q = K u, not computed when u = 0) ; rn2 += ||r||^2
__global__ void k_residual(int64_t N, Cases C, const uint8_t* __restrict__ nmask, const double* __restrict__ f,
                           const double* __restrict__ q, double* __restrict__ rv) {
  extern __shared__ double sm[];
  double acc = 0.0;
  const bool u_zero = C.done[2] != 0;
  VEC_LOOP_BEGIN
  const int mk = nmask[n];
  for (int c = 0; c < 3; ++c) {
    const double v = ((mk >> c) & 1) ? (u_zero ? f[o + c] : f[o + c] - q[o + c]) : 0.0;
    rv[o + c] = v;
    acc += v * v;
  }
  VEC_LOOP_END
  reduce_cases(acc, C.R, blockDim.x / C.R, sm, C.d + D_RN2 * C.R);
}

// PCG start: p = M^-1 r ; rho += (p, r)
__global__ void k_pcg_init(int64_t N, Cases C, const double* __restrict__ Bi, const double* __restrict__ rv,
                           double* __restrict__ p) {
  extern __shared__ double sm[];
  double acc = 0.0;
  VEC_LOOP_BEGIN
  double v[3] = {rv[o], rv[o + 1], rv[o + 2]}, z[3];
  mv3(Bi + 9 * n, v, z);
  for (int c = 0; c < 3; ++c) {
    p[o + c] = z[c];
    acc += z[c] * v[c];
  }
  VEC_LOOP_END
  reduce_cases(acc, C.R, blockDim.x / C.R, sm, C.d + D_RHO * C.R);
}

// PCG restart of the cases flagged RESTART (their r was replaced by the true
// residual): p = M^-1 r, rhoa += (M^-1 r, r) for those cases only
__global__ void k_pcg_restart(int64_t N, Cases C, const double* __restrict__ Bi, const double* __restrict__ rv,
                              double* __restrict__ p) {
  extern __shared__ double sm[];
  double acc = 0.0;
  VEC_LOOP_BEGIN
  if (C.I(I_RESTART, r)) {
    double v[3] = {rv[o], rv[o + 1], rv[o + 2]}, z[3];
    mv3(Bi + 9 * n, v, z);
    for (int c = 0; c < 3; ++c) {
      p[o + c] = z[c];
      acc += z[c] * v[c];
    }
  }
  VEC_LOOP_END
  reduce_cases(acc, C.R, blockDim.x / C.R, sm, C.d + D_RHOA * C.R);
}

// u_r = 0 for cases whose right-hand side is zero
__global__ void k_zero_trivial(int64_t N, Cases C, double* __restrict__ u) {
  VEC_LOOP_BEGIN
  if (!(C.D(D_FN2, r) > 0.0))
    for (int c = 0; c < 3; ++c) u[o + c] = 0.0;
  VEC_LOOP_END
}

// acc[field] += (a, b), inner loop (FP32) or outer (FP64); skipped when *skip
template <typename T>
__global__ void k_dot(int64_t N, Cases C, int field, const int* __restrict__ skip, const T* __restrict__ a,
                      const T* __restrict__ b) {
  extern __shared__ double sm[];
  if (skip && *skip) return;
  T acc = T(0);
  VEC_LOOP_BEGIN
  acc += a[o] * b[o] + a[o + 1] * b[o + 1] + a[o + 2] * b[o + 2];
  VEC_LOOP_END
  reduce_cases((double)acc, C.R, blockDim.x / C.R, sm, C.d + field * C.R);
}

// PCG update: u += a p ; r -= a q ; rhoa += (M^-1 r, r) ; rn2 += (r, r)
__global__ void k_pcg_update(int64_t N, Cases C, const double* __restrict__ Bi, double* __restrict__ u,
                             const double* __restrict__ p, double* __restrict__ rv, const double* __restrict__ q) {
  extern __shared__ double sm[];
  double a1 = 0.0, a2 = 0.0;
  VEC_LOOP_BEGIN
  if (C.I(I_ACTIVE, r)) {
    const double al = C.D(D_ALPHA, r);
    double v[3], z[3];
    for (int c = 0; c < 3; ++c) {
      u[o + c] += al * p[o + c];
      v[c] = rv[o + c] - al * q[o + c];
      rv[o + c] = v[c];
    }
    mv3(Bi + 9 * n, v, z);
    a1 += z[0] * v[0] + z[1] * v[1] + z[2] * v[2];
    a2 += v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  }
  VEC_LOOP_END
  reduce_cases(a1, C.R, blockDim.x / C.R, sm, C.d + D_RHOA * C.R);
  reduce_cases(a2, C.R, blockDim.x / C.R, sm, C.d + D_RN2 * C.R);
}

// PCG direction: p = M^-1 r + beta p (restarted cases: beta = 0)
__global__ void k_pcg_p(int64_t N, Cases C, const double* __restrict__ Bi, const double* __restrict__ rv,
                        double* __restrict__ p) {
  VEC_LOOP_BEGIN
  if (C.I(I_ACTIVE, r)) {
    const double be = C.D(D_BETA, r);
    double v[3] = {rv[o], rv[o + 1], rv[o + 2]}, z[3];
    mv3(Bi + 9 * n, v, z);
    for (int c = 0; c < 3; ++c) p[o + c] = z[c] + be * p[o + c];
  }
  VEC_LOOP_END
}

// FCG inner start (Algorithm 1(a)): rbar = (float) r ; ubar = Mbar^-1 rbar ;
// rbn2 += ||rbar||^2. Inactive cases get zeros.
__global__ void k_cast_start(int64_t N, Cases C, const float* __restrict__ Bi, const double* __restrict__ rv,
                             float* __restrict__ rb, float* __restrict__ ub) {
  extern __shared__ double sm[];
  float acc = 0.f;
  VEC_LOOP_BEGIN
  const bool act = C.I(I_ACTIVE, r);
  float v[3], z[3];
  for (int c = 0; c < 3; ++c) v[c] = act ? (float)rv[o + c] : 0.f;
  mv3(Bi + 9 * n, v, z);
  for (int c = 0; c < 3; ++c) {
    rb[o + c] = v[c];
    ub[o + c] = z[c];
    acc += v[c] * v[c];
  }
  VEC_LOOP_END
  reduce_cases((double)acc, C.R, blockDim.x / C.R, sm, C.d + D_RBN2 * C.R);
}

// Algorithm 1(b), start: e = rbar - Kbar ubar (q holds Kbar ubar); en2 += ||e||^2 ;
// rhoa += (Mbar^-1 e, e)
__global__ void k_inner_resid(int64_t N, Cases C, const float* __restrict__ Bi, const float* __restrict__ rb,
                              const float* __restrict__ qb, float* __restrict__ eb) {
  extern __shared__ double sm[];
  float a1 = 0.f, a2 = 0.f;
  VEC_LOOP_BEGIN
  float v[3], z[3];
  for (int c = 0; c < 3; ++c) {
    v[c] = rb[o + c] - qb[o + c];
    eb[o + c] = v[c];
  }
  mv3(Bi + 9 * n, v, z);
  a1 += v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  a2 += z[0] * v[0] + z[1] * v[1] + z[2] * v[2];
  VEC_LOOP_END
  reduce_cases((double)a1, C.R, blockDim.x / C.R, sm, C.d + D_EN2 * C.R);
  reduce_cases((double)a2, C.R, blockDim.x / C.R, sm, C.d + D_RHOA * C.R);
}

// Algorithm 1(b), search direction: pbar = Mbar^-1 e + beta pbar
__global__ void k_inner_p(int64_t N, Cases C, const float* __restrict__ Bi, const float* __restrict__ eb,
                          float* __restrict__ pb) {
  if (*C.done) return;
  VEC_LOOP_BEGIN
  const float be = (float)C.D(D_BETAI, r);
  float v[3] = {eb[o], eb[o + 1], eb[o + 2]}, z[3];
  mv3(Bi + 9 * n, v, z);
  // the first step (beta = 0) must not read pbar: it holds the previous solve's data
  if (be != 0.f)
    for (int c = 0; c < 3; ++c) pb[o + c] = z[c] + be * pb[o + c];
  else
    for (int c = 0; c < 3; ++c) pb[o + c] = z[c];
  VEC_LOOP_END
}

// Algorithm 1(b), update: e -= alpha q ; ubar += alpha p ; then en2, rhoa for the next step
__global__ void k_inner_update(int64_t N, Cases C, const float* __restrict__ Bi, float* __restrict__ eb,
                               const float* __restrict__ qb, float* __restrict__ ub, const float* __restrict__ pb) {
  extern __shared__ double sm[];
  if (*C.done) return;
  float a1 = 0.f, a2 = 0.f;
  VEC_LOOP_BEGIN
  const float al = (float)C.D(D_ALPHAI, r);
  float v[3], z[3];
  for (int c = 0; c < 3; ++c) {
    v[c] = eb[o + c] - al * qb[o + c];
    eb[o + c] = v[c];
    ub[o + c] += al * pb[o + c];
  }
  mv3(Bi + 9 * n, v, z);
  a1 += v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
  a2 += z[0] * v[0] + z[1] * v[1] + z[2] * v[2];
  VEC_LOOP_END
  reduce_cases((double)a1, C.R, blockDim.x / C.R, sm, C.d + D_EN2 * C.R);
  reduce_cases((double)a2, C.R, blockDim.x / C.R, sm, C.d + D_RHOA * C.R);
}

// zq += ((double) ubar, q_prev)
__global__ void k_outer_zq(int64_t N, Cases C, const float* __restrict__ ub, const double* __restrict__ q) {
  extern __shared__ double sm[];
  double acc = 0.0;
  VEC_LOOP_BEGIN
  acc += (double)ub[o] * q[o] + (double)ub[o + 1] * q[o + 1] + (double)ub[o + 2] * q[o + 2];
  VEC_LOOP_END
  reduce_cases(acc, C.R, blockDim.x / C.R, sm, C.d + D_ZQ * C.R);
}

// Algorithm 1(a), search direction: p = z + beta p with z = (double) ubar
__global__ void k_outer_p(int64_t N, Cases C, const float* __restrict__ ub, double* __restrict__ p) {
  VEC_LOOP_BEGIN
  if (C.I(I_ACTIVE, r)) {
    const double be = C.D(D_BETA, r);
    if (be != 0.0)
      for (int c = 0; c < 3; ++c) p[o + c] = (double)ub[o + c] + be * p[o + c];
    else
      for (int c = 0; c < 3; ++c) p[o + c] = (double)ub[o + c];
  }
  VEC_LOOP_END
}

// Algorithm 1(a): rho += (z, r) ; gam += (p, q)
__global__ void k_outer_dots(int64_t N, Cases C, const float* __restrict__ ub, const double* __restrict__ rv,
                             const double* __restrict__ p, const double* __restrict__ q) {
  extern __shared__ double sm[];
  double a1 = 0.0, a2 = 0.0;
  VEC_LOOP_BEGIN
  for (int c = 0; c < 3; ++c) {
    a1 += (double)ub[o + c] * rv[o + c];
    a2 += p[o + c] * q[o + c];
  }
  VEC_LOOP_END
  reduce_cases(a1, C.R, blockDim.x / C.R, sm, C.d + D_RHO * C.R);
  reduce_cases(a2, C.R, blockDim.x / C.R, sm, C.d + D_GAM * C.R);
}

// Algorithm 1(a), update: r -= alpha q ; u += alpha p ; rn2 += ||r||^2
__global__ void k_outer_update(int64_t N, Cases C, double* __restrict__ rv, const double* __restrict__ q,
                               double* __restrict__ u, const double* __restrict__ p) {
  extern __shared__ double sm[];
  double acc = 0.0;
  VEC_LOOP_BEGIN
  if (C.I(I_ACTIVE, r)) {
    const double al = C.D(D_ALPHA, r);
    for (int c = 0; c < 3; ++c) {
      const double v = rv[o + c] - al * q[o + c];
      rv[o + c] = v;
      u[o + c] += al * p[o + c];
      acc += v * v;
    }
  }
  VEC_LOOP_END
  reduce_cases(acc, C.R, blockDim.x / C.R, sm, C.d + D_RN2 * C.R);
}

// true residuals of the candidate cases from one all-case product t = K u:
// r_c = P f_c - t_c written for them, rt2[c] += ||r_c||^2
__global__ void k_cand_resid(int64_t N, Cases C, const uint8_t* __restrict__ nmask, const double* __restrict__ f,
                             const double* __restrict__ t, double* __restrict__ rv) {
  extern __shared__ double sm[];
  double acc = 0.0;
  VEC_LOOP_BEGIN
  if (C.I(I_CAND, r)) {
    const int mk = nmask[n];
    for (int c = 0; c < 3; ++c) {
      const double v = ((mk >> c) & 1) ? f[o + c] - t[o + c] : 0.0;
      rv[o + c] = v;
      acc += v * v;
    }
  }
  VEC_LOOP_END
  reduce_cases(acc, C.R, blockDim.x / C.R, sm, C.d + D_RT2 * C.R);
}

// single-case helpers for the true-residual confirmation
__global__ void k_gather_case(int64_t N, int R, int c, const double* __restrict__ u, double* __restrict__ t) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  for (int k = 0; k < 3; ++k) t[3 * n + k] = u[(n * R + c) * 3 + k];
}

// rt2[c] = ||P f_c - t||^2 ; if `write_r`, r_c = P f_c - t
__global__ void k_case_resid(int64_t N, int R, int c, const uint8_t* __restrict__ nmask, const double* __restrict__ f,
                             const double* __restrict__ t, double* __restrict__ rv, int write_r,
                             double* __restrict__ out) {
  __shared__ double sm[256];
  double acc = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const int mk = nmask[n];
    for (int k = 0; k < 3; ++k) {
      const double v = ((mk >> k) & 1) ? f[(n * R + c) * 3 + k] - t[3 * n + k] : 0.0;
      if (write_r) rv[(n * R + c) * 3 + k] = v;
      acc += v * v;
    }
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, sm[0]);
}

// ---------------------------------------------------------------------------
// slot management of the many-case driver
// ---------------------------------------------------------------------------
// slot r <- case: F[:, r, :] = f_case, U[:, r, :] = 0 (f_case is [N][3])
__global__ void k_load_case(int64_t N, int R, int r, const double* __restrict__ fc, double* __restrict__ F,
                            double* __restrict__ U) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  for (int k = 0; k < 3; ++k) {
    F[(n * R + r) * 3 + k] = fc[3 * n + k];
    U[(n * R + r) * 3 + k] = 0.0;
  }
}

// u_case <- U[:, r, :]
__global__ void k_store_case(int64_t N, int R, int r, const double* __restrict__ U, double* __restrict__ uc) {
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= N) return;
  for (int k = 0; k < 3; ++k) uc[3 * n + k] = U[(n * R + r) * 3 + k];
}

// slot r starts from u = 0: r = P f, ||P f||^2 into fn2 and rn2 (both zeroed before)
__global__ void k_slot_init(int64_t N, int R, int r, const uint8_t* __restrict__ nmask, const double* __restrict__ F,
                            double* __restrict__ rv, double* __restrict__ fn2, double* __restrict__ rn2) {
  __shared__ double sm[256];
  double acc = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const int mk = nmask[n];
    for (int k = 0; k < 3; ++k) {
      const int64_t o = (n * R + r) * 3 + k;
      const double v = ((mk >> k) & 1) ? F[o] : 0.0;
      rv[o] = v;
      acc += v * v;
    }
  }
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(fn2, sm[0]);
    atomicAdd(rn2, sm[0]);
  }
}

// per-case state of a freshly loaded slot (one thread)
__global__ void s_slot_start(Cases C, int r, int pcg) {
  const bool zero = !(C.D(D_FN2, r) > 0.0);
  C.I(I_ACTIVE, r) = zero ? 0 : 1;
  C.I(I_CAND, r) = 0;
  C.I(I_RESTART, r) = (!zero && pcg) ? 1 : 0;   // PCG: p and rho from r at the next restart pass
  C.I(I_FIRST, r) = 1;
  C.I(I_STATUS, r) = FE_OK;
  C.I(I_OUTER, r) = 0;
  C.I(I_INNER, r) = 0;
  C.I(I_INNER1, r) = 0;
  C.I(I_INNER2, r) = 0;
  C.D(D_RELRES, r) = 0.0;
}

// ---------------------------------------------------------------------------
// per-case scalar kernels (one block of R threads)
// ---------------------------------------------------------------------------
__global__ void s_init(Cases C) {
  const int r = threadIdx.x;
  for (int f = 0; f < D_COUNT; ++f) C.D(f, r) = 0.0;
  for (int f = 0; f < I_COUNT; ++f) C.I(f, r) = 0;
  C.I(I_FIRST, r) = 1;
  if (r == 0) {
    C.done[0] = 0;
    C.done[2] = 1;  // u = 0 until k_prepare finds a nonzero free component
  }
}

// after ||f||^2 and ||r||^2: cases with f = 0 are finished (u = 0); others start
__global__ void s_start(Cases C, double tol, int reset_u_for_zero_f) {
  const int r = threadIdx.x;
  const double fn2 = C.D(D_FN2, r);
  const bool zero = !(fn2 > 0.0);
  C.I(I_ACTIVE, r) = zero ? 0 : 1;
  C.I(I_STATUS, r) = FE_OK;
  C.D(D_RELRES, r) = zero ? 0.0 : sqrt(C.D(D_RN2, r) / fn2);
  if (!zero && C.D(D_RN2, r) <= tol * tol * fn2) {
    C.I(I_ACTIVE, r) = 0;   // the initial guess already meets the tolerance: confirm on the host
    C.I(I_CAND, r) = 1;
  }
  (void)reset_u_for_zero_f;
}

__global__ void s_pcg_restart(Cases C) {
  const int r = threadIdx.x;
  if (C.I(I_RESTART, r)) {
    C.D(D_RHO, r) = C.D(D_RHOA, r);
    C.I(I_RESTART, r) = 0;
  }
  C.D(D_RHOA, r) = 0.0;
}

// PCG: alpha = rho / (p, q)
__global__ void s_pcg_alpha(Cases C) {
  const int r = threadIdx.x;
  const double g = C.D(D_GAM, r);
  C.D(D_GAM, r) = 0.0;
  C.D(D_RHOA, r) = 0.0;
  C.D(D_RN2, r) = 0.0;
  if (!C.I(I_ACTIVE, r)) {
    C.D(D_ALPHA, r) = 0.0;
    return;
  }
  const double rho = C.D(D_RHO, r);
  if (!(g > 0.0) || !isfinite(g) || !isfinite(rho)) {
    C.I(I_ACTIVE, r) = 0;
    C.I(I_STATUS, r) = FE_EBREAKDOWN;
    C.D(D_ALPHA, r) = 0.0;
    return;
  }
  C.D(D_ALPHA, r) = rho / g;
}

// PCG: beta = rho_new / rho, convergence and iteration cap
__global__ void s_pcg_beta(Cases C, double tol, int max_it) {
  const int r = threadIdx.x;
  if (!C.I(I_ACTIVE, r)) {
    C.D(D_BETA, r) = 0.0;
    return;
  }
  const double rn = C.D(D_RHOA, r);
  C.D(D_BETA, r) = rn / C.D(D_RHO, r);
  C.D(D_RHO, r) = rn;
  const int k = C.I(I_OUTER, r);
  if (C.hist && k < C.hist_len) {
    C.hist[((int64_t)k * C.R + r) * 2] = C.D(D_ALPHA, r);
    C.hist[((int64_t)k * C.R + r) * 2 + 1] = C.D(D_BETA, r);
  }
  C.I(I_OUTER, r) += 1;
  const double rn2 = C.D(D_RN2, r), fn2 = C.D(D_FN2, r);
  if (!isfinite(rn2)) {
    C.I(I_ACTIVE, r) = 0;
    C.I(I_STATUS, r) = FE_EBREAKDOWN;
  } else if (rn2 <= tol * tol * fn2) {
    C.I(I_ACTIVE, r) = 0;
    C.I(I_CAND, r) = 1;
  } else if (C.I(I_OUTER, r) >= max_it) {
    C.I(I_ACTIVE, r) = 0;
    C.I(I_STATUS, r) = FE_ENOCONV;
  }
}

// FCG: start of one outer iteration
__global__ void s_outer_begin(Cases C) {
  const int r = threadIdx.x;
  C.D(D_RBN2, r) = 0.0;
  C.D(D_RBN21, r) = 0.0;
  C.D(D_RBN22, r) = 0.0;
  C.D(D_EN2, r) = 0.0;
  C.D(D_RHOA, r) = 0.0;
  C.D(D_ZQ, r) = 0.0;
  if (r == 0) {
    *C.done = 0;
    C.step() = 0;
  }
}

// between two inner loops of one outer iteration (level 1, then level 0)
__global__ void s_level_begin(Cases C) {
  const int r = threadIdx.x;
  C.D(D_EN2, r) = 0.0;
  C.D(D_RHOA, r) = 0.0;
  C.D(D_RHOB, r) = 0.0;
  C.D(D_GAMI, r) = 0.0;
  if (r == 0) {
    *C.done = 0;
    C.step() = 0;
  }
}

// inner stop test before the next step and inner beta (Algorithm 1(b)).
// The step index is the device counter; with `loop` set, the stop decision is
// also the condition of the graph's while node that repeats the inner step, so
// the loop ends on the device after at most n_inner steps.
__global__ void s_inner_check(Cases C, int n_inner, double eps, int f_rbn2, cudaGraphConditionalHandle loop,
                              int use_loop) {
  __shared__ int go;
  const int r = threadIdx.x;
  if (r == 0) go = 0;
  __syncthreads();
  if (*C.done) {
    if (use_loop && r == 0) cudaGraphSetConditional(loop, 0);
    return;
  }
  const int step = C.step();
  const double rb = C.D(f_rbn2, r);
  const bool act = C.I(I_ACTIVE, r) && rb > 0.0;
  const double ratio = C.D(D_EN2, r) / rb;
  if (act && !(ratio <= eps)) atomicOr(&go, 1);   // NaN counts as "not converged"
  __syncthreads();
  const bool stop = !go || step >= n_inner;
  const double rhob = C.D(D_RHOB, r);
  C.D(D_BETAI, r) = (step > 0 && rhob != 0.0 && act) ? C.D(D_RHOA, r) / rhob : 0.0;
  C.D(D_GAMI, r) = 0.0;
  if (r == 0) {
    if (stop) *C.done = 1;
    C.step() = step + 1;
    if (use_loop) cudaGraphSetConditional(loop, stop ? 0u : 1u);
  }
}

// inner alpha (Algorithm 1(b))
__global__ void s_inner_alpha(Cases C, int f_rbn2, int f_count) {
  const int r = threadIdx.x;
  if (*C.done) return;
  const double g = C.D(D_GAMI, r), rho = C.D(D_RHOA, r);
  const bool ok = C.I(I_ACTIVE, r) && C.D(f_rbn2, r) > 0.0 && g > 0.0 && isfinite(g) && isfinite(rho);
  C.D(D_ALPHAI, r) = ok ? rho / g : 0.0;
  C.D(D_RHOB, r) = rho;
  C.D(D_EN2, r) = 0.0;
  C.D(D_RHOA, r) = 0.0;
  if (C.I(I_ACTIVE, r)) C.I(f_count, r) += 1;
}

// outer beta (Algorithm 1(a), read as flexible CG unless literal)
__global__ void s_outer_beta(Cases C, int literal) {
  const int r = threadIdx.x;
  double be = 0.0;
  if (C.I(I_ACTIVE, r) && !C.I(I_FIRST, r) && !C.I(I_RESTART, r)) {
    const double zq = C.D(D_ZQ, r);
    be = literal ? zq / C.D(D_RHOP, r) : -zq / C.D(D_PQP, r);
    if (!isfinite(be)) be = 0.0;
  }
  if (C.I(I_ACTIVE, r)) {
    C.I(I_FIRST, r) = 0;
    C.I(I_RESTART, r) = 0;
  }
  C.D(D_BETA, r) = be;
  C.D(D_RHO, r) = 0.0;
  C.D(D_GAM, r) = 0.0;
}

// outer alpha (Algorithm 1(a)) and bookkeeping
__global__ void s_outer_alpha(Cases C) {
  const int r = threadIdx.x;
  C.D(D_RN2, r) = 0.0;
  if (!C.I(I_ACTIVE, r)) {
    C.D(D_ALPHA, r) = 0.0;
    return;
  }
  const double g = C.D(D_GAM, r), rho = C.D(D_RHO, r);
  if (!(g > 0.0) || !isfinite(g) || !isfinite(rho)) {
    C.I(I_ACTIVE, r) = 0;
    C.I(I_STATUS, r) = FE_EBREAKDOWN;
    C.D(D_ALPHA, r) = 0.0;
    return;
  }
  C.D(D_ALPHA, r) = rho / g;
  C.D(D_PQP, r) = g;
  C.D(D_RHOP, r) = rho;
  C.I(I_OUTER, r) += 1;
}

// outer stop test (Algorithm 1(a), per case) and iteration cap
__global__ void s_outer_check(Cases C, double tol, int max_outer) {
  const int r = threadIdx.x;
  if (!C.I(I_ACTIVE, r)) return;
  const double rn2 = C.D(D_RN2, r), fn2 = C.D(D_FN2, r);
  if (!isfinite(rn2)) {
    C.I(I_ACTIVE, r) = 0;
    C.I(I_STATUS, r) = FE_EBREAKDOWN;
  } else if (rn2 <= tol * tol * fn2) {
    C.I(I_ACTIVE, r) = 0;
    C.I(I_CAND, r) = 1;
  } else if (C.I(I_OUTER, r) >= max_outer) {
    C.I(I_ACTIVE, r) = 0;
    C.I(I_STATUS, r) = FE_ENOCONV;
  }
}

// ---------------------------------------------------------------------------
// One inner loop (Algorithm 1(b)) on an assembled block-CSR level (levels 1
// and 2) as a single persistent kernel. The per-step launches above cost more
// than the arithmetic on these levels (a few MB per vector), so here all steps
// run in one cooperative launch whose CTAs meet at grid-wide barriers: three
// per step (after the new search direction, after q = A p and its dot, after
// the update and its two dots). Every CTA evaluates the per-case scalars
// (alpha, beta, the stop rule) itself from the reduced sums, so they agree
// without a further exchange; CTA 0 records them and the step counts in the
// case state. The arithmetic of each vector pass is that of k_inner_resid,
// k_inner_p, k_dot and k_inner_update. A thread owns 4 cases of a node (R a
// power of two from 4 to 32), so its cases are the same in every pass.
// Each barrier wait is bounded (about a second of SM clock); a wait that runs
// out sets the mesh's status word, raises the kernel's abort flag (which the
// other CTAs see in their waits) and every CTA returns.
// ---------------------------------------------------------------------------
struct InnerArgs {
  int64_t N;
  Cases C;
  const float* B;                                  // [N][9] inverse diagonal blocks
  const float* rb;
  float *ub, *eb, *pb, *qb;                        // [N][R][3]
  const int32_t* rowptr;                           // [N + 1]
  const int32_t* cols;                             // plain block CSR [nnzb]
  const float* vals;                               // [nnzb][9]
  const int32_t* sl_off;                           // sliced copy (optional): [slices + 1]
  const int32_t* sl_cols;                          // [slots][8]
  const float* sl_vals;                            // [slots][9][8]
  int n_inner;
  double eps;
  int f_rbn2, f_count;
  double* acc;                                     // [2][3][R] per-parity sums: gamma, ||e||^2, rho
  unsigned* bar;                                   // [2] arrival count, generation
  int* abort_flag;
  int* status;
  long long timeout;
};

enum { A_GAM = 0, A_EN2 = 1, A_RHO = 2 };

__device__ __forceinline__ double* acc_at(const InnerArgs& A, int parity, int field) {
  return A.acc + ((size_t)parity * 3 + field) * A.C.R;
}

// grid-wide barrier of a cooperative launch; false once any CTA gave up a wait
__device__ __forceinline__ bool grid_barrier(const InnerArgs& A) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = A.bar + 1;
    volatile int* abort_flag = A.abort_flag;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(A.bar, 1u) == gridDim.x - 1) {
      atomicExch(A.bar, 0u);
      __threadfence();
      atomicAdd(A.bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g0 && !*abort_flag) {
        if (clock64() - t0 > A.timeout) {
          atomicExch(A.abort_flag, 1);
          atomicExch(A.status, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = !*abort_flag;
  }
  __syncthreads();
  return ok_s != 0;
}

// Two blocks, of which only block 0 reaches the grid-wide barrier: its wait, limited
// to A.timeout cycles, gives up, raises the abort flag and records it in *A.status.
__global__ void grid_wait_selftest_kernel(InnerArgs A) {
  if (blockIdx.x != 0) return;
  grid_barrier(A);
}

// q (12 values: 4 cases x 3) of block row a times x, cases r0 .. r0 + 3
template <bool SLICED>
__device__ __forceinline__ void row_times(const InnerArgs& A, int64_t a, int r0, const float* __restrict__ x,
                                          float acc[12]) {
  const int R = A.C.R;
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = 0.f;
  const int q0 = __ldg(A.rowptr + a), len = __ldg(A.rowptr + a + 1) - q0;
  const int rr = (int)(a & 7);
  const int64_t base = SLICED ? (int64_t)__ldg(A.sl_off + (a >> 3)) : 0;
  for (int t = 0; t < len; ++t) {
    int64_t b;
    float m[9];
    if (SLICED) {
      const int64_t slot = base + t;
      b = __ldg(A.sl_cols + slot * 8 + rr);
      const float* Bk = A.sl_vals + slot * 72 + rr;
#pragma unroll
      for (int k = 0; k < 9; ++k) m[k] = __ldg(Bk + 8 * k);
    } else {
      b = __ldg(A.cols + q0 + t);
      const float* Bk = A.vals + 9 * (int64_t)(q0 + t);
#pragma unroll
      for (int k = 0; k < 9; ++k) m[k] = __ldg(Bk + k);
    }
    // x was written by other CTAs earlier in this kernel: read through L2 (__ldcg),
    // never from a line this SM's L1 may still hold from an earlier step
    const float4* xb = reinterpret_cast<const float4*>(x + (b * R + r0) * 3);
    const float4 v0 = __ldcg(xb), v1 = __ldcg(xb + 1), v2 = __ldcg(xb + 2);
    const float v[12] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x, v2.y, v2.z, v2.w};
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        acc[3 * w + i] += m[3 * i] * v[3 * w] + m[3 * i + 1] * v[3 * w + 1] + m[3 * i + 2] * v[3 * w + 2];
  }
}

__device__ __forceinline__ void load12(const float* p, float v[12]) {
  const float4* q = reinterpret_cast<const float4*>(p);
  const float4 a = q[0], b = q[1], c = q[2];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  v[8] = c.x; v[9] = c.y; v[10] = c.z; v[11] = c.w;
}

__device__ __forceinline__ void store12(float* p, const float v[12]) {
  float4* q = reinterpret_cast<float4*>(p);
  q[0] = make_float4(v[0], v[1], v[2], v[3]);
  q[1] = make_float4(v[4], v[5], v[6], v[7]);
  q[2] = make_float4(v[8], v[9], v[10], v[11]);
}

__device__ __forceinline__ void load_block(const float* __restrict__ Bi, int64_t a, float m[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) m[k] = __ldg(Bi + 9 * a + k);
}

// adds a thread's 4-case partial sums (FP32, widened) of NF consecutive fields
// to the per-parity global sums at out[f R + r]: warp shuffles over the lanes
// holding the same cases,
// FP64 shared atomics per CTA, one FP64 global atomic per CTA, case and field
template <int NF>
__device__ __forceinline__ void reduce4(const InnerArgs& A, int r0, const float (&part)[NF][4], double* out,
                                        double* sm) {
  const int R = A.C.R, G = R / 4;
  for (int i = threadIdx.x; i < NF * R; i += blockDim.x) sm[i] = 0.0;
  __syncthreads();
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double v = (double)part[f][c];
      for (int off = 16; off >= G; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if ((threadIdx.x & 31) < G) atomicAdd(sm + f * R + r0 + c, v);
    }
  __syncthreads();
  for (int i = threadIdx.x; i < NF * R; i += blockDim.x) atomicAdd(out + i, sm[i]);
}

constexpr int kInnerThreads = 1024;   // one CTA per SM: fewer arrivals per grid barrier

template <bool SLICED>
__global__ void __launch_bounds__(kInnerThreads, 1) k_inner_persistent(InnerArgs A) {
  __shared__ double sm[3 * 32];
  __shared__ float s_alpha[32], s_beta[32];
  __shared__ double s_rhob[32], s_en2[32], s_rho[32];
  __shared__ int s_go;
  const Cases& C = A.C;
  const int R = C.R, G = R / 4;
  const int64_t items = A.N * G;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int r0 = (int)(gid % G) * 4;   // the same 4 cases in every pass (stride is a multiple of G)
  const bool lead = blockIdx.x == 0;

  // start: q = A ubar, e = rbar - q, ||e||^2 and (M^-1 e, e) (k_inner_resid)
  {
    float part[2][4] = {};
    for (int64_t i = gid; i < items; i += stride) {
      const int64_t a = i / G;
      const int64_t o = (a * R + r0) * 3;
      float q[12], rv[12], m[9];
      row_times<SLICED>(A, a, r0, A.ub, q);
      load12(A.rb + o, rv);
      load_block(A.B, a, m);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float v[3] = {rv[3 * c] - q[3 * c], rv[3 * c + 1] - q[3 * c + 1], rv[3 * c + 2] - q[3 * c + 2]}, z[3];
        rv[3 * c] = v[0];
        rv[3 * c + 1] = v[1];
        rv[3 * c + 2] = v[2];
        mv3(m, v, z);
        part[0][c] += v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        part[1][c] += z[0] * v[0] + z[1] * v[1] + z[2] * v[2];
      }
      store12(A.eb + o, rv);
    }
    reduce4<2>(A, r0, part, acc_at(A, 0, A_EN2), sm);   // EN2 and RHO are consecutive fields
  }
  if (!grid_barrier(A)) return;

  int step = 0;
  for (;; ++step) {
    const int par = step & 1;
    // stop test and beta (s_inner_check)
    if (threadIdx.x == 0) s_go = 0;
    __syncthreads();
    if (threadIdx.x < R) {
      const int r = threadIdx.x;
      const double rbn = C.D(A.f_rbn2, r);
      const bool act = C.I(I_ACTIVE, r) && rbn > 0.0;
      const double en2 = *(volatile double*)(acc_at(A, par, A_EN2) + r);
      const double rho = *(volatile double*)(acc_at(A, par, A_RHO) + r);
      if (act && !(en2 / rbn <= A.eps)) atomicOr(&s_go, 1);   // NaN counts as "not converged"
      const double rhob = step > 0 ? s_rhob[r] : 0.0;
      const double be = (step > 0 && rhob != 0.0 && act) ? rho / rhob : 0.0;
      s_beta[r] = (float)be;
      s_en2[r] = en2;
      s_rho[r] = rho;
      if (lead) {
        C.D(D_BETAI, r) = be;
        C.D(D_EN2, r) = en2;
        C.D(D_RHOA, r) = rho;
        C.D(D_GAMI, r) = 0.0;
      }
    }
    __syncthreads();
    const bool stop = !s_go || step >= A.n_inner;
    if (stop) break;

    // search direction: pbar = Mbar^-1 e + beta pbar (k_inner_p)
    for (int64_t i = gid; i < items; i += stride) {
      const int64_t a = i / G;
      const int64_t o = (a * R + r0) * 3;
      float e[12], p[12], m[9];
      load12(A.eb + o, e);
      load12(A.pb + o, p);
      load_block(A.B, a, m);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float be = s_beta[r0 + c];
        float z[3];
        mv3(m, e + 3 * c, z);
#pragma unroll
        for (int k = 0; k < 3; ++k) p[3 * c + k] = be != 0.f ? z[k] + be * p[3 * c + k] : z[k];
      }
      store12(A.pb + o, p);
    }
    if (!grid_barrier(A)) return;

    // q = Abar pbar and gamma = (pbar, q); CTA 0 clears the sums the next steps add to
    if (lead)
      for (int i = threadIdx.x; i < R; i += blockDim.x) {
        acc_at(A, par, A_EN2)[i] = 0.0;
        acc_at(A, par, A_RHO)[i] = 0.0;
        acc_at(A, par ^ 1, A_GAM)[i] = 0.0;
      }
    {
      float part[1][4] = {};
      for (int64_t i = gid; i < items; i += stride) {
        const int64_t a = i / G;
        const int64_t o = (a * R + r0) * 3;
        float q[12], p[12];
        row_times<SLICED>(A, a, r0, A.pb, q);
        store12(A.qb + o, q);
        load12(A.pb + o, p);
#pragma unroll
        for (int c = 0; c < 4; ++c) part[0][c] += p[3 * c] * q[3 * c] + p[3 * c + 1] * q[3 * c + 1] + p[3 * c + 2] * q[3 * c + 2];
      }
      reduce4<1>(A, r0, part, acc_at(A, par, A_GAM), sm);
    }
    if (!grid_barrier(A)) return;

    // alpha (s_inner_alpha)
    if (threadIdx.x < R) {
      const int r = threadIdx.x;
      const double g = *(volatile double*)(acc_at(A, par, A_GAM) + r), rho = s_rho[r];
      const bool ok = C.I(I_ACTIVE, r) && C.D(A.f_rbn2, r) > 0.0 && g > 0.0 && isfinite(g) && isfinite(rho);
      const double al = ok ? rho / g : 0.0;
      s_alpha[r] = (float)al;
      s_rhob[r] = rho;
      if (lead) {
        C.D(D_GAMI, r) = g;
        C.D(D_ALPHAI, r) = al;
        C.D(D_RHOB, r) = rho;
        if (C.I(I_ACTIVE, r)) C.I(A.f_count, r) += 1;
      }
    }
    __syncthreads();

    // e -= alpha q ; ubar += alpha p ; ||e||^2, (M^-1 e, e) (k_inner_update)
    {
      float part[2][4] = {};
      for (int64_t i = gid; i < items; i += stride) {
        const int64_t a = i / G;
        const int64_t o = (a * R + r0) * 3;
        float e[12], q[12], u[12], p[12], m[9];
        load12(A.eb + o, e);
        load12(A.qb + o, q);
        load12(A.ub + o, u);
        load12(A.pb + o, p);
        load_block(A.B, a, m);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float al = s_alpha[r0 + c];
          float v[3], z[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            v[k] = e[3 * c + k] - al * q[3 * c + k];
            e[3 * c + k] = v[k];
            u[3 * c + k] += al * p[3 * c + k];
          }
          mv3(m, v, z);
          part[0][c] += v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
          part[1][c] += z[0] * v[0] + z[1] * v[1] + z[2] * v[2];
        }
        store12(A.eb + o, e);
        store12(A.ub + o, u);
      }
      reduce4<2>(A, r0, part, acc_at(A, par ^ 1, A_EN2), sm);
    }
    if (!grid_barrier(A)) return;
  }
  // the loop's end state, as the per-step kernels leave it
  if (lead && threadIdx.x == 0) {
    *C.done = 1;
    C.step() = step + 1;
  }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
struct Solve {
  fe_mesh* m;
  SolverWork* w;
  int R;
  int64_t N;
  Cases C;
  VGeom g;
  size_t sm;  // shared bytes of reducing vector kernels
  int64_t N1 = 0;  // level-1 nodes (0: no coarse level)
  VGeom g1;
  int64_t N2 = 0;  // level-2 aggregates (0: no level 2)
  VGeom g2;
  bool assembled1 = false;  // level-1 operator: assembled block CSR, else element by element
  cudaStream_t s;
  const double* f;
  double* u;
  fe_solve_opts o;

  template <typename K, typename... A>
  void vec(K kern, A... args) {
    kern<<<g.grid, g.tpb, sm, s>>>(N, C, args...);
    FE_CHECK_LAUNCH();
  }
  // the same vector kernel over `n` nodes with launch geometry `gg` (level 1)
  template <typename K, typename... A>
  void vec_on(int64_t n, const VGeom& gg, K kern, A... args) {
    kern<<<gg.grid, gg.tpb, sm, s>>>(n, C, args...);
    FE_CHECK_LAUNCH();
  }
  template <typename K, typename... A>
  void scal(K kern, A... args) {
    kern<<<1, R, 0, s>>>(C, args...);
    FE_CHECK_LAUNCH();
  }

  // ||P f_c - K u_c|| / ||P f_c|| with an FP64 single-case product; if the
  // tolerance is not met and `reset`, r_c is replaced by that true residual.
  double true_relres(int c, double fn2, bool reset) {
    k_gather_case<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, R, c, u, w->tu.as<double>());
    FE_CHECK_LAUNCH();
    ebe_apply<double>(m, 1, w->tu.as<double>(), w->tq.as<double>(), s);
    double* out = w->d.as<double>() + D_RT2 * R + c;
    FE_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
    k_case_resid<<<(unsigned)std::min<int64_t>((N + 255) / 256, 1024), 256, 0, s>>>(
        N, R, c, m->nmask.as<uint8_t>(), f, w->tq.as<double>(), w->r.as<double>(), reset ? 1 : 0, out);
    FE_CHECK_LAUNCH();
    double rt2 = 0.0;
    FE_CUDA(cudaMemcpyAsync(&rt2, out, sizeof(double), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));
    return fn2 > 0.0 ? std::sqrt(rt2 / fn2) : 0.0;
  }
};

constexpr size_t kPersSums = 2 * 3 * 64 * sizeof(double);   // [2][3][R <= 64]
constexpr size_t kPersBytes = kPersSums + 64;               // + barrier count, generation, abort flag

void grid_wait_selftest(const fe_mesh* m, long long cycles, cudaStream_t s) {
  DevBuf words;
  words.alloc(64);   // barrier count, generation, abort flag
  FE_CUDA(cudaMemsetAsync(words.ptr, 0, 64, s));
  InnerArgs A{};
  A.bar = words.as<unsigned>();
  A.abort_flag = reinterpret_cast<int*>(words.as<unsigned char>() + 16);
  A.status = m->dev_status.as<int>();
  A.timeout = cycles;
  grid_wait_selftest_kernel<<<2, 32, 0, s>>>(A);
  FE_CHECK_LAUNCH();
  FE_CUDA(cudaStreamSynchronize(s));   // the words are freed on return
}

static SolverWork* get_work(fe_mesh* m, int R) {
  SolverWork* w = m->work;
  if (w && w->R == R) return w;
  free_solver_work(m);
  w = new SolverWork();
  m->work = w;
  const int64_t N = m->n_nodes;
  const size_t v = (size_t)N * R * 3;
  w->R = R;
  w->N = N;
  w->r.alloc(v * 8);
  w->p.alloc(v * 8);
  w->q.alloc(v * 8);
  w->rb.alloc(v * 4);
  w->ub.alloc(v * 4);
  w->eb.alloc(v * 4);
  w->pb.alloc(v * 4);
  w->qb.alloc(v * 4);
  w->tu.alloc((size_t)N * 3 * 8);
  w->tq.alloc((size_t)N * 3 * 8);
  w->d.alloc((size_t)D_COUNT * R * 8 + 64);
  w->i.alloc((size_t)I_COUNT * R * 4 + 64);
  w->pers.alloc(kPersBytes);
  FE_CUDA(cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking));
  FE_CUDA(cudaStreamCreateWithFlags(&w->body, cudaStreamNonBlocking));
  FE_CUDA(cudaEventCreateWithFlags(&w->ev, cudaEventDisableTiming));
  return w;
}

// One FP32 inner loop (Alg. 1(b)) on level `L`: e = rbar - Kbar ubar, then up to
// n steps of block-Jacobi CG until the max-over-cases stop rule holds. Steps after
// the stop are skipped on the device (the `done` flag), so the captured graph
// holds all n steps.
struct Level {
  int64_t N;
  const VGeom* g;
  const float* B;                 // FP32 inverse diagonal blocks [N][9]
  float *rb, *ub, *eb, *pb, *qb;  // [N][R][3]
  int level;                      // operator: TET10 (0), TET4 (1) or aggregation (2)
  int n;
  double eps;
  int f_rbn2, f_count;
};

static void level_apply(Solve& S, const Level& L, const float* x, float* y, const int* skip) {
  const Coarse& c = S.m->coarse;
  if (L.level == 2)
    bcsr_spmv(c.n_agg, S.R, c.rowptr2.as<int32_t>(), c.cols2.as<int32_t>(), c.vals2_32.as<float>(), x, y, S.s, skip);
  else if (L.level == 1 && S.assembled1)
    coarse_spmv(S.m, S.R, x, y, S.s, skip);
  else if (L.level == 1)
    ebe4_apply<float>(S.m, S.R, x, y, S.s, skip);
  else
    ebe_apply<float>(S.m, S.R, x, y, S.s, skip);
}

// one inner step (Algorithm 1(b)) and the stop test for the next one
static void inner_step(Solve& S, const Level& L, cudaGraphConditionalHandle loop, int use_loop) {
  S.vec_on(L.N, *L.g, k_inner_p, L.B, (const float*)L.eb, L.pb);
  level_apply(S, L, L.pb, L.qb, S.C.done);
  S.vec_on(L.N, *L.g, k_dot<float>, (int)D_GAMI, (const int*)S.C.done, (const float*)L.pb, (const float*)L.qb);
  S.scal(s_inner_alpha, L.f_rbn2, L.f_count);
  S.vec_on(L.N, *L.g, k_inner_update, L.B, L.eb, (const float*)L.qb, L.ub, (const float*)L.pb);
  S.scal(s_inner_check, L.n, L.eps, L.f_rbn2, loop, use_loop);
}

// the whole inner loop of an assembled level as one persistent cooperative kernel
// (k_inner_persistent); false when it does not apply (level 0, level 1 element by
// element, R not 4, 8, 16 or 32, or the caller asked for per-step launches)
static bool inner_loop_persistent(Solve& S, const Level& L) {
  const int R = S.R;
  if (S.o.inner_kernel != 0 || L.level == 0 || (L.level == 1 && !S.assembled1)) return false;
  if (R != 4 && R != 8 && R != 16 && R != 32) return false;
  const Coarse& c = S.m->coarse;
  InnerArgs A;
  A.N = L.N;
  A.C = S.C;
  A.B = L.B;
  A.rb = L.rb;
  A.ub = L.ub;
  A.eb = L.eb;
  A.pb = L.pb;
  A.qb = L.qb;
  A.sl_off = nullptr;
  A.sl_cols = nullptr;
  A.sl_vals = nullptr;
  if (L.level == 1) {
    A.rowptr = c.rowptr.as<int32_t>();
    A.cols = c.cols.as<int32_t>();
    A.vals = c.vals32.as<float>();
    if (c.sl_vals.ptr) {
      A.sl_off = c.sl_off.as<int32_t>();
      A.sl_cols = c.sl_cols.as<int32_t>();
      A.sl_vals = c.sl_vals.as<float>();
    }
  } else {
    A.rowptr = c.rowptr2.as<int32_t>();
    A.cols = c.cols2.as<int32_t>();
    A.vals = c.vals2_32.as<float>();
  }
  A.n_inner = L.n;
  A.eps = L.eps;
  A.f_rbn2 = L.f_rbn2;
  A.f_count = L.f_count;
  unsigned char* base = S.w->pers.as<unsigned char>();
  A.acc = reinterpret_cast<double*>(base);
  A.bar = reinterpret_cast<unsigned*>(base + kPersSums);
  A.abort_flag = reinterpret_cast<int*>(base + kPersSums + 8);
  A.status = S.m->dev_status.as<int>();
  A.timeout = 1LL << 31;   // about one second at 2 GHz
  const bool sliced = A.sl_vals != nullptr;
  const void* fn = sliced ? (const void*)k_inner_persistent<true> : (const void*)k_inner_persistent<false>;
  int per_sm = 0, sms = 0;
  FE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kInnerThreads, 0));
  FE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S.m->device));
  if (per_sm < 1) return false;
  const int64_t items = L.N * (R / 4);
  const int64_t need = (items + kInnerThreads - 1) / kInnerThreads;
  const int64_t cap = (int64_t)per_sm * sms;   // every CTA resident at once (a cooperative launch checks it)
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min(need, cap));
  FE_CUDA(cudaMemsetAsync(S.w->pers.ptr, 0, kPersBytes, S.s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kInnerThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = S.s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (sliced)
    FE_CUDA(cudaLaunchKernelEx(&cfg, k_inner_persistent<true>, A));
  else
    FE_CUDA(cudaLaunchKernelEx(&cfg, k_inner_persistent<false>, A));
  return true;
}

static void inner_loop(Solve& S, const Level& L) {
  if (inner_loop_persistent(S, L)) return;
  level_apply(S, L, L.ub, L.qb, nullptr);
  S.vec_on(L.N, *L.g, k_inner_resid, L.B, (const float*)L.rb, (const float*)L.qb, L.eb);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  FE_CUDA(cudaStreamIsCapturing(S.s, &cs));
  if (cs != cudaStreamCaptureStatusActive) {
    // direct launches: all n steps are issued; those after the stop return at once
    S.scal(s_inner_check, L.n, L.eps, L.f_rbn2, (cudaGraphConditionalHandle)0, 0);
    for (int step = 0; step < L.n; ++step) inner_step(S, L, (cudaGraphConditionalHandle)0, 0);
    return;
  }
  // recorded into a graph: a while node repeats one step while the stop test
  // says go (the body is recorded on a second stream into the node's own graph)
  cudaGraph_t graph = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t n_deps = 0;
  cudaGraphConditionalHandle loop;
  FE_CUDA(cudaStreamGetCaptureInfo(S.s, &cs, nullptr, &graph, &deps, &edges, &n_deps));
  FE_CUDA(cudaGraphConditionalHandleCreate(&loop, graph, 0, 0));
  S.scal(s_inner_check, L.n, L.eps, L.f_rbn2, loop, 1);
  FE_CUDA(cudaStreamGetCaptureInfo(S.s, &cs, nullptr, &graph, &deps, &edges, &n_deps));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = loop;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  FE_CUDA(cudaGraphAddNode(&node, graph, deps, edges, n_deps, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  const cudaStream_t outer = S.s;
  FE_CUDA(cudaStreamBeginCaptureToGraph(S.w->body, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  S.s = S.w->body;
  try {
    inner_step(S, L, loop, 1);
  } catch (...) {
    S.s = outer;
    cudaGraph_t g;
    cudaStreamEndCapture(S.w->body, &g);
    throw;
  }
  S.s = outer;
  FE_CUDA(cudaStreamEndCapture(S.w->body, &body));
  FE_CUDA(cudaStreamUpdateCaptureDependencies(S.s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
}

// the FCG outer iteration (Algorithm 1(a)): inner loop level 1 when the coarse
// level is on, with inner loop level 2 before it when the aggregation level is on
static void fcg_iteration(Solve& S) {
  SolverWork* w = S.w;
  fe_mesh* m = S.m;
  const float* B32 = m->binv32.as<float>();
  S.scal(s_outer_begin);
  S.vec(k_cast_start, B32, w->r.as<double>(), w->rb.as<float>(), w->ub.as<float>());
  if (S.N1 > 0) {
    Level L1{S.N1, &S.g1, m->coarse.binv32.as<float>(), w->rb1.as<float>(), w->ub1.as<float>(),
             w->eb1.as<float>(), w->pb1.as<float>(), w->qb1.as<float>(), 1, S.o.n_inner1, S.o.eps_inner1,
             (int)D_RBN21, (int)I_INNER1};
    coarse_restrict<float>(m, S.R, w->rb.as<float>(), L1.rb, S.s);
    coarse_restrict<float>(m, S.R, w->ub.as<float>(), L1.ub, S.s);
    S.vec_on(L1.N, *L1.g, k_dot<float>, (int)D_RBN21, (const int*)nullptr, (const float*)L1.rb,
             (const float*)L1.rb);
    if (S.N2 > 0) {
      Level L2{S.N2, &S.g2, m->coarse.binv2_32.as<float>(), w->rb2.as<float>(), w->ub2.as<float>(),
               w->eb2.as<float>(), w->pb2.as<float>(), w->qb2.as<float>(), 2, S.o.n_inner2, S.o.eps_inner2,
               (int)D_RBN22, (int)I_INNER2};
      level2_restrict(m, S.R, L1.rb, L2.rb, S.s);
      level2_restrict(m, S.R, L1.ub, L2.ub, S.s);
      S.vec_on(L2.N, *L2.g, k_dot<float>, (int)D_RBN22, (const int*)nullptr, (const float*)L2.rb,
               (const float*)L2.rb);
      inner_loop(S, L2);
      level2_prolong(m, S.R, (const float*)L2.ub, L1.ub, S.s);
      S.scal(s_level_begin);
    }
    inner_loop(S, L1);
    coarse_prolong<float>(m, S.R, (const float*)L1.ub, w->ub.as<float>(), S.s);
    S.scal(s_level_begin);
  }
  Level L0{S.N, &S.g, B32, w->rb.as<float>(), w->ub.as<float>(), w->eb.as<float>(), w->pb.as<float>(),
           w->qb.as<float>(), 0, S.o.n_inner, S.o.eps_inner, (int)D_RBN2, (int)I_INNER};
  inner_loop(S, L0);
  S.vec(k_outer_zq, (const float*)w->ub.as<float>(), (const double*)w->q.as<double>());
  S.scal(s_outer_beta, S.o.literal_beta);
  S.vec(k_outer_p, (const float*)w->ub.as<float>(), w->p.as<double>());
  ebe_apply<double>(m, S.R, w->p.as<double>(), w->q.as<double>(), S.s);
  S.vec(k_outer_dots, (const float*)w->ub.as<float>(), (const double*)w->r.as<double>(),
        (const double*)w->p.as<double>(), (const double*)w->q.as<double>());
  S.scal(s_outer_alpha);
  S.vec(k_outer_update, w->r.as<double>(), (const double*)w->q.as<double>(), S.u, (const double*)w->p.as<double>());
  S.scal(s_outer_check, S.o.tol, S.o.max_outer);
}

// one PCG iteration
static void pcg_iteration(Solve& S) {
  SolverWork* w = S.w;
  const double* B64 = S.m->binv64.as<double>();
  ebe_apply<double>(S.m, S.R, w->p.as<double>(), w->q.as<double>(), S.s);
  S.vec(k_dot<double>, (int)D_GAM, (const int*)nullptr, (const double*)w->p.as<double>(),
        (const double*)w->q.as<double>());
  S.scal(s_pcg_alpha);
  S.vec(k_pcg_update, B64, S.u, (const double*)w->p.as<double>(), w->r.as<double>(),
        (const double*)w->q.as<double>());
  S.scal(s_pcg_beta, S.o.tol, S.o.max_outer);
  S.vec(k_pcg_p, B64, (const double*)w->r.as<double>(), w->p.as<double>());
}

// Many-case mode: n_cases right-hand sides stream through R slots. f and u of
// run_solve are then the slot buffers; a slot whose case finished is stored to
// u_all and refilled with the next pending case between two iterations.
struct Many {
  int n_cases = 0;
  const double* f_all = nullptr;   // [n_cases][N][3]
  double* u_all = nullptr;         // [n_cases][N][3]
  fe_solve_stats* stats = nullptr; // [n_cases]
  int next = 0;
  std::vector<int> slot_case;      // [R], -1 = idle
};

static fe_status run_solve(fe_mesh* m, int R, const double* f, double* u, const fe_solve_opts& o,
                           fe_solve_stats* stats, cudaStream_t user, Many* many = nullptr) {
  SolverWork* w = get_work(m, R);
  cudaStream_t s = w->stream;
  // order after the caller's pending work on `user`
  FE_CUDA(cudaEventRecord(w->ev, user));
  FE_CUDA(cudaStreamWaitEvent(s, w->ev, 0));
  build_block_jacobi(m, s);
  int sms = 0;
  FE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
  Solve S;
  S.m = m;
  S.w = w;
  S.R = R;
  S.N = m->n_nodes;
  S.C = Cases{w->d.as<double>(), w->i.as<int>(), w->i.as<int>() + I_COUNT * R, R};
  DevBuf hist;   // CG coefficients of PCG64, when the caller asked for them
  if (o.solver == FE_SOLVER_PCG64 && o.cg_coef && o.cg_coef_len > 0 && !many) {
    hist.alloc((size_t)o.cg_coef_len * R * 2 * sizeof(double));
    FE_CUDA(cudaMemsetAsync(hist.ptr, 0, hist.bytes, s));
    S.C.hist = hist.as<double>();
    S.C.hist_len = o.cg_coef_len;
  }
  S.g = vgeom(S.N, R, sms);
  S.sm = (size_t)S.g.tpb * sizeof(double);
  S.s = s;
  S.f = f;
  S.u = u;
  S.o = o;
  const bool pcg = o.solver == FE_SOLVER_PCG64;
  if (o.solver == FE_SOLVER_FCG_MG || o.solver == FE_SOLVER_FCG_AMG) {
    const bool amg = o.solver == FE_SOLVER_FCG_AMG;
    build_coarse_jacobi(m, s);
    S.assembled1 = (amg || o.coarse_op != 2) && build_coarse_matrix(m, s, amg);
    FE_REQUIRE(!amg || S.assembled1, "level 2 needs the assembled coarse matrices: not enough free device memory");
    FE_REQUIRE(o.coarse_op != 1 || S.assembled1, "not enough free device memory for the assembled coarse matrix");
    if (!S.assembled1) build_coarse_geometry(m, s);
    if (amg) {
      S.N2 = m->coarse.n_agg;
      S.g2 = vgeom(S.N2, R, sms);
      const size_t v2 = (size_t)S.N2 * R * 3 * sizeof(float);
      for (DevBuf* b : {&w->rb2, &w->ub2, &w->eb2, &w->pb2, &w->qb2})
        if (b->bytes != v2) {
          b->release();
          b->alloc(v2);
        }
      FE_CUDA(cudaMemsetAsync(w->pb2.ptr, 0, v2, s));
    }
    S.N1 = m->coarse.n_nodes;
    S.g1 = vgeom(S.N1, R, sms);
    const size_t v1 = (size_t)S.N1 * R * 3 * sizeof(float);
    for (DevBuf* b : {&w->rb1, &w->ub1, &w->eb1, &w->pb1, &w->qb1})
      if (b->bytes != v1) {
        b->release();
        b->alloc(v1);
      }
    FE_CUDA(cudaMemsetAsync(w->pb1.ptr, 0, v1, s));
  }

  if (many) {
    // the first R cases into the slots (idle slots hold f = 0 and stay inactive)
    FE_CUDA(cudaMemsetAsync(const_cast<double*>(f), 0, (size_t)S.N * R * 3 * sizeof(double), s));
    many->slot_case.assign((size_t)R, -1);
    for (int r = 0; r < R && many->next < many->n_cases; ++r, ++many->next) {
      k_load_case<<<(unsigned)((S.N + 255) / 256), 256, 0, s>>>(S.N, R, r, many->f_all + (size_t)many->next * S.N * 3,
                                                               const_cast<double*>(f), u);
      FE_CHECK_LAUNCH();
      many->slot_case[(size_t)r] = many->next;
    }
  }
  // start: u = P u, r = P f - K u, ||f||, ||r|| (the product is skipped when u = 0)
  S.scal(s_init);
  S.vec(k_prepare, m->nmask.as<uint8_t>(), f, u);
  ebe_apply<double>(m, R, u, w->q.as<double>(), s, S.C.done + 2);
  S.vec(k_residual, m->nmask.as<uint8_t>(), f, (const double*)w->q.as<double>(), w->r.as<double>());
  S.scal(s_start, o.tol, 0);
  S.vec(k_zero_trivial, u);
  FE_CUDA(cudaMemsetAsync(w->q.ptr, 0, w->q.bytes, s));
  FE_CUDA(cudaMemsetAsync(w->p.ptr, 0, w->p.bytes, s));
  FE_CUDA(cudaMemsetAsync(w->pb.ptr, 0, w->pb.bytes, s));
  if (pcg) S.vec(k_pcg_init, m->binv64.as<double>(), (const double*)w->r.as<double>(), w->p.as<double>());

  // capture one iteration as a graph
  cudaGraphExec_t exec = nullptr;
  if (o.use_graph) {
    cudaGraph_t graph;
    FE_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
      if (pcg) pcg_iteration(S); else fcg_iteration(S);
    } catch (...) {
      cudaStreamEndCapture(s, &graph);
      throw;
    }
    FE_CUDA(cudaStreamEndCapture(s, &graph));
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    FE_CUDA(e);
  }

  std::vector<int> hi((size_t)I_COUNT * R);
  std::vector<double> hd((size_t)D_COUNT * R);
  const int check = o.check_every < 1 ? 1 : o.check_every;
  fe_status result = FE_OK;
  try {
    // the iteration loop: replay, then read the per-case flags every `check` iterations
    for (int64_t it = 0;; ++it) {
      FE_CUDA(cudaMemcpyAsync(hi.data(), w->i.ptr, hi.size() * 4, cudaMemcpyDeviceToHost, s));
      FE_CUDA(cudaMemcpyAsync(hd.data(), w->d.ptr, hd.size() * 8, cudaMemcpyDeviceToHost, s));
      FE_CUDA(cudaStreamSynchronize(s));
      // confirm candidates with the true FP64 residual: one all-case product when
      // a quarter or more of the cases are candidates, else one product per case
      bool any_active = false;
      int n_cand = 0;
      for (int c = 0; c < R; ++c) n_cand += hi[I_CAND * R + c] ? 1 : 0;
      const bool batched = R > 1 && 4 * n_cand >= R;
      if (batched) {
        if (!w->tall.ptr) w->tall.alloc((size_t)S.N * R * 3 * sizeof(double));
        ebe_apply<double>(m, R, u, w->tall.as<double>(), s);
        FE_CUDA(cudaMemsetAsync(w->d.as<double>() + D_RT2 * R, 0, R * sizeof(double), s));
        S.vec(k_cand_resid, m->nmask.as<uint8_t>(), f, (const double*)w->tall.as<double>(), w->r.as<double>());
        FE_CUDA(cudaMemcpyAsync(hd.data() + D_RT2 * R, w->d.as<double>() + D_RT2 * R, R * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
        FE_CUDA(cudaStreamSynchronize(s));
      }
      for (int c = 0; c < R; ++c) {
        if (hi[I_CAND * R + c]) {
          const double fn2 = hd[D_FN2 * R + c];
          const double rel = batched ? (fn2 > 0.0 ? std::sqrt(hd[D_RT2 * R + c] / fn2) : 0.0)
                                     : S.true_relres(c, fn2, true);
          int one = 1, zero = 0;
          FE_CUDA(cudaMemcpyAsync(w->i.as<int>() + I_CAND * R + c, &zero, 4, cudaMemcpyHostToDevice, s));
          if (rel <= o.tol) {
            FE_CUDA(cudaMemcpyAsync(w->d.as<double>() + D_RELRES * R + c, &rel, 8, cudaMemcpyHostToDevice, s));
          } else {
            // recursive residual drifted from the true one: continue from the true residual
            FE_CUDA(cudaMemcpyAsync(w->i.as<int>() + I_ACTIVE * R + c, &one, 4, cudaMemcpyHostToDevice, s));
            FE_CUDA(cudaMemcpyAsync(w->i.as<int>() + I_RESTART * R + c, &one, 4, cudaMemcpyHostToDevice, s));
            any_active = true;
          }
          FE_CUDA(cudaStreamSynchronize(s));
        }
        if (hi[I_ACTIVE * R + c]) any_active = true;
      }
      if (many) {
        // finished slots: store the case, refill with the next pending case
        FE_CUDA(cudaMemcpyAsync(hi.data(), w->i.ptr, hi.size() * 4, cudaMemcpyDeviceToHost, s));
        FE_CUDA(cudaMemcpyAsync(hd.data(), w->d.ptr, hd.size() * 8, cudaMemcpyDeviceToHost, s));
        FE_CUDA(cudaStreamSynchronize(s));
        for (int r = 0; r < R; ++r) {
          const int cs = many->slot_case[(size_t)r];
          if (cs < 0 || hi[I_ACTIVE * R + r] || hi[I_CAND * R + r]) continue;
          const int st = hi[I_STATUS * R + r];
          double rel = hd[D_RELRES * R + r];
          if (st != FE_OK) rel = S.true_relres(r, hd[D_FN2 * R + r], false);
          k_store_case<<<(unsigned)((S.N + 255) / 256), 256, 0, s>>>(S.N, R, r, u, many->u_all + (size_t)cs * S.N * 3);
          FE_CHECK_LAUNCH();
          if (many->stats) {
            many->stats[cs].outer_iters = hi[I_OUTER * R + r];
            many->stats[cs].inner_iters = hi[I_INNER * R + r];
            many->stats[cs].relres = rel;
            many->stats[cs].status = st;
            many->stats[cs].inner1_iters = hi[I_INNER1 * R + r];
            many->stats[cs].inner2_iters = hi[I_INNER2 * R + r];
            many->stats[cs].pad = 0;
          }
          if (st == FE_EBREAKDOWN) result = FE_EBREAKDOWN;
          else if (st == FE_ENOCONV && result == FE_OK) result = FE_ENOCONV;
          many->slot_case[(size_t)r] = -1;
          if (many->next < many->n_cases) {
            const int nc = many->next++;
            k_load_case<<<(unsigned)((S.N + 255) / 256), 256, 0, s>>>(S.N, R, r, many->f_all + (size_t)nc * S.N * 3,
                                                                     const_cast<double*>(f), u);
            FE_CHECK_LAUNCH();
            FE_CUDA(cudaMemsetAsync(w->d.as<double>() + D_FN2 * R + r, 0, 8, s));
            FE_CUDA(cudaMemsetAsync(w->d.as<double>() + D_RN2 * R + r, 0, 8, s));
            k_slot_init<<<(unsigned)std::min<int64_t>((S.N + 255) / 256, 1024), 256, 0, s>>>(
                S.N, R, r, m->nmask.as<uint8_t>(), f, w->r.as<double>(), w->d.as<double>() + D_FN2 * R + r,
                w->d.as<double>() + D_RN2 * R + r);
            FE_CHECK_LAUNCH();
            s_slot_start<<<1, 1, 0, s>>>(S.C, r, pcg ? 1 : 0);
            FE_CHECK_LAUNCH();
            many->slot_case[(size_t)r] = nc;
            any_active = true;
          }
        }
      }
      if (pcg) {
        // cases whose recursive residual drifted (or freshly loaded slots) restart CG from r
        FE_CUDA(cudaMemsetAsync(w->d.as<double>() + D_RHOA * R, 0, R * 8, s));
        S.vec(k_pcg_restart, m->binv64.as<double>(), (const double*)w->r.as<double>(), w->p.as<double>());
        S.scal(s_pcg_restart);
      }
      if (!any_active) break;
      for (int k = 0; k < check; ++k) {
        if (exec) {
          FE_CUDA(cudaGraphLaunch(exec, s));
        } else if (pcg) {
          pcg_iteration(S);
        } else {
          fcg_iteration(S);
        }
      }
    }
    FE_CUDA(cudaMemcpyAsync(hi.data(), w->i.ptr, hi.size() * 4, cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaMemcpyAsync(hd.data(), w->d.ptr, hd.size() * 8, cudaMemcpyDeviceToHost, s));
    if (hist.ptr) FE_CUDA(cudaMemcpyAsync(o.cg_coef, hist.ptr, hist.bytes, cudaMemcpyDeviceToHost, s));
    int32_t dev_status = 0;   // a bounded device-side wait of an EBE kernel gave up during the solve
    FE_CUDA(cudaMemcpyAsync(&dev_status, m->dev_status.ptr, sizeof(dev_status), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));
    if (dev_status != 0) {
      FE_CUDA(cudaMemsetAsync(m->dev_status.ptr, 0, sizeof(int32_t), s));
      set_error("fe_pcg_solve: a device-side wait of the EBE kernel gave up; the solution is invalid");
      throw Failure{FE_ETIMEOUT};
    }
    for (int c = 0; c < R && !many; ++c) {
      int st = hi[I_STATUS * R + c];
      double rel = hd[D_RELRES * R + c];
      if (st != FE_OK) rel = S.true_relres(c, hd[D_FN2 * R + c], false);
      if (stats) {
        stats[c].outer_iters = hi[I_OUTER * R + c];
        stats[c].inner_iters = hi[I_INNER * R + c];
        stats[c].relres = rel;
        stats[c].status = st;
        stats[c].inner1_iters = hi[I_INNER1 * R + c];
        stats[c].inner2_iters = hi[I_INNER2 * R + c];
        stats[c].pad = 0;
      }
      if (st == FE_EBREAKDOWN) result = FE_EBREAKDOWN;
      else if (st == FE_ENOCONV && result == FE_OK) result = FE_ENOCONV;
    }
  } catch (...) {
    if (exec) cudaGraphExecDestroy(exec);
    throw;
  }
  if (exec) cudaGraphExecDestroy(exec);
  // the caller's stream continues after the solve
  FE_CUDA(cudaEventRecord(w->ev, s));
  FE_CUDA(cudaStreamWaitEvent(user, w->ev, 0));
  if (result != FE_OK) set_error("fe_pcg_solve: %s", result == FE_EBREAKDOWN ? "breakdown in at least one case"
                                                                            : "iteration cap reached in at least one case");
  return result;
}

static void check_opts(const fe_solve_opts& o) {
  FE_REQUIRE(o.solver >= FE_SOLVER_PCG64 && o.solver <= FE_SOLVER_FCG_AMG, "unknown solver %d", o.solver);
  FE_REQUIRE(o.tol > 0.0 && o.tol < 1.0, "tol must lie in (0, 1)");
  FE_REQUIRE(o.max_outer >= 1, "max_outer must be >= 1");
  FE_REQUIRE(o.n_inner >= 0 && o.n_inner <= 100000, "n_inner out of range");
  FE_REQUIRE(o.eps_inner >= 0.0, "eps_inner must be >= 0");
  if (o.solver == FE_SOLVER_FCG_AMG) {
    FE_REQUIRE(o.n_inner2 >= 0 && o.n_inner2 <= 100000, "n_inner2 out of range");
    FE_REQUIRE(o.eps_inner2 >= 0.0, "eps_inner2 must be >= 0");
  }
  if (o.solver == FE_SOLVER_FCG_MG || o.solver == FE_SOLVER_FCG_AMG) {
    FE_REQUIRE(o.n_inner1 >= 0 && o.n_inner1 <= 100000, "n_inner1 out of range");
    FE_REQUIRE(o.eps_inner1 >= 0.0, "eps_inner1 must be >= 0");
    FE_REQUIRE(o.coarse_op >= 0 && o.coarse_op <= 2, "coarse_op must be 0, 1 or 2");
  }
  FE_REQUIRE(o.cg_coef_len >= 0 && o.cg_coef_len <= (1 << 24) && (o.cg_coef_len == 0 || o.cg_coef != nullptr),
             "cg_coef_len must lie in [0, 2^24], with cg_coef set when it is positive");
  FE_REQUIRE(o.inner_kernel == 0 || o.inner_kernel == 1, "inner_kernel must be 0 or 1");
}

}  // namespace fe

extern "C" fe_status fe_pcg_solve(const fe_mesh* mesh, int32_t R, const double* f, double* u,
                                  const fe_solve_opts* opts, fe_solve_stats* stats, void* stream) {
  try {
    fe::clear_error();
    FE_REQUIRE(mesh != nullptr, "mesh is NULL");
    FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range [1, 64]", R);
    FE_REQUIRE(f != nullptr && u != nullptr, "NULL vector");
    fe_solve_opts o;
    fe_solve_opts_default(&o);
    if (opts) o = *opts;
    fe::check_opts(o);
    fe_mesh* m = const_cast<fe_mesh*>(mesh);
    fe::DeviceGuard dg(m->device);
    return fe::run_solve(m, R, f, u, o, stats, (cudaStream_t)stream);
  } catch (const fe::Failure& x) {
    return x.status;
  } catch (...) {
    fe::set_error("unexpected C++ exception");
    return FE_EINVAL;
  }
}

namespace fe {

// free device memory -> slot count (largest of 32, 16, 8, 4, 2, 1 that fits with a margin)
static int choose_slots(const fe_mesh* m, int n_cases) {
  size_t free_b = 0, total_b = 0;
  FE_CUDA(cudaMemGetInfo(&free_b, &total_b));
  // per slot: FP64 F, U, r, p, q and the all-case true-residual product, FP32
  // rbar, ubar, e, pbar, qbar vectors of [N][3] (the coarse levels' vectors are
  // a tenth of that and the float-float geometry E x 128 B, inside the margin)
  const double per_slot = (double)m->n_nodes * 3 * (6 * 8 + 5 * 4);
  const double budget = 0.7 * (double)free_b;
  int R = 32;
  while (R > 1 && (R > n_cases || R * per_slot > budget)) R /= 2;
  return R;
}

// kernels for the products a solve with R slots runs, tuned on first use
static void tune_if_unset(fe_mesh* m, int R, cudaStream_t s) {
  int32_t v = 0, us = 0;
  const int todo[3][2] = {{R, FE_F32}, {R, FE_F64}, {1, FE_F64}};
  for (const auto& t : todo) {
    if (m->variant[t[1] == FE_F32 ? 1 : 0][t[0]] >= 0) continue;
    const fe_status st = fe_ebe_tune(m, t[0], (fe_dtype)t[1], s, &v, &us);
    if (st != FE_OK) throw Failure{st};
  }
}

}  // namespace fe

extern "C" fe_status fe_solve_many(const fe_mesh* mesh, int32_t n_cases, const double* f_dev, double* u_dev,
                                   int32_t R_slots, const fe_solve_opts* opts, fe_solve_stats* stats, int32_t* R_used,
                                   void* stream) {
  try {
    fe::clear_error();
    FE_REQUIRE(mesh != nullptr, "mesh is NULL");
    FE_REQUIRE(n_cases >= 1, "n_cases must be >= 1");
    FE_REQUIRE(f_dev != nullptr && u_dev != nullptr, "NULL vector");
    FE_REQUIRE(R_slots >= 0 && R_slots <= 64, "R_slots = %d out of range [0, 64]", R_slots);
    fe_solve_opts o;
    fe_solve_opts_default(&o);
    if (opts) o = *opts;
    fe::check_opts(o);
    fe_mesh* m = const_cast<fe_mesh*>(mesh);
    fe::DeviceGuard dg(m->device);
    const int R = R_slots > 0 ? (R_slots < n_cases ? R_slots : n_cases) : fe::choose_slots(m, n_cases);
    if (R_used) *R_used = R;
    fe::tune_if_unset(m, R, (cudaStream_t)stream);
    fe::DevBuf F, U;
    F.alloc((size_t)m->n_nodes * R * 3 * sizeof(double));
    U.alloc((size_t)m->n_nodes * R * 3 * sizeof(double));
    fe::Many many;
    many.n_cases = n_cases;
    many.f_all = f_dev;
    many.u_all = u_dev;
    many.stats = stats;
    const fe_status st = fe::run_solve(m, R, F.as<double>(), U.as<double>(), o, nullptr, (cudaStream_t)stream, &many);
    FE_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return st;
  } catch (const fe::Failure& x) {
    return x.status;
  } catch (...) {
    fe::set_error("unexpected C++ exception");
    return FE_EINVAL;
  }
}

extern "C" fe_status fe_block_jacobi(const fe_mesh* mesh, double* binv_dev, void* stream) {
  try {
    fe::clear_error();
    FE_REQUIRE(mesh != nullptr && binv_dev != nullptr, "NULL argument");
    fe_mesh* m = const_cast<fe_mesh*>(mesh);
    fe::DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    fe::build_block_jacobi(m, s);
    FE_CUDA(cudaMemcpyAsync(binv_dev, m->binv64.ptr, m->binv64.bytes, cudaMemcpyDeviceToDevice, s));
    return FE_OK;
  } catch (const fe::Failure& x) {
    return x.status;
  } catch (...) {
    fe::set_error("unexpected C++ exception");
    return FE_EINVAL;
  }
}

// ---------------------------------------------------------------------------
// Allocation-free build of the block-Jacobi preconditioner.
//
// Some callers cannot allocate device memory at the point where they need the
// preconditioner: latency-critical loops that must not take the allocator's lock,
// and processes whose device memory is already reserved by another allocator's
// pool (a framework's caching allocator), where a fresh cudaMalloc can fail
// mid-run. For them fe_block_jacobi_noalloc keeps its scratch (the FP64 [N][9]
// accumulator of diagonal blocks, the FP32 copy of the inverse the shared kernel
// also writes, and an error flag) in the fixed file-scope array below instead of
// allocating it. Every GPU that loads this library holds the array until the
// process exits. The call synchronises its stream (it reads the error flag back).
// ---------------------------------------------------------------------------
namespace fe {

constexpr int64_t kNoAllocMaxNodes = 131072;                       // largest mesh served
constexpr size_t kNoAllocD = (size_t)kNoAllocMaxNodes * 9 * sizeof(double);   // offset of FP32 blocks
constexpr size_t kNoAllocFlag = kNoAllocD + (size_t)kNoAllocMaxNodes * 9 * sizeof(float);
constexpr size_t kNoAllocBytes = kNoAllocFlag + 256;               // about 13.5 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device ordinal, looked up once per
// device (the host-side name of the array is only a stand-in, not a device address)
// and kept for the life of the process; it does not survive a reset of the
// device's primary context.
static void* g_noalloc_addr[256];
static std::mutex g_noalloc_mutex;

static void* noalloc_scratch(int device) {
  FE_REQUIRE(device >= 0 && device < 256, "device ordinal %d out of range", device);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    FE_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));   // the device is current (DeviceGuard)
    g_noalloc_addr[device] = p;
  }
  return g_noalloc_addr[device];
}

}  // namespace fe

extern "C" fe_status fe_block_jacobi_noalloc(const fe_mesh* mesh, double* binv_dev, void* stream) {
  try {
    fe::clear_error();
    FE_REQUIRE(mesh != nullptr && binv_dev != nullptr, "NULL argument");
    FE_REQUIRE(mesh->n_nodes <= fe::kNoAllocMaxNodes,
               "fe_block_jacobi_noalloc serves meshes of at most %lld nodes (this mesh has %lld); "
               "use fe_block_jacobi", (long long)fe::kNoAllocMaxNodes, (long long)mesh->n_nodes);
    fe::DeviceGuard dg(mesh->device);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = static_cast<unsigned char*>(fe::noalloc_scratch(mesh->device));
    double* D = reinterpret_cast<double*>(base);
    float* B32 = reinterpret_cast<float*>(base + fe::kNoAllocD);
    int* bad = reinterpret_cast<int*>(base + fe::kNoAllocFlag);
    const int64_t N = mesh->n_nodes, E = mesh->n_elem;
    // the array keeps the previous call's contents: clear the accumulator and the flag
    FE_CUDA(cudaMemsetAsync(D, 0, (size_t)N * 9 * sizeof(double), s));
    FE_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    fe::jacobi_diag_kernel<<<(unsigned)((E + 127) / 128), 128, 0, s>>>(mesh->view<double>(), D);
    FE_CHECK_LAUNCH();
    fe::jacobi_invert_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, mesh->nmask.as<uint8_t>(), D, binv_dev,
                                                                         B32, bad);
    FE_CHECK_LAUNCH();
    int hbad = 0;
    FE_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));
    FE_REQUIRE(hbad == 0, "block Jacobi: a free node has a singular or indefinite diagonal block "
                          "(node touched by no element, or a degenerate material)");
    return FE_OK;
  } catch (const fe::Failure& x) {
    return x.status;
  } catch (...) {
    fe::set_error("unexpected C++ exception");
    return FE_EINVAL;
  }
}
