// Adjoint element sensitivity g_e = -sum_r (P lambda_r)_e^T K_e (P u_r)_e.
//
// With m_e = log E_e and Poisson ratio fixed, K_e is proportional to E_e, so
// dK_bc/dm_e = P Q_e K_e Q_e^T P and dJ/dm_e = -lambda^T (dK_bc/dm_e) u for the
// adjoint state lambda = K_bc^-1 dJ/du. The element product is the EBE
// arithmetic of Eq. 3, reduced against lambda_e instead of scattered. The paper
// has no adjoint; this kernel is an addition of this library.
#include "fe_element.cuh"
#include "fe_internal.cuh"

namespace fe {

namespace {

constexpr int kThreads = 128;

__global__ void __launch_bounds__(kThreads) adjoint_kernel(MeshView<double> M, int R, const int64_t* __restrict__ perm,
                                                           const double* __restrict__ u,
                                                           const double* __restrict__ lam, double* __restrict__ g) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= M.n_elem) return;
  int nd[10];
  const int2* c2 = reinterpret_cast<const int2*>(M.conn + 10 * e);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int2 v = __ldg(c2 + q);
    nd[2 * q] = v.x;
    nd[2 * q + 1] = v.y;
  }
  double xc[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) xc[k][i] = __ldg(M.xyz + 3 * (int64_t)nd[k] + i);
  ElemGeo<double> G;
  elem_geometry(xc[0], xc[1], xc[2], xc[3], __ldg(M.mat + 2 * e), __ldg(M.mat + 2 * e + 1), G);
  int mk[10];
#pragma unroll
  for (int a = 0; a < 10; ++a) mk[a] = __ldg(M.nmask + nd[a]);
  double acc = 0.0;
  for (int r = 0; r < R; ++r) {
    double ue[10][3], le[10][3];
#pragma unroll
    for (int a = 0; a < 10; ++a) {
      const int64_t b = ((int64_t)nd[a] * R + r) * 3;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const bool f = (mk[a] >> c) & 1;
        ue[a][c] = f ? __ldg(u + b + c) : 0.0;
        le[a][c] = f ? __ldg(lam + b + c) : 0.0;
      }
    }
    acc += elem_bilinear(G, le, ue);
  }
  g[perm[e]] = -acc;
}

}  // namespace

void adjoint_grad(const fe_mesh* m, int R, const double* u, const double* lam, double* g, cudaStream_t s) {
  const MeshView<double> M = m->view<double>();
  const int64_t blocks = (M.n_elem + kThreads - 1) / kThreads;
  adjoint_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(M, R, m->perm.as<int64_t>(), u, lam, g);
  FE_CHECK_LAUNCH();
}

}  // namespace fe

extern "C" fe_status fe_adjoint_grad(const fe_mesh* m, int32_t R, const double* u, const double* lam, double* g,
                                     void* stream) {
  try {
    fe::clear_error();
    FE_REQUIRE(m != nullptr, "mesh is NULL");
    FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range [1, 64]", R);
    FE_REQUIRE(u && lam && g, "NULL vector");
    fe::DeviceGuard dg(m->device);
    fe::adjoint_grad(m, R, u, lam, g, (cudaStream_t)stream);
    return FE_OK;
  } catch (const fe::Failure& f) {
    return f.status;
  } catch (...) {
    fe::set_error("unexpected C++ exception");
    return FE_EINVAL;
  }
}
