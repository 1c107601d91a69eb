// Adjoint element sensitivity g_e = -sum_r (P lambda_r)_e^T K_e (P u_r)_e.
//
// With m_e = log E_e and Poisson ratio fixed, K_e is proportional to E_e, so
// dK_bc/dm_e = P Q_e K_e Q_e^T P and dJ/dm_e = -lambda^T (dK_bc/dm_e) u for the
// adjoint state lambda = K_bc^-1 dJ/du. The element product is the EBE
// arithmetic of Eq. 3, reduced against lambda_e instead of scattered. The paper
// has no adjoint; this kernel is an addition of this library.
#include <cmath>

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

// ---------------------------------------------------------------------------
// Observation operator and the vector steps of the gradient (no counterpart in
// the paper; they complete the adjoint workflow around fe_adjoint_grad).
//   u_obs[p][r][c] = sum_j w[p][j] u[node[p][j]][r][c]             (fe_obs_apply)
//   out = P (Obs^T g): out[n][r][c] = sum_{(p,j): node[p][j] = n} w[p][j] g[p][r][c]
//         on free DOFs, 0 on constrained ones                        (fe_obs_adjoint)
//   u[n][c] = sum_r a_r G[n][r][c]                                   (fe_combine_cases)
//   out_r = sum_{n, c free} f[n][r][c] lam[n][c]                     (fe_case_dots)
// ---------------------------------------------------------------------------
struct fe_obs {
  int device = 0;
  int64_t n_obs = 0, n_nodes = 0;
  int32_t n_per = 0;
  fe::DevBuf node;    // int32 [P][J]
  fe::DevBuf weight;  // double [P][J]
};

namespace fe {

namespace {

__global__ void obs_apply_kernel(int64_t P, int J, int R, const int32_t* __restrict__ node,
                                 const double* __restrict__ w, const double* __restrict__ u, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)R * 3;
  if (i >= P * per) return;
  const int64_t p = i / per;
  const int64_t rc = i - p * per;
  double acc = 0.0;
  for (int j = 0; j < J; ++j) acc += w[p * J + j] * u[(int64_t)node[p * J + j] * per + rc];
  out[i] = acc;
}

__global__ void obs_adjoint_kernel(int64_t P, int J, int R, const int32_t* __restrict__ node,
                                   const double* __restrict__ w, const uint8_t* __restrict__ nmask,
                                   const double* __restrict__ g, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)R * 3;
  if (i >= P * J * per) return;
  const int64_t pj = i / per;
  const int64_t rc = i - pj * per;
  const int64_t p = pj / J;
  const int32_t n = node[pj];
  if (!((nmask[n] >> (int)(rc % 3)) & 1)) return;   // constrained DOF: P keeps it at zero
  atomicAdd(out + (int64_t)n * per + rc, w[pj] * g[p * per + rc]);
}

__global__ void combine_kernel(int64_t N, int R, const double* __restrict__ G, const double* __restrict__ a,
                               double* __restrict__ u) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N * 3) return;
  const int64_t n = i / 3;
  const int c = (int)(i - n * 3);
  double acc = 0.0;
  for (int r = 0; r < R; ++r) acc += a[r] * G[(n * R + r) * 3 + c];
  u[i] = acc;
}

// one partial sum per (block, case) in shared memory, then one atomic add per (block, case)
__global__ void case_dots_kernel(int64_t N, int R, const uint8_t* __restrict__ nmask, const double* __restrict__ f,
                                 const double* __restrict__ lam, double* __restrict__ out) {
  __shared__ double part[64];
  for (int r = threadIdx.x; r < R; r += blockDim.x) part[r] = 0.0;
  __syncthreads();
  const int64_t total = N * R;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = i / R;
    const int r = (int)(i - n * R);
    const int mk = nmask[n];
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if ((mk >> c) & 1) v += f[i * 3 + c] * lam[n * 3 + c];
    atomicAdd(&part[r], v);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) atomicAdd(out + r, part[r]);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

}  // namespace fe

extern "C" fe_status fe_obs_create(const fe_mesh* m, int64_t n_obs, int32_t n_per, const int32_t* node,
                                   const double* weight, fe_obs** out) {
  if (out) *out = nullptr;
  fe_obs* o = nullptr;
  const fe_status st = fe::guarded([&] {
    FE_REQUIRE(m != nullptr && out != nullptr, "NULL argument");
    FE_REQUIRE(n_obs >= 1 && n_obs < ((int64_t)1 << 31), "n_obs = %lld out of range", (long long)n_obs);
    FE_REQUIRE(n_per >= 1 && n_per <= 64, "n_per = %d out of range [1, 64]", n_per);
    FE_REQUIRE(node != nullptr && weight != nullptr, "NULL node or weight array");
    for (int64_t i = 0; i < n_obs * n_per; ++i) {
      FE_REQUIRE(node[i] >= 0 && node[i] < m->n_nodes, "observation %lld: node id %d out of range",
                 (long long)(i / n_per), node[i]);
      FE_REQUIRE(std::isfinite(weight[i]), "observation %lld: weight is not finite", (long long)(i / n_per));
    }
    fe::DeviceGuard dg(m->device);
    o = new fe_obs();
    o->device = m->device;
    o->n_obs = n_obs;
    o->n_per = n_per;
    o->n_nodes = m->n_nodes;
    o->node.alloc((size_t)(n_obs * n_per) * sizeof(int32_t));
    o->weight.alloc((size_t)(n_obs * n_per) * sizeof(double));
    FE_CUDA(cudaMemcpy(o->node.ptr, node, o->node.bytes, cudaMemcpyHostToDevice));
    FE_CUDA(cudaMemcpy(o->weight.ptr, weight, o->weight.bytes, cudaMemcpyHostToDevice));
    *out = o;
  });
  if (st != FE_OK) {
    delete o;
    if (out) *out = nullptr;
  }
  return st;
}

extern "C" void fe_obs_destroy(fe_obs* o) {
  if (!o) return;
  try {
    fe::DeviceGuard dg(o->device);
    delete o;
  } catch (...) {
  }
}

extern "C" fe_status fe_obs_apply(const fe_obs* o, int32_t R, const double* u, double* u_obs, void* stream) {
  return fe::guarded([&] {
    FE_REQUIRE(o != nullptr && u != nullptr && u_obs != nullptr, "NULL argument");
    FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range [1, 64]", R);
    fe::DeviceGuard dg(o->device);
    const int64_t n = o->n_obs * R * 3;
    fe::obs_apply_kernel<<<fe::blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(
        o->n_obs, o->n_per, R, o->node.as<int32_t>(), o->weight.as<double>(), u, u_obs);
    FE_CHECK_LAUNCH();
  });
}

extern "C" fe_status fe_obs_adjoint(const fe_mesh* m, const fe_obs* o, int32_t R, const double* g, double* out,
                                    void* stream) {
  return fe::guarded([&] {
    FE_REQUIRE(m != nullptr && o != nullptr && g != nullptr && out != nullptr, "NULL argument");
    FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range [1, 64]", R);
    FE_REQUIRE(o->n_nodes == m->n_nodes && o->device == m->device, "observation operator built for another mesh");
    FE_REQUIRE((const void*)g != (const void*)out, "g and out must not alias");
    fe::DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    FE_CUDA(cudaMemsetAsync(out, 0, (size_t)m->n_nodes * R * 3 * sizeof(double), s));
    const int64_t n = o->n_obs * o->n_per * R * 3;
    fe::obs_adjoint_kernel<<<fe::blocks_for(n, 256), 256, 0, s>>>(o->n_obs, o->n_per, R, o->node.as<int32_t>(),
                                                                   o->weight.as<double>(), m->nmask.as<uint8_t>(),
                                                                   g, out);
    FE_CHECK_LAUNCH();
  });
}

extern "C" fe_status fe_combine_cases(const fe_mesh* m, int32_t R, const double* G, const double* a, double* u,
                                      void* stream) {
  return fe::guarded([&] {
    FE_REQUIRE(m != nullptr && G != nullptr && a != nullptr && u != nullptr, "NULL argument");
    FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range [1, 64]", R);
    fe::DeviceGuard dg(m->device);
    const int64_t n = m->n_nodes * 3;
    fe::combine_kernel<<<fe::blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(m->n_nodes, R, G, a, u);
    FE_CHECK_LAUNCH();
  });
}

extern "C" fe_status fe_case_dots(const fe_mesh* m, int32_t R, const double* f, const double* lam, double* out,
                                  void* stream) {
  return fe::guarded([&] {
    FE_REQUIRE(m != nullptr && f != nullptr && lam != nullptr && out != nullptr, "NULL argument");
    FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range [1, 64]", R);
    fe::DeviceGuard dg(m->device);
    cudaStream_t s = (cudaStream_t)stream;
    FE_CUDA(cudaMemsetAsync(out, 0, (size_t)R * sizeof(double), s));
    int sms = 0;
    FE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    fe::case_dots_kernel<<<(unsigned)(2 * sms), 256, 0, s>>>(m->n_nodes, R, m->nmask.as<uint8_t>(), f, lam, out);
    FE_CHECK_LAUNCH();
  });
}
