// Inner loop level 2 of Algorithm 1(a): an algebraic coarsening of the TET4 level
// (Sec. 2: the first-order grid coarsened by algebraic multigrid so that the
// low-frequency part of the solution is resolved by a CG on far fewer DOFs).
//
//  * aggregation of the coarse nodes over the graph of K1's block pattern, two
//    passes in node order: a node with no aggregated neighbour starts an
//    aggregate of itself and all its neighbours; every node left over joins the
//    first-pass aggregate of its lowest-numbered neighbour that has one;
//  * P2 copies an aggregate's value to its members' free DOFs (one translation
//    per component), P2^T sums the members' free values;
//  * A2 = P2^T K1_bc P2 on the aggregate DOFs with a free member, identity on the
//    others, assembled from the FP64 K1 blocks, stored in FP32 block CSR and
//    applied with the same multi-vector block SpMV as K1; its block Jacobi is
//    inverted in FP64.
// The aggregation and A2's pattern depend only on the mesh and are built once
// on the host; A2's values are rebuilt with K1 when the materials change.
#include <algorithm>
#include <vector>

#include "fe_internal.cuh"

namespace fe {

namespace {

constexpr int kThreads = 256;

unsigned blocks_for(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + kThreads - 1) / kThreads); }

// A2 += masked K1 blocks: thread = K1 block row a
__global__ void galerkin2_kernel(int64_t N4, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ cols,
                                 const uint8_t* __restrict__ nmask4, const int32_t* __restrict__ pos2,
                                 const double* __restrict__ k1, double* __restrict__ a2) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= N4) return;
  const int ma = nmask4[a];
  for (int q = rowptr[a]; q < rowptr[a + 1]; ++q) {
    const int mb = nmask4[cols[q]];
    const double* src = k1 + 9 * (int64_t)q;
    double* dst = a2 + 9 * (int64_t)pos2[q];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        if (((ma >> i) & 1) && ((mb >> j) & 1)) atomicAdd(dst + 3 * i + j, src[3 * i + j]);
  }
}

// per aggregate: unit diagonal on DOFs without a free member, FP32 copy of the
// row, inverse of the diagonal block (FP64 and FP32)
__global__ void finish2_kernel(int64_t NA, const int32_t* __restrict__ rowptr2, const int32_t* __restrict__ cols2,
                               const uint8_t* __restrict__ nmask2, double* __restrict__ a2, float* __restrict__ a2f,
                               double* __restrict__ B64, float* __restrict__ B32, int* __restrict__ bad) {
  const int64_t A = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (A >= NA) return;
  const int mk = nmask2[A];
  int diag = -1;
  for (int q = rowptr2[A]; q < rowptr2[A + 1]; ++q) {
    if (cols2[q] == A) {
      diag = q;
      for (int i = 0; i < 3; ++i)
        if (!((mk >> i) & 1)) a2[9 * (int64_t)q + 4 * i] = 1.0;
    }
    for (int k = 0; k < 9; ++k) a2f[9 * (int64_t)q + k] = (float)a2[9 * (int64_t)q + k];
  }
  if (diag < 0) {
    atomicExch(bad, 1);
    return;
  }
  const double* M = a2 + 9 * (int64_t)diag;
  const double c00 = M[4] * M[8] - M[5] * M[7], c01 = M[5] * M[6] - M[3] * M[8], c02 = M[3] * M[7] - M[4] * M[6];
  const double det = M[0] * c00 + M[1] * c01 + M[2] * c02;
  if (!(det > 0.0) || !isfinite(det)) {
    atomicExch(bad, 1);
    return;
  }
  const double id = 1.0 / det;
  const double I[9] = {c00 * id, (M[2] * M[7] - M[1] * M[8]) * id, (M[1] * M[5] - M[2] * M[4]) * id,
                       c01 * id, (M[0] * M[8] - M[2] * M[6]) * id, (M[2] * M[3] - M[0] * M[5]) * id,
                       c02 * id, (M[1] * M[6] - M[0] * M[7]) * id, (M[0] * M[4] - M[1] * M[3]) * id};
  for (int k = 0; k < 9; ++k) {
    B64[9 * A + k] = I[k];
    B32[9 * A + k] = (float)I[k];
  }
}

// r2 = P2^T r4: thread = (aggregate, case), members' free values summed
__global__ void __launch_bounds__(kThreads) restrict2_kernel(int64_t NA, int R, const int32_t* __restrict__ mptr,
                                                             const int32_t* __restrict__ members,
                                                             const uint8_t* __restrict__ nmask4,
                                                             const float* __restrict__ r4, float* __restrict__ r2,
                                                             const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= NA * R) return;
  const int64_t A = gid / R;
  const int r = (int)(gid - A * R);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  const int k1 = __ldg(mptr + A + 1);
  for (int k = __ldg(mptr + A); k < k1; ++k) {
    const int64_t a = __ldg(members + k);
    const int mk = __ldg(nmask4 + a);
    const float* v = r4 + (a * R + r) * 3;
    if (mk & 1) s0 += __ldg(v);
    if (mk & 2) s1 += __ldg(v + 1);
    if (mk & 4) s2 += __ldg(v + 2);
  }
  float* o = r2 + gid * 3;
  o[0] = s0;
  o[1] = s1;
  o[2] = s2;
}

// u4 = P2 u2: thread = (coarse node, case)
__global__ void __launch_bounds__(kThreads) prolong2_kernel(int64_t N4, int R, const int32_t* __restrict__ agg,
                                                            const uint8_t* __restrict__ nmask4,
                                                            const float* __restrict__ u2, float* __restrict__ u4,
                                                            const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= N4 * R) return;
  const int64_t a = gid / R;
  const int r = (int)(gid - a * R);
  const int mk = __ldg(nmask4 + a);
  const float* v = u2 + ((int64_t)__ldg(agg + a) * R + r) * 3;
  float* o = u4 + gid * 3;
  o[0] = (mk & 1) ? __ldg(v) : 0.f;
  o[1] = (mk & 2) ? __ldg(v + 1) : 0.f;
  o[2] = (mk & 4) ? __ldg(v + 2) : 0.f;
}

// aggregation and A2 pattern (host, once per mesh)
void build_level2_pattern(fe_mesh* m, cudaStream_t s) {
  Coarse& c = m->coarse;
  const int64_t N4 = c.n_nodes;
  const std::vector<int32_t>& rp = c.rowptr_host;
  const std::vector<int32_t>& cl = c.cols_host;
  FE_REQUIRE((int64_t)rp.size() == N4 + 1, "coarse pattern missing");
  std::vector<int32_t> agg((size_t)N4, -1);
  int64_t na = 0;
  for (int64_t n = 0; n < N4; ++n) {
    if (agg[(size_t)n] >= 0) continue;
    bool open = true;
    for (int32_t q = rp[(size_t)n]; q < rp[(size_t)n + 1] && open; ++q)
      if (cl[(size_t)q] != n && agg[(size_t)cl[(size_t)q]] >= 0) open = false;
    if (!open) continue;
    for (int32_t q = rp[(size_t)n]; q < rp[(size_t)n + 1]; ++q) agg[(size_t)cl[(size_t)q]] = (int32_t)na;
    agg[(size_t)n] = (int32_t)na;
    ++na;
  }
  const std::vector<int32_t> first = agg;
  for (int64_t n = 0; n < N4; ++n) {
    if (first[(size_t)n] >= 0) continue;
    int32_t best = -1;  // columns are sorted: the first aggregated neighbour is the lowest-numbered
    for (int32_t q = rp[(size_t)n]; q < rp[(size_t)n + 1]; ++q) {
      const int32_t j = cl[(size_t)q];
      if (j != n && first[(size_t)j] >= 0) {
        best = j;
        break;
      }
    }
    FE_REQUIRE(best >= 0, "aggregation: coarse node %lld has no aggregated neighbour", (long long)n);
    agg[(size_t)n] = first[(size_t)best];
  }
  // members of each aggregate, free-DOF bits
  std::vector<int32_t> mptr((size_t)na + 1, 0), members((size_t)N4);
  for (int64_t n = 0; n < N4; ++n) ++mptr[(size_t)agg[(size_t)n] + 1];
  for (int64_t A = 0; A < na; ++A) mptr[(size_t)A + 1] += mptr[(size_t)A];
  {
    std::vector<int32_t> fill(mptr.begin(), mptr.end() - 1);
    for (int64_t n = 0; n < N4; ++n) members[(size_t)fill[(size_t)agg[(size_t)n]]++] = (int32_t)n;
  }
  std::vector<uint8_t> mk2((size_t)na, 0);
  for (int64_t n = 0; n < N4; ++n) mk2[(size_t)agg[(size_t)n]] |= c.nmask4_host[(size_t)n];
  // A2 pattern: aggregates coupled by some K1 block; pos2 maps each K1 block to its A2 block
  std::vector<int32_t> rowptr2((size_t)na + 1, 0), cols2;
  std::vector<int32_t> pos2(cl.size());
  std::vector<int32_t> row;
  for (int64_t A = 0; A < na; ++A) {
    row.clear();
    for (int32_t k = mptr[(size_t)A]; k < mptr[(size_t)A + 1]; ++k) {
      const int32_t a = members[(size_t)k];
      for (int32_t q = rp[(size_t)a]; q < rp[(size_t)a + 1]; ++q) row.push_back(agg[(size_t)cl[(size_t)q]]);
    }
    std::sort(row.begin(), row.end());
    row.erase(std::unique(row.begin(), row.end()), row.end());
    const int32_t base = (int32_t)cols2.size();
    cols2.insert(cols2.end(), row.begin(), row.end());
    rowptr2[(size_t)A + 1] = (int32_t)cols2.size();
    for (int32_t k = mptr[(size_t)A]; k < mptr[(size_t)A + 1]; ++k) {
      const int32_t a = members[(size_t)k];
      for (int32_t q = rp[(size_t)a]; q < rp[(size_t)a + 1]; ++q) {
        const int32_t B = agg[(size_t)cl[(size_t)q]];
        pos2[(size_t)q] = base + (int32_t)(std::lower_bound(row.begin(), row.end(), B) - row.begin());
      }
    }
  }
  c.n_agg = na;
  c.nnzb2 = (int64_t)cols2.size();
  c.agg.alloc(agg.size() * 4);
  c.mptr.alloc(mptr.size() * 4);
  c.members.alloc(members.size() * 4);
  c.nmask2.alloc(std::max<size_t>(mk2.size(), 1));
  c.pos2.alloc(pos2.size() * 4);
  c.rowptr2.alloc(rowptr2.size() * 4);
  c.cols2.alloc(cols2.size() * 4);
  FE_CUDA(cudaMemcpyAsync(c.agg.ptr, agg.data(), agg.size() * 4, cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(c.mptr.ptr, mptr.data(), mptr.size() * 4, cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(c.members.ptr, members.data(), members.size() * 4, cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(c.nmask2.ptr, mk2.data(), mk2.size(), cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(c.pos2.ptr, pos2.data(), pos2.size() * 4, cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(c.rowptr2.ptr, rowptr2.data(), rowptr2.size() * 4, cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaMemcpyAsync(c.cols2.ptr, cols2.data(), cols2.size() * 4, cudaMemcpyHostToDevice, s));
  FE_CUDA(cudaStreamSynchronize(s));
  c.l2_pattern = true;
}

}  // namespace

size_t level2_bytes(const fe_mesh* m) {
  // an aggregate holds about 20 coarse nodes and couples about 27 aggregates
  const int64_t na = m->coarse.l2_pattern ? m->coarse.n_agg : m->coarse.n_nodes / 10 + 1;
  const int64_t nnz = m->coarse.l2_pattern ? m->coarse.nnzb2 : na * 40;
  return (size_t)m->coarse.nnzb * 4 + (size_t)nnz * 9 * (sizeof(double) + sizeof(float)) +
         (size_t)na * 9 * (sizeof(double) + sizeof(float)) + (size_t)m->coarse.n_nodes * 8;
}

void build_level2(fe_mesh* m, const double* k1_64, cudaStream_t s) {
  Coarse& c = m->coarse;
  if (!c.l2_pattern) build_level2_pattern(m, s);
  const int64_t NA = c.n_agg;
  DevBuf a2, bad;
  a2.alloc((size_t)c.nnzb2 * 9 * sizeof(double));
  bad.alloc(sizeof(int));
  if (!c.vals2_32.ptr) c.vals2_32.alloc((size_t)c.nnzb2 * 9 * sizeof(float));
  if (!c.binv2_64.ptr) c.binv2_64.alloc((size_t)NA * 9 * sizeof(double));
  if (!c.binv2_32.ptr) c.binv2_32.alloc((size_t)NA * 9 * sizeof(float));
  FE_CUDA(cudaMemsetAsync(a2.ptr, 0, a2.bytes, s));
  FE_CUDA(cudaMemsetAsync(bad.ptr, 0, sizeof(int), s));
  galerkin2_kernel<<<blocks_for(c.n_nodes), kThreads, 0, s>>>(c.n_nodes, c.rowptr.as<int32_t>(), c.cols.as<int32_t>(),
                                                              c.nmask4.as<uint8_t>(), c.pos2.as<int32_t>(), k1_64,
                                                              a2.as<double>());
  FE_CHECK_LAUNCH();
  finish2_kernel<<<blocks_for(NA), kThreads, 0, s>>>(NA, c.rowptr2.as<int32_t>(), c.cols2.as<int32_t>(),
                                                     c.nmask2.as<uint8_t>(), a2.as<double>(), c.vals2_32.as<float>(),
                                                     c.binv2_64.as<double>(), c.binv2_32.as<float>(), bad.as<int>());
  FE_CHECK_LAUNCH();
  int hbad = 0;
  FE_CUDA(cudaMemcpyAsync(&hbad, bad.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  FE_CUDA(cudaStreamSynchronize(s));
  FE_REQUIRE(hbad == 0, "level 2: an aggregate has a singular diagonal block");
  c.l2_ready = true;
}

void level2_restrict(const fe_mesh* m, int R, const float* r4, float* r2, cudaStream_t s, const int* skip) {
  const Coarse& c = m->coarse;
  FE_REQUIRE(c.l2_ready, "level 2 not built");
  restrict2_kernel<<<blocks_for(c.n_agg * R), kThreads, 0, s>>>(c.n_agg, R, c.mptr.as<int32_t>(),
                                                                c.members.as<int32_t>(), c.nmask4.as<uint8_t>(), r4,
                                                                r2, skip);
  FE_CHECK_LAUNCH();
}

void level2_prolong(const fe_mesh* m, int R, const float* u2, float* u4, cudaStream_t s, const int* skip) {
  const Coarse& c = m->coarse;
  FE_REQUIRE(c.l2_ready, "level 2 not built");
  prolong2_kernel<<<blocks_for(c.n_nodes * R), kThreads, 0, s>>>(c.n_nodes, R, c.agg.as<int32_t>(),
                                                                 c.nmask4.as<uint8_t>(), u2, u4, skip);
  FE_CHECK_LAUNCH();
}

}  // namespace fe

// ---------------------------------------------------------------------------
// C ABI of level 2
// ---------------------------------------------------------------------------
namespace {
fe_mesh* level2_ready(const fe_mesh* mesh, cudaStream_t s) {
  FE_REQUIRE(mesh != nullptr, "mesh is NULL");
  fe_mesh* m = const_cast<fe_mesh*>(mesh);
  FE_REQUIRE(fe::build_coarse_matrix(m, s, true), "not enough free device memory for the coarse matrices");
  return m;
}

void vec_args(int32_t R, const void* in, void* out) {
  FE_REQUIRE(in != nullptr && out != nullptr, "NULL argument");
  FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range [1, 64]", R);
  FE_REQUIRE(in != out, "input and output must not alias");
}
}  // namespace

extern "C" fe_status fe_level2_info(const fe_mesh* mesh, int64_t* n_agg, int32_t* agg_host, void* stream) {
  return fe::guarded([&] {
    FE_REQUIRE(mesh != nullptr, "mesh is NULL");
    fe::DeviceGuard dg(mesh->device);
    fe_mesh* m = level2_ready(mesh, (cudaStream_t)stream);
    if (n_agg) *n_agg = m->coarse.n_agg;
    if (agg_host) FE_CUDA(cudaMemcpy(agg_host, m->coarse.agg.ptr, m->coarse.agg.bytes, cudaMemcpyDeviceToHost));
  });
}

extern "C" fe_status fe_coarse_matrix_info(const fe_mesh* mesh, int64_t* n_blocks1, int64_t* n_blocks2,
                                           void* stream) {
  return fe::guarded([&] {
    FE_REQUIRE(mesh != nullptr, "mesh is NULL");
    fe::DeviceGuard dg(mesh->device);
    fe_mesh* m = level2_ready(mesh, (cudaStream_t)stream);
    if (n_blocks1) *n_blocks1 = m->coarse.nnzb;
    if (n_blocks2) *n_blocks2 = m->coarse.nnzb2;
  });
}

extern "C" fe_status fe_level2_apply(const fe_mesh* mesh, int32_t R, const float* x2, float* y2, void* stream) {
  return fe::guarded([&] {
    vec_args(R, x2, y2);
    FE_REQUIRE(mesh != nullptr, "mesh is NULL");
    fe::DeviceGuard dg(mesh->device);
    cudaStream_t s = (cudaStream_t)stream;
    fe_mesh* m = level2_ready(mesh, s);
    const fe::Coarse& c = m->coarse;
    fe::bcsr_spmv(c.n_agg, R, c.rowptr2.as<int32_t>(), c.cols2.as<int32_t>(), c.vals2_32.as<float>(), x2, y2, s,
                  nullptr);
  });
}

extern "C" fe_status fe_level2_restrict(const fe_mesh* mesh, int32_t R, const float* r4, float* r2, void* stream) {
  return fe::guarded([&] {
    vec_args(R, r4, r2);
    FE_REQUIRE(mesh != nullptr, "mesh is NULL");
    fe::DeviceGuard dg(mesh->device);
    cudaStream_t s = (cudaStream_t)stream;
    fe::level2_restrict(level2_ready(mesh, s), R, r4, r2, s);
  });
}

extern "C" fe_status fe_level2_prolong(const fe_mesh* mesh, int32_t R, const float* u2, float* u4, void* stream) {
  return fe::guarded([&] {
    vec_args(R, u2, u4);
    FE_REQUIRE(mesh != nullptr, "mesh is NULL");
    fe::DeviceGuard dg(mesh->device);
    cudaStream_t s = (cudaStream_t)stream;
    fe::level2_prolong(level2_ready(mesh, s), R, u2, u4, s);
  });
}

extern "C" fe_status fe_level2_block_jacobi(const fe_mesh* mesh, double* binv2_dev, void* stream) {
  return fe::guarded([&] {
    FE_REQUIRE(mesh != nullptr && binv2_dev != nullptr, "NULL argument");
    fe::DeviceGuard dg(mesh->device);
    cudaStream_t s = (cudaStream_t)stream;
    fe_mesh* m = level2_ready(mesh, s);
    FE_CUDA(cudaMemcpyAsync(binv2_dev, m->coarse.binv2_64.ptr, m->coarse.binv2_64.bytes, cudaMemcpyDeviceToDevice,
                            s));
  });
}
