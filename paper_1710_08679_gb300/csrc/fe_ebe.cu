// EBE product y = K_bc x for R cases (Eq. 3, multiple vectors of Sec. 3.1).
//
// Two kernels compute the same thing:
//  * EBE_DIRECT: one thread per (element, case). The thread recomputes the
//    element geometry, gathers its 30 inputs straight from global memory (the R
//    threads of one element read the node's 3R contiguous values together) and
//    scatters 30 results with atomic adds, as the paper's GPU port does
//    (Sec. 3.2.2: atomics keep node data local in L2 instead of colouring).
//  * EBE_TILED: elements are grouped into tiles whose nodes are staged in shared
//    memory. One CTA gathers the tile's input values once (coalesced, each node
//    contributing 3R contiguous values), computes every (element, case) product
//    of the tile from shared memory, accumulates them in shared memory and adds
//    each tile node's total to global memory once. This replaces ~10 global
//    atomics per element and case with ~(tile nodes / tile elements) of them.
// Both first write y = (I - P) x (constrained DOFs copy x, free DOFs start at
// zero) and only ever add into free DOFs, which yields P K P x + (I - P) x.
#include <algorithm>
#include <cstdio>

#include "fe_element.cuh"
#include "fe_internal.cuh"

namespace fe {

namespace {

constexpr int kThreads = 256;

// y = 0 with 16-byte stores (write-only pass before the atomic accumulation)
template <typename T>
__global__ void __launch_bounds__(kThreads) zero_kernel(int64_t n, T* __restrict__ y, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t n4 = n * (int64_t)sizeof(T) / 16;
  float4* y4 = reinterpret_cast<float4*>(y);
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += stride) y4[i] = z;
  // tail (n * sizeof(T) not a multiple of 16)
  for (int64_t i = n4 * 16 / (int64_t)sizeof(T) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = T(0);
}

template <typename T>
__device__ __forceinline__ void load_conn(const int32_t* __restrict__ conn, int64_t e, int nd[10]) {
  const int2* c2 = reinterpret_cast<const int2*>(conn + 10 * e);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int2 v = __ldg(c2 + q);
    nd[2 * q] = v.x;
    nd[2 * q + 1] = v.y;
  }
}

template <typename T>
__device__ __forceinline__ void load_geometry(const MeshView<T>& M, int64_t e, const int nd[10], ElemGeo<T>& G) {
  T xc[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) xc[k][i] = __ldg(M.xyz + 3 * (int64_t)nd[k] + i);
  elem_geometry(xc[0], xc[1], xc[2], xc[3], __ldg(M.mat + 2 * e), __ldg(M.mat + 2 * e + 1), G);
}

// ---------------------------------------------------------------------------
// direct kernel: thread = (element, case)
// ---------------------------------------------------------------------------
// FP32: at most 128 registers so that two 256-thread blocks fit per SM
template <typename T>
struct MinBlocks {
  static constexpr int value = sizeof(T) == 4 ? 2 : 1;
};

template <typename T>
__global__ void __launch_bounds__(kThreads, MinBlocks<T>::value) ebe_direct_kernel(MeshView<T> M, int R, const uint16_t* __restrict__ own,
                                                              const T* __restrict__ x, T* __restrict__ y,
                                                              const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= M.n_elem * R) return;
  const int64_t e = gid / R;
  const int r = (int)(gid - e * R);
  int nd[10];
  load_conn<T>(M.conn, e, nd);
  ElemGeo<T> G;
  load_geometry(M, e, nd, G);
  T u[10][3];
  int mk[10];
#pragma unroll
  for (int a = 0; a < 10; ++a) {
    mk[a] = __ldg(M.nmask + nd[a]);
    const T* xa = x + ((int64_t)nd[a] * R + r) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) u[a][c] = ((mk[a] >> c) & 1) ? __ldg(xa + c) : T(0);
  }
  T yl[10][3];
  elem_apply(G, u, yl);
  const int ow = __ldg(own + e);
#pragma unroll
  for (int a = 0; a < 10; ++a) {
    T* ya = y + ((int64_t)nd[a] * R + r) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if ((mk[a] >> c) & 1)
        atomicAdd(ya + c, yl[a][c]);
      else if ((ow >> a) & 1)   // constrained DOF: (I - P) x, written once by the node's owner element
        ya[c] = __ldg(x + ((int64_t)nd[a] * R + r) * 3 + c);
    }
  }
}

// ---------------------------------------------------------------------------
// tiled kernel: CTA = tile of elements. Shared memory holds the tile's node
// inputs and accumulated outputs as [local node][R][3], the element geometry
// (computed once per element, shared by its R case threads) and the local
// connectivity.
// ---------------------------------------------------------------------------
constexpr int kGeo = 16;   // per element: g[4][3], lam, mu, c (15 used)

template <typename T>
__global__ void __launch_bounds__(kThreads) ebe_tiled_kernel(MeshView<T> M, int R, int tile_elems,
                                                             const int32_t* __restrict__ node_ptr,
                                                             const int32_t* __restrict__ node_ids,
                                                             const uint8_t* __restrict__ node_own,
                                                             const uint16_t* __restrict__ lconn,
                                                             const T* __restrict__ x, T* __restrict__ y,
                                                             const int* __restrict__ skip) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (skip && *skip) return;
  const int64_t tile = blockIdx.x;
  const int nb = __ldg(node_ptr + tile);
  const int nn = __ldg(node_ptr + tile + 1) - nb;
  const int64_t e0 = tile * (int64_t)tile_elems;
  const int64_t rem = M.n_elem - e0;
  const int ne = rem < (int64_t)tile_elems ? (int)rem : tile_elems;
  const int vr = 3 * R;                                           // values per node
  T* xs = reinterpret_cast<T*>(smem_raw);                         // [nn][3R] masked inputs
  T* ys = xs + (size_t)nn * vr;                                   // [nn][3R] accumulated outputs
  T* geo = ys + (size_t)nn * vr;                                  // [ne][kGeo]
  uint16_t* lc = reinterpret_cast<uint16_t*>(geo + (size_t)tile_elems * kGeo);  // [ne][10]
  int* ids = reinterpret_cast<int*>(lc + (size_t)tile_elems * 10 + (tile_elems & 1) * 2);  // [nn]
  unsigned char* mks = reinterpret_cast<unsigned char*>(ids + nn);                        // [nn]
  unsigned char* own = mks + nn;                                                           // [nn]

  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const int g = __ldg(node_ids + nb + i);
    ids[i] = g;
    mks[i] = __ldg(M.nmask + g);
    own[i] = __ldg(node_own + nb + i);
  }
  for (int i = threadIdx.x; i < ne * 10; i += blockDim.x) lc[i] = __ldg(lconn + 10 * e0 + i);
  // element geometry, once per element
  for (int le = threadIdx.x; le < ne; le += blockDim.x) {
    int nd[10];
    load_conn<T>(M.conn, e0 + le, nd);
    ElemGeo<T> G;
    load_geometry(M, e0 + le, nd, G);
    T* gp = geo + le * kGeo;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) gp[3 * k + i] = G.g[k][i];
    gp[12] = G.lam;
    gp[13] = G.mu;
    gp[14] = G.c;
  }
  __syncthreads();
  // gather inputs: consecutive threads read consecutive values of one node's 3R run
  const int total = nn * vr;
  for (int k = threadIdx.x; k < total; k += blockDim.x) {
    const int ln = k / vr;
    const int w = k - ln * vr;
    const int c = w % 3;
    const T v = __ldg(x + (int64_t)ids[ln] * vr + w);
    xs[k] = ((mks[ln] >> c) & 1) ? v : T(0);
    ys[k] = T(0);
  }
  __syncthreads();

  const int items = ne * R;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int le = it / R;
    const int r = it - le * R;
    ElemGeo<T> G;
    const T* gp = geo + le * kGeo;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) G.g[k][i] = gp[3 * k + i];
    G.lam = gp[12];
    G.mu = gp[13];
    G.c = gp[14];
    int ln[10];
#pragma unroll
    for (int a = 0; a < 10; ++a) ln[a] = lc[10 * le + a];
    T u[10][3];
#pragma unroll
    for (int a = 0; a < 10; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) u[a][c] = xs[ln[a] * vr + 3 * r + c];
    T yl[10][3];
    elem_apply(G, u, yl);
#pragma unroll
    for (int a = 0; a < 10; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) atomicAdd(ys + ln[a] * vr + 3 * r + c, yl[a][c]);
  }
  __syncthreads();
  // one global add per tile node value (free DOFs); constrained DOFs: y = x,
  // stored once by the node's owner tile
  for (int k = threadIdx.x; k < total; k += blockDim.x) {
    const int lnn = k / vr;
    const int w = k - lnn * vr;
    const int c = w % 3;
    const int64_t gi = (int64_t)ids[lnn] * vr + w;
    if ((mks[lnn] >> c) & 1)
      atomicAdd(y + gi, ys[k]);
    else if (own[lnn])
      y[gi] = __ldg(x + gi);
  }
}

template <typename T>
size_t tiled_smem_bytes(int max_nodes, int tile_elems, int R) {
  size_t b = (size_t)max_nodes * 3 * R * sizeof(T) * 2 + (size_t)tile_elems * kGeo * sizeof(T) +
             (size_t)tile_elems * 10 * sizeof(uint16_t) + 4 + (size_t)max_nodes * (sizeof(int) + 2);
  return (b + 15) & ~size_t(15);
}

}  // namespace

template <typename T>
static void launch_direct(const fe_mesh* m, int R, const T* x, T* y, cudaStream_t s, const int* skip) {
  const MeshView<T> M = m->view<T>();
  const int64_t total = M.n_elem * R;
  const int64_t blocks = (total + kThreads - 1) / kThreads;
  ebe_direct_kernel<T><<<(unsigned)blocks, kThreads, 0, s>>>(M, R, m->own_elem.as<uint16_t>(), x, y, skip);
  FE_CHECK_LAUNCH();
}

static int max_smem_optin(int device) {
  int v = 0;
  FE_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  return v;
}

bool tiled_fits(const fe_mesh* m, int tile_elems, int R, int is_f32) {
  auto it = m->tilings.find(tile_elems);
  // before the tiling exists, bound its node count by 10 nodes per element
  const int nodes = it != m->tilings.end() ? it->second->max_nodes : 10 * tile_elems;
  const size_t smem =
      is_f32 ? tiled_smem_bytes<float>(nodes, tile_elems, R) : tiled_smem_bytes<double>(nodes, tile_elems, R);
  return smem <= (size_t)max_smem_optin(m->device);
}

template <typename T>
static void launch_tiled(const fe_mesh* m, const Tiling& t, int R, const T* x, T* y, cudaStream_t s,
                         const int* skip) {
  const size_t smem = tiled_smem_bytes<T>(t.max_nodes, t.tile_elems, R);
  FE_REQUIRE(smem <= (size_t)max_smem_optin(m->device), "tile of %d elements needs %zu B shared memory",
             t.tile_elems, smem);
  FE_CUDA(cudaFuncSetAttribute(ebe_tiled_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const MeshView<T> M = m->view<T>();
  ebe_tiled_kernel<T><<<(unsigned)t.n_tiles, kThreads, smem, s>>>(
      M, R, t.tile_elems, t.node_ptr.as<int32_t>(), t.node_ids.as<int32_t>(), t.node_own.as<uint8_t>(),
      t.lconn.as<uint16_t>(), x, y, skip);
  FE_CHECK_LAUNCH();
}

int ebe_get_variant(const fe_mesh* m, int R, int is_f32) {
  const int v = m->variant[is_f32 ? 1 : 0][R];
  return v < 0 ? 0 : v;
}

void ebe_set_variant(fe_mesh* m, int R, int is_f32, int variant) {
  m->variant[is_f32 ? 1 : 0][R] = (int16_t)variant;
}

template <typename T>
void ebe_apply(const fe_mesh* m, int R, const T* x, T* y, cudaStream_t s, const int* skip) {
  const int64_t nv = m->n_nodes * (int64_t)R * 3;
  int sms = 0;
  FE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
  const int64_t zb = (nv * (int64_t)sizeof(T) / 16 + kThreads - 1) / kThreads;
  zero_kernel<T><<<(unsigned)(zb < (int64_t)sms * 16 ? (zb > 0 ? zb : 1) : (int64_t)sms * 16), kThreads, 0, s>>>(
      nv, y, skip);
  FE_CHECK_LAUNCH();
  const int v = ebe_get_variant(m, R, sizeof(T) == 4);
  if (v > 0) {
    auto it = m->tilings.find(v);
    FE_REQUIRE(it != m->tilings.end(), "tiling of %d elements was not built", v);
    launch_tiled<T>(m, *it->second, R, x, y, s, skip);
    return;
  }
  launch_direct<T>(m, R, x, y, s, skip);
}

template void ebe_apply<float>(const fe_mesh*, int, const float*, float*, cudaStream_t, const int*);
template void ebe_apply<double>(const fe_mesh*, int, const double*, double*, cudaStream_t, const int*);

// Times each candidate kernel for (R, precision) on this mesh (scratch vectors
// of ones, 2 warm-up and 5 timed products each, CUDA events on `s`) and keeps
// the fastest. Candidates: direct, and tiled with 24..384 elements per tile
// where the tile's shared-memory footprint fits.
template <typename T>
static void tune(fe_mesh* m, int R, cudaStream_t s, int* best_variant, float* best_ms) {
  const size_t n = (size_t)m->n_nodes * R * 3;
  DevBuf xb, yb;
  xb.alloc(n * sizeof(T));
  yb.alloc(n * sizeof(T));
  FE_CUDA(cudaMemsetAsync(xb.ptr, 0, n * sizeof(T), s));
  cudaEvent_t e0, e1;
  FE_CUDA(cudaEventCreate(&e0));
  FE_CUDA(cudaEventCreate(&e1));
  std::vector<int> cands = {0};
  for (int te : {24, 48, 96, 192, 384})
    if (tiled_fits(m, te, R, sizeof(T) == 4)) cands.push_back(te);
  *best_variant = 0;
  *best_ms = 1e30f;
  const int old = m->variant[sizeof(T) == 4][R];
  for (int v : cands) {
    if (v > 0) {
      get_tiling(m, v, s);
      if (!tiled_fits(m, v, R, sizeof(T) == 4)) continue;
    }
    ebe_set_variant(m, R, sizeof(T) == 4, v);
    for (int i = 0; i < 2; ++i) ebe_apply<T>(m, R, xb.as<T>(), yb.as<T>(), s);
    FE_CUDA(cudaEventRecord(e0, s));
    for (int i = 0; i < 5; ++i) ebe_apply<T>(m, R, xb.as<T>(), yb.as<T>(), s);
    FE_CUDA(cudaEventRecord(e1, s));
    FE_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    FE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    ms /= 5.f;
    if (ms < *best_ms) {
      *best_ms = ms;
      *best_variant = v;
    }
  }
  m->variant[sizeof(T) == 4][R] = (int16_t)old;
  ebe_set_variant(m, R, sizeof(T) == 4, *best_variant);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

}  // namespace fe

// Picks the fastest EBE kernel for (R, dtype) on this mesh by timing (see tune()).
// Synchronous. *variant = 0 (direct) or the tile size of the tiled kernel;
// *us = its time per product in microseconds.
extern "C" fe_status fe_ebe_tune(fe_mesh* m, int32_t R, fe_dtype dtype, void* stream, int32_t* variant, int32_t* us) {
  try {
    fe::clear_error();
    FE_REQUIRE(m != nullptr, "mesh is NULL");
    FE_REQUIRE(R >= 1 && R <= 64, "R = %d out of range", R);
    fe::DeviceGuard dg(m->device);
    int v = 0;
    float ms = 0.f;
    if (dtype == FE_F32)
      fe::tune<float>(m, R, (cudaStream_t)stream, &v, &ms);
    else
      fe::tune<double>(m, R, (cudaStream_t)stream, &v, &ms);
    if (variant) *variant = v;
    if (us) *us = (int32_t)(ms * 1000.f);
    return FE_OK;
  } catch (const fe::Failure& f) {
    return f.status;
  } catch (...) {
    fe::set_error("unexpected C++ exception");
    return FE_EINVAL;
  }
}
